// Order dispatch and the small order-independent kernels.
#include "kernels.cuh"
#include "launch.hpp"

namespace swe {

const Launchers<float>* launchers_f32_n2();
const Launchers<float>* launchers_f32_n3();
const Launchers<float>* launchers_f32_n4();
const Launchers<float>* launchers_f32_n5();
const Launchers<double>* launchers_f64_n2();
const Launchers<double>* launchers_f64_n3();
const Launchers<double>* launchers_f64_n4();
const Launchers<double>* launchers_f64_n5();

template <>
const Launchers<float>* launchers_for<float>(int N) {
  switch (N) {
    case 2: return launchers_f32_n2();
    case 3: return launchers_f32_n3();
    case 4: return launchers_f32_n4();
    case 5: return launchers_f32_n5();
    default: return nullptr;
  }
}

template <>
const Launchers<double>* launchers_for<double>(int N) {
  switch (N) {
    case 2: return launchers_f64_n2();
    case 3: return launchers_f64_n3();
    case 4: return launchers_f64_n4();
    case 5: return launchers_f64_n5();
    default: return nullptr;
  }
}

namespace {

__global__ void k_advance(long long* macro) { *macro += 1; }

__global__ void k_stats_finalize(const double* partials, int nblocks, double* out) {
  __shared__ double sm[256];
  __shared__ double sh[256];
  double m = 0.0, h = 1e300;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
    m += partials[2 * i];
    h = fmin(h, partials[2 * i + 1]);
  }
  sm[threadIdx.x] = m;
  sh[threadIdx.x] = h;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sm[threadIdx.x] += sm[threadIdx.x + w];
      sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sm[0];
    out[1] = sh[0];
  }
}

}  // namespace

cudaError_t launch_advance(long long* macro, cudaStream_t st) {
  k_advance<<<1, 1, 0, st>>>(macro);
  return cudaGetLastError();
}

cudaError_t launch_stats_finalize(const double* partials, int nblocks, double* out, cudaStream_t st) {
  k_stats_finalize<<<1, 256, 0, st>>>(partials, nblocks, out);
  return cudaGetLastError();
}

}  // namespace swe
