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
const Launchers<float>* launchers_f32_n18();
const Launchers<float>* launchers_f32_n19();
const Launchers<float>* launchers_f32_n20();
const Launchers<float>* launchers_f32_n21();
const Launchers<double>* launchers_f64_n18();
const Launchers<double>* launchers_f64_n19();
const Launchers<double>* launchers_f64_n20();
const Launchers<double>* launchers_f64_n21();

template <>
const Launchers<float>* launchers_for<float>(int N) {
  switch (N) {
    case 2: return launchers_f32_n2();
    case 3: return launchers_f32_n3();
    case 4: return launchers_f32_n4();
    case 5: return launchers_f32_n5();
    case kColloc + 2: return launchers_f32_n18();
    case kColloc + 3: return launchers_f32_n19();
    case kColloc + 4: return launchers_f32_n20();
    case kColloc + 5: return launchers_f32_n21();
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
    case kColloc + 2: return launchers_f64_n18();
    case kColloc + 3: return launchers_f64_n19();
    case kColloc + 4: return launchers_f64_n20();
    case kColloc + 5: return launchers_f64_n21();
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

__global__ void k_check_finite(const double* __restrict__ x, size_t n, int* flag) {
  bool bad = false;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    bad |= !isfinite(x[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

// one thread per (caller element c, node j): coalesced FP64 reads of the
// caller's layout, writes to the node planes of device element iperm[c]
template <typename T>
__global__ void k_pack_state(const double* __restrict__ x, const double* __restrict__ Bc,
                             const int* __restrict__ iperm, int K, int KS, int Np, T* __restrict__ q) {
  const size_t n = (size_t)K * Np, fs = (size_t)Np * KS;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i / Np), j = (int)(i % Np);
    const size_t d = (size_t)j * KS + __ldg(iperm + c);
    q[d] = (T)(x[i] + Bc[i]);
    q[fs + d] = (T)x[n + i];
    q[2 * fs + d] = (T)x[2 * n + i];
  }
}

template <typename T>
__global__ void k_unpack_state(const T* __restrict__ q, const double* __restrict__ Bc,
                               const int* __restrict__ iperm, Sched sc, long long k, int Np,
                               double* __restrict__ x) {
  const int K = sc.K;
  const size_t n = (size_t)K * Np, fs = (size_t)Np * sc.KS, bs = 3 * fs;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i / Np), j = (int)(i % Np);
    const int e = __ldg(iperm + c);
    const int cur = (int)((k >> (level_of(sc, e) - 1)) & 1);
    const size_t d = (size_t)cur * bs + (size_t)j * sc.KS + e;
    x[i] = (double)q[d] - (double)(T)Bc[i];
    x[n + i] = (double)q[fs + d];
    x[2 * n + i] = (double)q[2 * fs + d];
  }
}

int grid_elems(size_t n) {
  const size_t b = (n + 255) / 256;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

cudaError_t launch_check_finite(const double* x, size_t n, int* flag, cudaStream_t st) {
  k_check_finite<<<grid_elems(n), 256, 0, st>>>(x, n, flag);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pack_state(const double* x, const double* Bc, const int* iperm, int K, int KS, int Np,
                              T* q, cudaStream_t st) {
  k_pack_state<T><<<grid_elems((size_t)K * Np), 256, 0, st>>>(x, Bc, iperm, K, KS, Np, q);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_unpack_state(const T* q, const double* Bc, const int* iperm, const Sched& sc, long long k,
                                int Np, double* x, cudaStream_t st) {
  k_unpack_state<T><<<grid_elems((size_t)sc.K * Np), 256, 0, st>>>(q, Bc, iperm, sc, k, Np, x);
  return cudaGetLastError();
}

template cudaError_t launch_pack_state<float>(const double*, const double*, const int*, int, int, int, float*,
                                              cudaStream_t);
template cudaError_t launch_pack_state<double>(const double*, const double*, const int*, int, int, int, double*,
                                               cudaStream_t);
template cudaError_t launch_unpack_state<float>(const float*, const double*, const int*, const Sched&, long long,
                                                int, double*, cudaStream_t);
template cudaError_t launch_unpack_state<double>(const double*, const double*, const int*, const Sched&, long long,
                                                 int, double*, cudaStream_t);

cudaError_t launch_advance(long long* macro, cudaStream_t st) {
  k_advance<<<1, 1, 0, st>>>(macro);
  return cudaGetLastError();
}

cudaError_t launch_stats_finalize(const double* partials, int nblocks, double* out, cudaStream_t st) {
  k_stats_finalize<<<1, 256, 0, st>>>(partials, nblocks, out);
  return cudaGetLastError();
}

}  // namespace swe
