// Allocation-free mass / minimum-depth reduction over caller-owned device arrays.
//
// This is the reduction behind swe_stats, but its per-block partial sums live in
// a fixed array compiled into this library instead of a solver workspace, so the
// caller needs no device allocation of any kind: it passes the nodal depth, the
// element areas and a two-double output, all device memory it already owns.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/swe.h"
#include "refelem.hpp"

namespace swe {
void set_last_error(const std::string& msg);  // defined with the other entry points
}

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 1024;   // the scratch holds the partials of at most 1024 blocks
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device: 2 doubles (mass, hmin) per block,
// 16 KiB in total, resident on each GPU that loads the library until exit. Each
// call's first kernel writes every slot its second kernel reads, so nothing has
// to start at zero; calls whose kernels overlap on the GPU race on this array.
static __device__ __align__(256) double g_partials[2 * kMaxBlocks];

struct MeanWeights {
  double w[28];
};

// Minimum that keeps a NaN: fmin() returns the other operand when one is NaN, which
// would let a non-finite depth vanish from the minimum.
__device__ __forceinline__ double min_keep_nan(double a, double b) {
  return a != a ? a : (b != b ? b : fmin(a, b));
}

__global__ void __launch_bounds__(kThreads) k_mass_hmin_partials(const double* __restrict__ h,
                                                                 const double* __restrict__ area,
                                                                 int K, int np, MeanWeights mw,
                                                                 double* partials) {
  __shared__ double sm[kThreads];
  __shared__ double sh[kThreads];
  double mass = 0.0, hmin = 1e300;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K; e += gridDim.x * blockDim.x) {
    const double* he = h + (size_t)e * np;
    double hb = 0.0;
    for (int j = 0; j < np; ++j) {
      hb += mw.w[j] * he[j];
      hmin = min_keep_nan(hmin, he[j]);
    }
    mass += area[e] * hb;
  }
  sm[threadIdx.x] = mass;
  sh[threadIdx.x] = hmin;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sm[threadIdx.x] += sm[threadIdx.x + s];
      sh[threadIdx.x] = min_keep_nan(sh[threadIdx.x], sh[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = sm[0];
    partials[2 * blockIdx.x + 1] = sh[0];
  }
}

__global__ void __launch_bounds__(kThreads) k_mass_hmin_final(const double* partials, int nblocks,
                                                              double* out) {
  __shared__ double sm[kThreads];
  __shared__ double sh[kThreads];
  double m = 0.0, h = 1e300;
  for (int i = threadIdx.x; i < nblocks; i += kThreads) {
    m += partials[2 * i];
    h = min_keep_nan(h, partials[2 * i + 1]);
  }
  sm[threadIdx.x] = m;
  sh[threadIdx.x] = h;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sm[threadIdx.x] += sm[threadIdx.x + s];
      sh[threadIdx.x] = min_keep_nan(sh[threadIdx.x], sh[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sm[0];
    out[1] = sh[0];
  }
}

std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};   // device address of g_partials, per device
MeanWeights g_weights[6];                  // element-mean weights per order, built once
bool g_have_weights[6] = {};

int fail_na(int code, const std::string& msg) {
  swe::set_last_error(msg);
  return code;
}

}  // namespace

extern "C" int swe_mass_hmin_static(int32_t N, int32_t K, const double* dev_h, const double* dev_area,
                                    double* dev_out, void* stream) {
  if (N < 1 || N > 5) return fail_na(SWE_EINVAL, "swe_mass_hmin_static: N must be in 1..5");
  const int np = (N + 1) * (N + 2) / 2;
  if (K < 1 || (int64_t)K * np > INT32_MAX)
    return fail_na(SWE_EINVAL, "swe_mass_hmin_static: K must satisfy 1 <= K and K*Np <= 2^31-1");
  if (!dev_h || !dev_area || !dev_out) return fail_na(SWE_EINVAL, "swe_mass_hmin_static: NULL device pointer");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_na(SWE_ECUDA, std::string("swe_mass_hmin_static: cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail_na(SWE_EINVAL, "swe_mass_hmin_static: device index beyond 63");
  double* scratch;
  MeanWeights mw;
  {
    // once per device, with that device current: the host-side name g_partials is
    // only a stand-in, the kernels need its device address. The address belongs to
    // the context current at that first call (the device's primary context for a
    // runtime-API caller); it is not looked up again, so the call assumes that
    // context for the life of the process (no cudaDeviceReset in between).
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_partials);
      if (e != cudaSuccess || !p)
        return fail_na(SWE_ECUDA, std::string("swe_mass_hmin_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_ptr[dev];
    if (!g_have_weights[N]) {
      swe::RefElem ref = swe::RefElem::build(N);
      g_weights[N] = MeanWeights{};
      for (int j = 0; j < np; ++j) g_weights[N].w[j] = ref.mean_w[j];
      g_have_weights[N] = true;
    }
    mw = g_weights[N];
  }
  int nb = (K + kThreads - 1) / kThreads;
  if (nb > kMaxBlocks) nb = kMaxBlocks;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  k_mass_hmin_partials<<<nb, kThreads, 0, st>>>(dev_h, dev_area, K, np, mw, scratch);
  k_mass_hmin_final<<<1, kThreads, 0, st>>>(scratch, nb, dev_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail_na(SWE_ECUDA, std::string("swe_mass_hmin_static: launch: ") + cudaGetErrorString(e));
  return SWE_OK;
}
