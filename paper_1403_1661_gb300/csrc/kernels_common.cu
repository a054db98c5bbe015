// Order dispatch and the small order-independent kernels.
#include "kernels.cuh"
#include "launch.hpp"

namespace swe {

const Launchers<float>* launchers_f32_n1();
const Launchers<float>* launchers_f32_n2();
const Launchers<float>* launchers_f32_n3();
const Launchers<float>* launchers_f32_n4();
const Launchers<float>* launchers_f32_n5();
const Launchers<double>* launchers_f64_n1();
const Launchers<double>* launchers_f64_n2();
const Launchers<double>* launchers_f64_n3();
const Launchers<double>* launchers_f64_n4();
const Launchers<double>* launchers_f64_n5();
const Launchers<float>* launchers_f32_n18();
const Launchers<float>* launchers_f32_n19();
const Launchers<float>* launchers_f32_n20();
const Launchers<float>* launchers_f32_n21();
const Launchers<float>* launchers_f32_n34();
const Launchers<float>* launchers_f32_n35();
const Launchers<float>* launchers_f32_n36();
const Launchers<float>* launchers_f32_n37();
const Launchers<double>* launchers_f64_n18();
const Launchers<double>* launchers_f64_n19();
const Launchers<double>* launchers_f64_n20();
const Launchers<double>* launchers_f64_n21();
const Launchers<double>* launchers_f64_n34();
const Launchers<double>* launchers_f64_n35();
const Launchers<double>* launchers_f64_n36();
const Launchers<double>* launchers_f64_n37();

template <>
const Launchers<float>* launchers_for<float>(int N) {
  switch (N) {
    case 1: return launchers_f32_n1();
    case 2: return launchers_f32_n2();
    case 3: return launchers_f32_n3();
    case 4: return launchers_f32_n4();
    case 5: return launchers_f32_n5();
    case kColloc + 2: return launchers_f32_n18();
    case kColloc + 3: return launchers_f32_n19();
    case kColloc + 4: return launchers_f32_n20();
    case kColloc + 5: return launchers_f32_n21();
    case kReduced + 2: return launchers_f32_n34();
    case kReduced + 3: return launchers_f32_n35();
    case kReduced + 4: return launchers_f32_n36();
    case kReduced + 5: return launchers_f32_n37();
    default: return nullptr;
  }
}

template <>
const Launchers<double>* launchers_for<double>(int N) {
  switch (N) {
    case 1: return launchers_f64_n1();
    case 2: return launchers_f64_n2();
    case 3: return launchers_f64_n3();
    case 4: return launchers_f64_n4();
    case 5: return launchers_f64_n5();
    case kColloc + 2: return launchers_f64_n18();
    case kColloc + 3: return launchers_f64_n19();
    case kColloc + 4: return launchers_f64_n20();
    case kColloc + 5: return launchers_f64_n21();
    case kReduced + 2: return launchers_f64_n34();
    case kReduced + 3: return launchers_f64_n35();
    case kReduced + 4: return launchers_f64_n36();
    case kReduced + 5: return launchers_f64_n37();
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

// ---- level regrouping on the device ----------------------------------------

// max over all nodes of the depth h = eta - B (FP64 from the device values),
// clamped at 0: non-negative doubles order like their bit patterns
template <typename T>
__global__ void k_depth_max(const T* __restrict__ q, const T* __restrict__ B, Sched sc, long long k, int NP,
                            unsigned long long* out) {
  const int K = sc.K;
  const size_t fs = (size_t)NP * sc.KS, bs = 3 * fs, n = (size_t)K * NP;
  double m = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int e = (int)(i % K), j = (int)(i / K);
    const int cur = (int)((k >> (level_of(sc, e) - 1)) & 1);
    const size_t o = (size_t)j * sc.KS + e;
    m = fmax(m, (double)q[cur * bs + o] - (double)B[o]);
  }
  for (int d = 16; d > 0; d >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, d));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// dt_k = C H_k / a_k (Eq. cfl), a_k = max over the nodes of |u| + sqrt(g max(h, href)),
// href = 1e-2 max h, u = hu/h where h > href; H_k the inradius (device order)
template <typename T>
__global__ void k_element_dt(const T* __restrict__ q, const T* __restrict__ B, Sched sc, long long k, int NP,
                             const unsigned long long* hmax_bits, const double* __restrict__ H, double g, double C,
                             double* __restrict__ dt) {
  const size_t fs = (size_t)NP * sc.KS, bs = 3 * fs;
  const double href = 1e-2 * __longlong_as_double((long long)*hmax_bits);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < sc.K; e += gridDim.x * blockDim.x) {
    const int cur = (int)((k >> (level_of(sc, e) - 1)) & 1);
    const T* qe = q + cur * bs + e;
    double amax = 0.0;
    for (int j = 0; j < NP; ++j) {
      const size_t o = (size_t)j * sc.KS;
      const double h = (double)qe[o] - (double)B[o + e];
      const double hh = fmax(h, href);
      double u = 0.0, v = 0.0;
      if (h > href) {
        u = (double)qe[fs + o] / h;
        v = (double)qe[2 * fs + o] / h;
      }
      amax = fmax(amax, hypot(u, v) + sqrt(g * hh));
    }
    dt[e] = C * H[e] / amax;
  }
}

__device__ __forceinline__ int ring_slot(long long a) { return (int)(((a % 3) + 3) % 3); }

// In the old order, in place: an element moved from level l0 to l1 gets R at
// t_k - s dt_l1 (s = 1, 2, 3) from the quadratic through its R at t_k - s dt_l0
// (ring slot of activation a: a mod 3, a = k >> (level - 1)).
template <typename T>
__global__ void k_ring_reinterp(T* ring, int K, int KS, int NP, const uint8_t* lev_old, const uint8_t* lev_new,
                                long long k) {
  const size_t fs = (size_t)NP * KS, bs = 3 * fs, n = (size_t)K * NP;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int e = (int)(i % K), j = (int)(i / K);
    const int l0 = lev_old[e], l1 = lev_new[e];
    if (l0 == l1) continue;
    const long long a0 = k >> (l0 - 1), a1 = k >> (l1 - 1);
    const double r = ldexp(1.0, l1 - l0);
    for (int f = 0; f < 3; ++f) {
      const size_t o = f * fs + (size_t)j * KS + e;
      const double H0 = (double)ring[ring_slot(a0 - 1) * bs + o];
      const double H1 = (double)ring[ring_slot(a0 - 2) * bs + o];
      const double H2 = (double)ring[ring_slot(a0 - 3) * bs + o];
      for (int sn = 1; sn <= 3; ++sn) {
        const double x = -sn * r;   // Lagrange weights of tau = -1, -2, -3 at x
        const double w0 = (x + 2) * (x + 3) / 2.0, w1 = -(x + 1) * (x + 3), w2 = (x + 1) * (x + 2) / 2.0;
        ring[ring_slot(a1 - sn) * bs + o] = (T)(w0 * H0 + w1 * H1 + w2 * H2);
      }
    }
  }
}

// dst[p][e] = src[p][pi[e]] for P planes of stride KS (pi: new index -> old index)
template <typename E>
__global__ void k_gather_planes(const E* __restrict__ src, E* __restrict__ dst, int P, int KS, int K,
                                const int* __restrict__ pi) {
  const size_t n = (size_t)P * K;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(i / K), e = (int)(i % K);
    dst[(size_t)p * KS + e] = src[(size_t)p * KS + pi[e]];
  }
}

// planes p0 .. p0+P-1 of the (field, node) planes of each element's current buffer
template <typename T>
__global__ void k_gather_state(const T* __restrict__ q, T* __restrict__ dst, int p0, int P, int KS, int K, int NP,
                               const int* __restrict__ pi, const uint8_t* __restrict__ lev_old, long long k) {
  const size_t bs = (size_t)3 * NP * KS, n = (size_t)P * K;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(i / K), e = (int)(i % K);
    const int eo = pi[e];
    const int cur = (int)((k >> (lev_old[eo] - 1)) & 1);
    dst[(size_t)p * KS + e] = q[cur * bs + (size_t)(p0 + p) * KS + eo];
  }
}

// dst[e][w] = src[pi[e]][w] for records of W values
template <typename E>
__global__ void k_gather_rows(const E* __restrict__ src, E* __restrict__ dst, int W, int K,
                              const int* __restrict__ pi) {
  const size_t n = (size_t)W * K;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int e = (int)(i / W), w = (int)(i % W);
    dst[i] = src[(size_t)pi[e] * W + w];
  }
}

// connectivity in the new order: neighbours renumbered, "has a finer neighbour"
// (bit 12 of .w) recomputed from the new levels
__global__ void k_remap_conn(const int4* __restrict__ src, int4* __restrict__ dst, int K, const int* __restrict__ pi,
                             const int* __restrict__ sigma, const uint8_t* __restrict__ lev_new) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K; e += gridDim.x * blockDim.x) {
    int4 c = src[pi[e]];
    int nb[3] = {c.x, c.y, c.z};
    int w = c.w & ~(1 << 12);
    for (int f = 0; f < 3; ++f) {
      if (nb[f] < 0) continue;
      nb[f] = sigma[nb[f]];
      if (lev_new[nb[f]] < lev_new[e]) w |= 1 << 12;
    }
    dst[e] = make_int4(nb[0], nb[1], nb[2], w);
  }
}

}  // namespace

template <typename T>
cudaError_t launch_element_dt(const T* q, const T* B, const Sched& sc, long long k, int NP, const double* H,
                              double g, double C, unsigned long long* scratch, double* dt, cudaStream_t st) {
  cudaError_t err = cudaMemsetAsync(scratch, 0, 8, st);
  if (err) return err;
  k_depth_max<T><<<grid_elems((size_t)sc.K * NP), 256, 0, st>>>(q, B, sc, k, NP, scratch);
  k_element_dt<T><<<grid_elems((size_t)sc.K), 256, 0, st>>>(q, B, sc, k, NP, scratch, H, g, C, dt);
  return cudaGetLastError();
}

template cudaError_t launch_element_dt<float>(const float*, const float*, const Sched&, long long, int,
                                              const double*, double, double, unsigned long long*, double*,
                                              cudaStream_t);
template cudaError_t launch_element_dt<double>(const double*, const double*, const Sched&, long long, int,
                                               const double*, double, double, unsigned long long*, double*,
                                               cudaStream_t);

template <typename T>
cudaError_t launch_ring_reinterp(T* ring, int K, int KS, int NP, const uint8_t* lev_old, const uint8_t* lev_new,
                                 long long k, cudaStream_t st) {
  k_ring_reinterp<T><<<grid_elems((size_t)K * NP), 256, 0, st>>>(ring, K, KS, NP, lev_old, lev_new, k);
  return cudaGetLastError();
}

template <typename E>
cudaError_t launch_gather_planes(const E* src, E* dst, int P, int KS, int K, const int* pi, cudaStream_t st) {
  k_gather_planes<E><<<grid_elems((size_t)P * K), 256, 0, st>>>(src, dst, P, KS, K, pi);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather_state(const T* q, T* dst, int p0, int P, int KS, int K, int NP, const int* pi,
                                const uint8_t* lev_old, long long k, cudaStream_t st) {
  k_gather_state<T><<<grid_elems((size_t)P * K), 256, 0, st>>>(q, dst, p0, P, KS, K, NP, pi, lev_old, k);
  return cudaGetLastError();
}

template <typename E>
cudaError_t launch_gather_rows(const E* src, E* dst, int W, int K, const int* pi, cudaStream_t st) {
  k_gather_rows<E><<<grid_elems((size_t)W * K), 256, 0, st>>>(src, dst, W, K, pi);
  return cudaGetLastError();
}

cudaError_t launch_remap_conn(const int4* src, int4* dst, int K, const int* pi, const int* sigma,
                              const uint8_t* lev_new, cudaStream_t st) {
  k_remap_conn<<<grid_elems((size_t)K), 256, 0, st>>>(src, dst, K, pi, sigma, lev_new);
  return cudaGetLastError();
}

template cudaError_t launch_ring_reinterp<float>(float*, int, int, int, const uint8_t*, const uint8_t*, long long,
                                                 cudaStream_t);
template cudaError_t launch_ring_reinterp<double>(double*, int, int, int, const uint8_t*, const uint8_t*, long long,
                                                  cudaStream_t);
template cudaError_t launch_gather_planes<float>(const float*, float*, int, int, int, const int*, cudaStream_t);
template cudaError_t launch_gather_planes<double>(const double*, double*, int, int, int, const int*, cudaStream_t);
template cudaError_t launch_gather_state<float>(const float*, float*, int, int, int, int, int, const int*,
                                                const uint8_t*, long long, cudaStream_t);
template cudaError_t launch_gather_state<double>(const double*, double*, int, int, int, int, int, const int*,
                                                 const uint8_t*, long long, cudaStream_t);
template cudaError_t launch_gather_rows<float>(const float*, float*, int, int, const int*, cudaStream_t);
template cudaError_t launch_gather_rows<double>(const double*, double*, int, int, const int*, cudaStream_t);
template cudaError_t launch_gather_rows<uint8_t>(const uint8_t*, uint8_t*, int, int, const int*, cudaStream_t);

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

// After a persistent batch kernel: the macro counters of the scenarios that
// completed advance by their macro steps of the call.
template <typename T>
__global__ void k_batch_finish(const __grid_constant__ BatchLaunch<T> bl, const int* n_macro) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < bl.nscn && bl.status[i] == 0) *bl.scn[i].s.macro += n_macro[i];
}

template <typename T>
cudaError_t launch_batch_finish(const BatchLaunch<T>& bl, const int* n_macro, cudaStream_t st) {
  k_batch_finish<T><<<1, kBatchMaxScn, 0, st>>>(bl, n_macro);
  return cudaGetLastError();
}

template cudaError_t launch_batch_finish<float>(const BatchLaunch<float>&, const int*, cudaStream_t);
template cudaError_t launch_batch_finish<double>(const BatchLaunch<double>&, const int*, cudaStream_t);

}  // namespace swe
