// Host-side launch entry points of the device kernels (one translation unit per
// polynomial order instantiates them; dispatch by N happens in kernels_common.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernel_types.hpp"

namespace swe {

// Per (precision, order) kernel configuration: shared-memory bytes of the
// operator block and the number of CTAs that fill the GPU once.
struct KernelCfg {
  int smem_bytes = 0;      // the whole operator block (SIMT stage kernel)
  int smem_lim = 0;        // the per-element operators (limiter kernels)
  int grid_stage = 0, grid_pos = 0, grid_tvb = 0, grid_stats = 0;
  int smem_tc = 0, grid_tc = 0;   // tensor-core stage kernel (FP32 only)
  int tc_warps = 4;               // warps per CTA of the tensor-core stage and batch kernels
  int grid_stage_g = 0;           // stage kernel with the operators in global memory
  int grid_split_t = 0, grid_split_v = 0, grid_split_s = 0;   // kernel-split ablation
  int smem_batch = 0, occ_batch = 0;         // persistent batch kernel, SIMT body
  int smem_batch_tc = 0, occ_batch_tc = 0;   // persistent batch kernel, tensor-core body (FP32)
};

template <typename T>
struct Launchers {
  cudaError_t (*prepare)(KernelCfg*);
  cudaError_t (*stage)(const StageParams<T>&, const KernelCfg&, cudaStream_t);
  cudaError_t (*stage_tc)(const StageParams<T>&, const KernelCfg&, cudaStream_t);  // nullptr for FP64
  cudaError_t (*positivity)(const LimitParams<T>&, const KernelCfg&, cudaStream_t);
  cudaError_t (*tvb)(const LimitParams<T>&, const KernelCfg&, cudaStream_t);
  cudaError_t (*stats)(const DevState<T>&, const Sched&, int nblocks, double* partials,
                       cudaStream_t);
  int op_size;  // elements of the operator block
  // Ablations of the fused stage kernel (R only, mode 1): the operators read from
  // global memory; the three-kernel split with stored face traces. qg holds
  // split_planes planes and rg 3 NP planes, each of stride KS.
  cudaError_t (*stage_global_ops)(const StageParams<T>&, const KernelCfg&, cudaStream_t);
  cudaError_t (*split_rhs)(const StageParams<T>&, T* qg, T* rg, const KernelCfg&, cudaStream_t);
  int split_planes;
  // Persistent batch kernel over a group of scenarios of this order (tc: the
  // tensor-core stage body, FP32 only), grid CTAs.
  cudaError_t (*batch)(const BatchLaunch<T>& bl, bool tc, int grid, const KernelCfg&, cudaStream_t);
  // Warps per CTA of the tensor-core kernels (FP32 only): sets tc_warps, their
  // shared memory and grids in cfg; cudaErrorInvalidValue when that many warps'
  // tiles do not fit on an SM.
  cudaError_t (*tc_config)(KernelCfg* cfg, int warps);
};

// Registered per order by kernels_n*.cu; nullptr when the order is not built.
template <typename T>
const Launchers<T>* launchers_for(int N);

cudaError_t launch_advance(long long* macro, cudaStream_t st);

// State transfer between the caller's layout ([3][K][Np] FP64, caller element
// order, depth h) and the device planes (eta = h + B in device precision, level
// order). x: staging copy of the caller arrays in device memory; Bc: the bed in
// caller order (FP64); iperm: caller index -> device index.
cudaError_t launch_check_finite(const double* x, size_t n, int* flag, cudaStream_t st);
template <typename T>
cudaError_t launch_pack_state(const double* x, const double* Bc, const int* iperm, int K, int KS, int Np,
                              T* q, cudaStream_t st);
// Reverse: each element's current buffer from its level, h = eta - (device-precision B).
template <typename T>
cudaError_t launch_unpack_state(const T* q, const double* Bc, const int* iperm, const Sched& sc,
                                long long k, int Np, double* x, cudaStream_t st);
cudaError_t launch_stats_finalize(const double* partials, int nblocks, double* out, cudaStream_t st);

// After a persistent batch kernel: advance the macro counters of the scenarios that
// completed by n_macro (device, per scenario).
template <typename T>
cudaError_t launch_batch_finish(const BatchLaunch<T>& bl, const int* n_macro, cudaStream_t st);

// Level regrouping on the device (re-interpolated history, then every per-element
// array gathered into the new order; pi: new index -> old index, sigma: old -> new).
// Per-element CFL step of Eq. cfl from the current state (device order); H: the
// inradii in device order; scratch: 8 bytes for the maximum depth.
template <typename T>
cudaError_t launch_element_dt(const T* q, const T* B, const Sched& sc, long long k, int NP, const double* H,
                              double g, double C, unsigned long long* scratch, double* dt, cudaStream_t st);
template <typename T>
cudaError_t launch_ring_reinterp(T* ring, int K, int KS, int NP, const uint8_t* lev_old, const uint8_t* lev_new,
                                 long long k, cudaStream_t st);
template <typename E>
cudaError_t launch_gather_planes(const E* src, E* dst, int P, int KS, int K, const int* pi, cudaStream_t st);
template <typename T>
cudaError_t launch_gather_state(const T* q, T* dst, int p0, int P, int KS, int K, int NP, const int* pi,
                                const uint8_t* lev_old, long long k, cudaStream_t st);
template <typename E>
cudaError_t launch_gather_rows(const E* src, E* dst, int W, int K, const int* pi, cudaStream_t st);
cudaError_t launch_remap_conn(const int4* src, int4* dst, int K, const int* pi, const int* sigma,
                              const uint8_t* lev_new, cudaStream_t st);

}  // namespace swe
