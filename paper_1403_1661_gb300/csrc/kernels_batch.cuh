// Persistent batched launch: many scenarios of one (tier, scheme and order) group
// advanced by one kernel that takes its work from a device ticket queue.
//
// A ticket is one tile of elements (kBatchStageTile for the stage kernel: R,
// Adams-Bashforth commit and positivity limiter, Algorithms 1 and 3; kBatchTvbTile
// for the TVB limiter, Section 5.3) of one phase of one scenario, a phase being one
// of those two kernels at one finest substep of the scenario's multirate schedule.
// Tickets are ordered phase by phase, round-robin over the scenarios (the host builds
// the segment table), and a ticket runs only after every tile of its scenario's
// earlier phases has completed, since a neighbour of any element may sit in any tile.
// Every wait is bounded in time: a scenario whose wait gives up is marked
// SWE_ETIMEOUT in its status word and the rest of its tickets are skipped, while the
// other scenarios carry on. The first phase of a scenario also waits for its release
// flag, which the host sets for every scenario it does not hold back.
//
// Memory ordering: a CTA that finishes a tile makes its stores visible (a
// device-scope fence in every thread, then a barrier) before it adds to its
// scenario's counter; a CTA that
// waits reads the counter with acquire semantics, then the arrays other CTAs wrote
// with ordinary (coherent) loads, never through the read-only data path.
#pragma once

#include <cstddef>

#include "kernels.cuh"
#include "kernels_tc.cuh"

namespace swe {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 of the CTA: wait until ticket segment S may run. Returns 1 to run the
// tile, 0 to skip it (its scenario failed, or this wait gave up and failed it).
template <typename T>
__device__ __forceinline__ int batch_wait(const BatchLaunch<T>& bl, const BatchSeg& S) {
  const int i = S.scn;
  if (ld_acquire(bl.status + i) != 0) return 0;
  const unsigned long long limit = (unsigned long long)__ldcg(&bl.ctl->wait_ns);
  const unsigned long long t0 = global_ns();
  if (S.first) {
    while (ld_acquire(bl.release + i) == 0) {
      if (global_ns() - t0 > limit) {
        atomicCAS(bl.status + i, 0, -5 /* SWE_ETIMEOUT */);
        return 0;
      }
      __nanosleep(256);
    }
  }
  while (ld_acquire(bl.done + i) < S.need) {
    if (ld_acquire(bl.status + i) != 0) return 0;
    if (global_ns() - t0 > limit) {
      atomicCAS(bl.status + i, 0, -5 /* SWE_ETIMEOUT */);
      return 0;
    }
    __nanosleep(64);
  }
  return 1;
}

// kTC: the tensor-core stage body (FP32 tier); otherwise the SIMT body (T = float
// or double). The CTA has kBatchTile threads: four warps with two warp-tiles of 32
// elements each per stage ticket for the tensor-core body, elements strided over
// the threads for the SIMT body and the TVB limiter.
template <typename T, int N, bool kTC>
__global__ void __launch_bounds__(kBatchTile, kTC ? 2 : 1) k_batch(const __grid_constant__ BatchLaunch<T> bl) {
  static_assert(kBatchTile == kTcBlock && kBatchStageTile % (32 * kTcWarps) == 0,
                "a tensor-core stage ticket is a whole number of warp-tiles per warp of the CTA");
  static_assert(sizeof(BatchLaunch<T>) <= 32000, "batch launch parameters exceed the kernel-parameter space");
  static_assert(offsetof(StageParams<T>, s) == offsetof(BatchScn<T>, s) &&
                    offsetof(StageParams<T>, sc) == offsetof(BatchScn<T>, sc) &&
                    offsetof(StageParams<T>, ph) == offsetof(BatchScn<T>, ph) &&
                    offsetof(LimitParams<T>, ph) == offsetof(BatchScn<T>, ph),
                "StageParams and LimitParams begin with the members of BatchScn");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ StageParams<T> s_p;
  __shared__ LimitParams<T> s_lp;
  __shared__ int s_seg, s_tile, s_go;
  T* sops = reinterpret_cast<T*>(smem_raw);
  // every scenario of the group has the same operators: stage the first one's
  if constexpr (kTC) {
    stage_ops<T, N, TcSmem<N>::OPS>(sops, bl.scn[0].s.ops);
  } else {
    stage_ops<T, N>(sops, bl.scn[0].s.ops);
  }
  const int total = __ldcg(&bl.ctl->total);
  // thread 0 takes the next ticket and looks up its segment while the CTA works on
  // the current one, so that the atomic and the lookups do not stall the CTA
  int ticket = 0, next_sg = -1;
  if (threadIdx.x == 0) {
    ticket = atomicAdd(&bl.ctl->head, 1);
    if (ticket < total) next_sg = __ldcg(bl.seg_of + ticket);
  }
  for (;;) {
    if (threadIdx.x == 0) {
      int sg = -1, tile = 0, go = 0;
      if (ticket < total) {
        sg = next_sg;
        tile = ticket - __ldcg(&bl.segs[sg].t0);
        go = batch_wait(bl, bl.segs[sg]);
        ticket = atomicAdd(&bl.ctl->head, 1);
        if (ticket < total) next_sg = __ldcg(bl.seg_of + ticket);
      }
      s_seg = sg;
      s_tile = tile;
      s_go = go;
    }
    __syncthreads();
    const int sg = s_seg;
    if (sg < 0) break;
    const BatchSeg S = bl.segs[sg];
    if (s_go) {
      // the scenario's parameters: StageParams and LimitParams begin with the
      // members of BatchScn (DevState, Sched, Phys), copied a word per thread
      {
        static_assert(sizeof(BatchScn<T>) % 4 == 0, "word copy");
        const int* src = reinterpret_cast<const int*>(&bl.scn[S.scn]);
        int* dp = reinterpret_cast<int*>(&s_p);
        int* dl = reinterpret_cast<int*>(&s_lp);
        for (int w = threadIdx.x; w < (int)(sizeof(BatchScn<T>) / 4); w += blockDim.x) {
          const int v = src[w];
          dp[w] = v;
          dl[w] = v;
        }
      }
      if (threadIdx.x == 0) {
        s_p.j = S.j;
        s_p.nactive = S.nactive;
        s_p.mode = 0;
        s_p.out = nullptr;
        s_p.perm = nullptr;
        s_lp.j = S.j;
        s_lp.nactive = S.nactive;
        s_lp.post_stage = 1;
      }
      __syncthreads();
      // the substep count: the scenario's macro counter (advanced only after the
      // launch) times its period, plus the phase's offset in this call
      const long long k = __ldcg(s_p.s.macro) * (long long)bl.period[S.scn] + S.kofs;
      // the same out-of-line bodies as the separate launches, over this ticket's tile
      double injected = 0.0;
      if (S.kind == 0) {
        if constexpr (kTC) {
          // warp w takes warp-tiles t0 + w and t0 + w + 4 of the ticket's eight,
          // prefetching the second while it works on the first
          const int warp = threadIdx.x >> 5;
          float* sw = sops + TcSmem<N>::OPS + warp * TcSmem<N>::WARP;
          const int t0 = s_tile * (kBatchStageTile / 32);
          injected = stage_tc_range<N>(s_p, k, sops, sw, t0 + warp, kTcWarps,
                                       min(t0 + kBatchStageTile / 32, (S.nactive + 31) / 32), true);
        } else {
          const int e0 = s_tile * kBatchStageTile;
          injected = stage_range<T, N>(s_p, sops, e0 + threadIdx.x, kBatchTile,
                                       min(e0 + kBatchStageTile, S.nactive), k);
        }
      } else {
        const int e0 = s_tile * kBatchTvbTile;
        tvb_range<T, N>(s_lp, sops, e0 + threadIdx.x, kBatchTile, min(e0 + kBatchTvbTile, S.nactive), k);
      }
      if (injected != 0.0) atomicAdd(s_p.s.acc, injected);
    }
    __threadfence();   // this thread's stores of the tile are visible device-wide
    __syncthreads();
    if (threadIdx.x == 0) {
      if (s_go) atomicAdd(bl.ran + S.scn, 1);
      atomicAdd(bl.done + S.scn, 1);
    }
  }
}

}  // namespace swe
