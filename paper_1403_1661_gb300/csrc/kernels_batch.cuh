// Persistent batched launch: many scenarios of one (tier, scheme and order) group
// advanced by one kernel that takes its work from a device ticket queue.
//
// A ticket, taken by one warp, is one tile of elements (kBatchStageTile for the stage kernel: R,
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
// Memory ordering: a warp that finishes a tile orders its lanes' stores before its
// counter update with a warp barrier followed by a device-scope fence in the lane
// that updates the counter (cumulative over what the barrier ordered, the pattern of
// a grid-wide barrier); a warp that
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

// L2 prefetch of the node planes of the state and the bed of elements [e0, e0 + n)
// of a scenario at substep k (the buffer each element reads: the parity of its
// level's activation count), one 128-byte line per lane and plane. Hints only:
// every address lies inside its array.
template <typename T, int N>
__device__ __forceinline__ void batch_prefetch_stage(const StageParams<T>& B, long long k, int e0, int n, int lane) {
  constexpr int NP = Dims<N>::NP;
  const size_t ks = (size_t)B.sc.KS, fstride = (size_t)NP * ks;
  const long long a = k >> (level_of(B.sc, e0) - 1);
  const T* q = B.s.q + (size_t)(a & 1) * 3 * fstride + e0;
  constexpr int per_line = 128 / sizeof(T);
  const int lines = (n + per_line - 1) / per_line;
  for (int w = lane; w < 4 * NP * lines; w += 32) {
    const int pl = w / lines, ln = w - pl * lines;
    const T* base = pl < 3 * NP ? q + (size_t)pl * ks : B.s.B + e0 + (size_t)(pl - 3 * NP) * ks;
    prefetch_l2(base + ln * per_line);
  }
}

__device__ __forceinline__ BatchSeg load_seg(const BatchSeg* p) {
  BatchSeg S;
  const int4* src = reinterpret_cast<const int4*>(p);
  int4* dst = reinterpret_cast<int4*>(&S);
  dst[0] = __ldg(src);
  dst[1] = __ldg(src + 1);
  dst[2] = __ldg(src + 2);
  return S;
}

// kTC: the tensor-core stage body (FP32 tier); otherwise the SIMT body (T = float
// or double). Every warp of the CTA takes tickets on its own (no barrier in the
// loop): a stage ticket is two warp-tiles of 32 elements, a TVB ticket 128 elements,
// four to a lane. Lane 0 holds the warp's next ticket with its segment record,
// fetched while the warp works on the current one, and waits only when a ticket
// opens a segment it has not yet waited for (the tiles a segment needs are the same
// for all its tickets). The warp prefetches the next stage ticket's node planes to
// L2, as the separate launch does a tile ahead.
template <typename T, int N, bool kTC>
__global__ void __launch_bounds__(kTC ? kTcMaxBlock : kBatchTile, 1) k_batch(const __grid_constant__ BatchLaunch<T> bl) {
  static_assert(kBatchStageTile % 32 == 0 && kBatchTvbTile % 32 == 0, "whole warp-tiles per ticket");
  static_assert(sizeof(BatchLaunch<T>) <= 32000, "batch launch parameters exceed the kernel-parameter space");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long s_k0[kBatchMaxScn];   // finest substep count at the start of the call
  T* sops = reinterpret_cast<T*>(smem_raw);
  // the macro counters move only after the launch (the finish kernel): read once
  for (int i = threadIdx.x; i < bl.nscn; i += blockDim.x)
    s_k0[i] = __ldcg(bl.scn[i].s.macro) * (long long)bl.period[i];
  // every scenario of the group has the same operators: stage the first one's
  // (the staging ends with a CTA barrier, which also publishes s_k0)
  if constexpr (kTC) {
    stage_ops<T, N, TcSmem<N>::OPS>(sops, bl.scn[0].s.ops);
  } else {
    stage_ops<T, N>(sops, bl.scn[0].s.ops);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int total = __ldcg(&bl.ctl->total);
  // lane 0: the next ticket and its segment
  int ticket = 0, nsg = -1, ok_sg = -1;
  BatchSeg nS;
  if (lane == 0) {
    ticket = atomicAdd(&bl.ctl->head, 1);
    if (ticket < total) {
      nsg = __ldg(bl.seg_of + ticket);
      nS = load_seg(bl.segs + nsg);
    }
  }
  for (;;) {
    // lane 0 takes the held ticket, waits if it opens a segment, and fetches the next
    int sg = -1, tile = 0, go = 0, scn = 0, kind = 0, nactive = 0, kofs = 0;
    int pkind = -1, pscn = 0, pe0 = 0, pn = 0, pkofs = 0;   // the next ticket, for the prefetch
    if (lane == 0 && nsg >= 0) {
      const BatchSeg S = nS;
      sg = nsg;
      tile = ticket - S.t0;
      scn = S.scn;
      kind = S.kind;
      nactive = S.nactive;
      kofs = S.kofs;
      go = sg == ok_sg ? 1 : batch_wait(bl, S);
      if (go) ok_sg = sg;
      ticket = atomicAdd(&bl.ctl->head, 1);
      nsg = -1;
      if (ticket < total) {
        nsg = __ldg(bl.seg_of + ticket);
        nS = load_seg(bl.segs + nsg);
        pkind = nS.kind;
        pscn = nS.scn;
        pe0 = (ticket - nS.t0) * kBatchStageTile;
        pn = min(kBatchStageTile, nS.nactive - pe0);
        pkofs = nS.kofs;
      }
    }
    sg = __shfl_sync(0xffffffffu, sg, 0);
    if (sg < 0) break;
    tile = __shfl_sync(0xffffffffu, tile, 0);
    go = __shfl_sync(0xffffffffu, go, 0);
    scn = __shfl_sync(0xffffffffu, scn, 0);
    kind = __shfl_sync(0xffffffffu, kind, 0);
    nactive = __shfl_sync(0xffffffffu, nactive, 0);
    kofs = __shfl_sync(0xffffffffu, kofs, 0);
    pkind = __shfl_sync(0xffffffffu, pkind, 0);
    if (go) {
      // the scenario's parameters, in the kernel-parameter space
      const StageParams<T>& wp = bl.scn[scn];
      // the substep count: the scenario's count at the start of the call plus the
      // phase's offset in this call
      const long long k = s_k0[scn] + kofs;
      // the warp's next stage ticket: its planes start moving to L2 now
      if (pkind == 0) {
        pscn = __shfl_sync(0xffffffffu, pscn, 0);
        pe0 = __shfl_sync(0xffffffffu, pe0, 0);
        pn = __shfl_sync(0xffffffffu, pn, 0);
        pkofs = __shfl_sync(0xffffffffu, pkofs, 0);
        batch_prefetch_stage<T, N>(bl.scn[pscn], s_k0[pscn] + pkofs, pe0, pn, lane);
      }
      double injected = 0.0;
      if (kind == 0) {
        if constexpr (kTC) {
          float* sw = sops + TcSmem<N>::OPS + warp * TcSmem<N>::WARP;
          const int t0 = tile * (kBatchStageTile / 32);
          const int t1 = min(t0 + kBatchStageTile / 32, (nactive + 31) / 32);
          injected = stage_tc_range<N>(wp, k, nactive, sops, sw, t0, 1, t1, true);
        } else {
          const int e0 = tile * kBatchStageTile;
          injected = stage_range<T, N>(wp, sops, e0 + lane, 32, min(e0 + kBatchStageTile, nactive), k);
        }
      } else {
        const int e0 = tile * kBatchTvbTile;
        tvb_range<T, N>(wp, 1, sops, e0 + lane, 32, min(e0 + kBatchTvbTile, nactive), k);
      }
      if (injected != 0.0) atomicAdd(wp.s.acc, injected);
    }
    __syncwarp();   // the lanes' stores of the tile are issued and ordered before lane 0's
    if (lane == 0) {
      __threadfence();   // ... which a device-scope fence makes visible before the counter moves
      if (go) atomicAdd(bl.ran + scn, 1);
      atomicAdd(bl.done + scn, 1);
    }
  }
}

}  // namespace swe
