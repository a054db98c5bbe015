// Stage kernel with the volume contractions and the lift on tensor cores (FP32
// tier with split-BF16 products, Section 7.1's N(Q) = Pr cF1 + Ps cF2 + P cS and
// Section 7.2's R = N - L^g F).
//
// Each warp owns 32 elements (two 16-row m-tiles). First one thread per element
// computes the face traces and well-balanced fluxes at its 3 Ng Gauss points
// (shared with the SIMT kernel) into the warp's shared flux tile. Then per m-tile
// and per tile of 8 cubature points:
//   interpolation  D[16 el x 8 pts] = State[16 el x Np] * Op^T  (mma m16n8k16),
//                  for eta, hu, hv, B with Ic and for B with Icr, Ics;
//   flux           evaluated in registers on the accumulator layout: lane (g, t)
//                  holds elements g, g+8 at cubature points 2t, 2t+1, which is
//                  exactly the A-fragment layout of the next product;
//   projection     R[16 el x Np] += Flux[16 el x 8 pts] * Pr^T (Ps^T, P^T)
//                  (mma m16n8k8), accumulated over all cubature tiles;
// and, on the same accumulators, per tile of 8 face points
//   lift           R[16 el x Np] -= SurfaceFlux[16 el x 8 pts] * L^g^T (m16n8k8).
// Every product is split: a = a_hi + a_lo in bfloat16 (operators and data), and
// a*b ~ a_hi*b_hi + a_hi*b_lo + a_lo*b_hi with FP32 accumulation (relative error
// of order 2^-16 per product). The warp then hands R and the state to one thread
// per element through shared memory for the Adams-Bashforth commit and the
// positivity limiter, which are shared with the SIMT kernel.
#pragma once

#include <cuda_bf16.h>

#include "kernels.cuh"

namespace swe {

constexpr int kTcWarps = 4;                  // warps per CTA unless a solver sets another count
constexpr int kTcBlock = 32 * kTcWarps;
constexpr int kTcMaxWarps = 8;               // 8 warps x 32 threads x 255 registers fill the register file
constexpr int kTcMaxBlock = 32 * kTcMaxWarps;

__device__ __forceinline__ void mma_k16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_k8(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(b0));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// float -> (hi, lo) TF32 pair: hi rounded to 10 mantissa bits, lo the remainder
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(x));
  lo = __float_as_uint(x - __uint_as_float(hi));
}

// two floats -> (hi, lo) bf16x2 pairs; the first float goes to the low half
__device__ __forceinline__ void split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Per-warp shared tiles are node-major with the 32 elements of the warp
// contiguous and a stride of LS = 36 words per node: one thread per element
// reads a node of its own element without bank conflicts, and the mma fragment
// reads (rows g, g+8, nodes 2t, 2t+1) land on 32 distinct banks.
constexpr int LS = 36;

template <int N>
struct TcSmem {
  using D = Dims<N>;
  using C = TcDims<N>;
  // per warp: state [4 fields][KP nodes][LS]; surface fluxes [3][KF face points][LS],
  // later R [3][NPT nodes][LS] in the same rows (field stride FR); geo [32][4];
  // pressure form md [32]
  static constexpr int STATE = 0;
  static constexpr int FRT = STATE + 4 * C::KP * LS;
  static constexpr int GEO = FRT + 3 * C::FR * LS;
  static constexpr int MD = GEO + 32 * 4;
  static constexpr int WARP = MD + 32;                   // floats per warp
  static constexpr int OPS = OpLayout<N>::TAIL;          // floats of per-element operators (staged first)
  // dynamic shared memory of a CTA of `warps` warps: one operator copy, one tile set per warp
  static constexpr int bytes(int warps) { return (OPS + warps * WARP) * 4; }
  static constexpr int BYTES = bytes(kTcWarps);
};

// One warp-tile of 32 elements (element e = 32 tile + lane): load, surface fluxes,
// volume term and lift on tensor cores, commit and limiter. k: the finest substep
// count of the schedule; nactive: elements [0, nactive) are active at this substep;
// next_tile: the warp's next tile (its planes are prefetched to L2), or -1; sw: the
// warp's shared tiles; kComp: compensated state update in the commit.
template <int N, bool kComp = false>
__device__ __forceinline__ void stage_tc_warp(const StageParams<float>& p, long long k, int nactive,
                                              const float* sops, float* sw, int tile, int next_tile,
                                              double* injected) {
  using D = Dims<N>;
  using C = TcDims<N>;
  using TL = TcLayout<N>;
  using SM = TcSmem<N>;
  constexpr int NP = D::NP, NPP = D::NPP, KP = C::KP, KSTEP = C::KSTEP, CT = C::CT, NT = C::NT;
  constexpr int NG = D::NG, KT = C::KT, KF = C::KF, FR = C::FR;
  // operator fragments stay in global memory: every warp reads the same few KB,
  // which the L1 cache serves
  const uint32_t* __restrict__ stc = p.s.tcops;
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  float* s_state = sw + SM::STATE;
  float* s_FR = sw + SM::FRT;
  float* s_geo = sw + SM::GEO;
  float* s_md = sw + SM::MD;
  const Sched& sc = p.sc;
  const float gg = (float)p.ph.g, hvel = (float)p.ph.hvel, hg = 0.5f * gg;
  const size_t ks = (size_t)sc.KS, fstride = (size_t)NP * ks, bstride = 3 * fstride;
  // ---- load: lane = element; each node plane is one coalesced 128-byte line ----
  const int e = tile * 32 + lane;
  const bool valid = e < nactive;
  int lev = 1;
  long long a = 0;
  if (valid) {
    lev = level_of(sc, e);
    a = k >> (lev - 1);
    const float* qe = p.s.q + (size_t)(a & 1) * bstride + e;
#pragma unroll
    for (int f = 0; f < 3; ++f)
#pragma unroll
      for (int i = 0; i < NP; ++i) s_state[(f * KP + i) * LS + lane] = ldm(qe + f * fstride + i * ks);
#pragma unroll
    for (int i = 0; i < NP; ++i) s_state[(3 * KP + i) * LS + lane] = __ldg(p.s.B + e + i * ks);
    reinterpret_cast<float4*>(s_geo)[lane] = __ldg(reinterpret_cast<const float4*>(p.s.geo) + e);
    // depth form of the pressure for dry elements (exact rules only)
    s_md[lane] = (Dims<N>::EXACT && ldm(p.s.dry + e)) ? 1.f : 0.f;
  } else {
    s_md[lane] = 0.f;
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int i = 0; i < NP; ++i) s_state[(f * KP + i) * LS + lane] = 0.f;
    reinterpret_cast<float4*>(s_geo)[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int i = NP; i < KP; ++i) s_state[(f * KP + i) * LS + lane] = 0.f;
  __syncwarp();

  // the next tile's planes and this tile's older R slots start moving now: one
  // 128-byte line per lane and plane (the parity of the first element stands for
  // the tile; these are hints, every address lies inside its array)
  {
    const int e0n = next_tile * 32;
    if (next_tile >= 0 && e0n < nactive) {
      const long long an = k >> (level_of(sc, e0n) - 1);
      const float* qn = p.s.q + (size_t)(an & 1) * bstride + e0n;
      for (int pl = lane; pl < 4 * NP; pl += 32)
        prefetch_l2(pl < 3 * NP ? qn + pl * ks : p.s.B + e0n + (pl - 3 * NP) * ks);
    }
    const long long a0 = __shfl_sync(0xffffffffu, a, 0);
    if (p.mode == 0) {
      const int e0 = tile * 32;
      for (int s = 1; s < 3 && s <= a0; ++s) {
        const float* rs = p.s.ring + (size_t)((a0 - s) % 3) * bstride + e0;
        for (int pl = lane; pl < 3 * NP; pl += 32) prefetch_l2(rs + pl * ks);
      }
      if constexpr (kComp)
        for (int pl = lane; pl < 3 * NP; pl += 32) prefetch_l2(p.s.comp + e0 + pl * ks);
    }
  }

  // ---- surface fluxes, one thread per element, into the warp's flux tile ----
  {
    float* sf = s_FR + lane;
    for (int q = 3 * NG; q < KF; ++q) {  // padding points: zero rows for the lift
      sf[(0 * FR + q) * LS] = 0.f;
      sf[(1 * FR + q) * LS] = 0.f;
      sf[(2 * FR + q) * LS] = 0.f;
    }
    if (valid) {
      const float4 ge = reinterpret_cast<const float4*>(s_geo)[lane];
      const float* my = s_state + lane;
      auto own = [&](int f, int jn) -> float { return my[(f * KP + jn) * LS]; };
      // the element's node-0 flux, subtracted here and from the volume fluxes (see
      // the reference flux below): constant fluxes contribute nothing to R
      const float hu0 = my[(1 * KP) * LS], hv0 = my[(2 * KP) * LS], d0 = my[0] - my[(3 * KP) * LS];
      const float id0 = d0 > hvel ? recip(d0) : 0.f;
      const float u0 = hu0 * id0, v0 = hv0 * id0;
      surface_fluxes<float, N, true>(p, sops, e, k, own, ge.x, ge.y, ge.z, ge.w, s_md[lane],
                                     [&](int f, int gq, float f0, float f1, float f2, float vx, float vy) {
                                       const int q = f * NG + gq;
                                       const float fr = hu0 * vx + hv0 * vy;
                                       sf[(0 * FR + q) * LS] = f0 - fr;
                                       sf[(1 * FR + q) * LS] = f1 - u0 * fr;
                                       sf[(2 * FR + q) * LS] = f2 - v0 * fr;
                                     });
    } else {
      for (int q = 0; q < 3 * NG; ++q) {
        sf[(0 * FR + q) * LS] = 0.f;
        sf[(1 * FR + q) * LS] = 0.f;
        sf[(2 * FR + q) * LS] = 0.f;
      }
    }
  }
  __syncwarp();

  // ---- volume term and lift on tensor cores, one m-tile of 16 elements at a time ----
#pragma unroll 1
  for (int mt = 0; mt < 2; ++mt) {
    const int r0 = 16 * mt + g, r1 = r0 + 8;
    // State A fragments (rows r0, r1; nodes 16ks + {2t, 2t+1, 2t+8, 2t+9}), hi and
    // lo. The surface and the bed enter relative to their values at node 0 of the
    // element (eta0, B0): the interpolation of a constant is exact and its
    // derivatives vanish (Ic B = B0 + Ic (B - B0), Icr B = Icr (B - B0)), so only
    // the within-element variation carries the split-product error, whether the
    // bed is thousands of metres deep or the water a millimetre thin.
    // All four fields enter relative to their node-0 values (c0 for row r0, c1 for r1).
    float c0[4], c1[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      c0[f] = s_state[(f * KP) * LS + r0];
      c1[f] = s_state[(f * KP) * LS + r1];
    }
    const float cE0 = c0[0], cE1 = c1[0], cB0 = c0[3], cB1 = c1[3];
    uint32_t ah[4][KSTEP][4], al[4][KSTEP][4];
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int ks = 0; ks < KSTEP; ++ks) {
        const float* sn = s_state + (f * KP + 16 * ks + 2 * t) * LS;   // node 16ks + 2t
        const float d0 = c0[f], d1 = c1[f];
        const float2 v00 = make_float2(sn[r0] - d0, sn[LS + r0] - d0);
        const float2 v10 = make_float2(sn[r1] - d1, sn[LS + r1] - d1);
        const float2 v01 = make_float2(sn[8 * LS + r0] - d0, sn[9 * LS + r0] - d0);
        const float2 v11 = make_float2(sn[8 * LS + r1] - d1, sn[9 * LS + r1] - d1);
        split2(v00.x, v00.y, ah[f][ks][0], al[f][ks][0]);
        split2(v10.x, v10.y, ah[f][ks][1], al[f][ks][1]);
        split2(v01.x, v01.y, ah[f][ks][2], al[f][ks][2]);
        split2(v11.x, v11.y, ah[f][ks][3], al[f][ks][3]);
      }
    const float4 ge0 = reinterpret_cast<const float4*>(s_geo)[r0];
    const float4 ge1 = reinterpret_cast<const float4*>(s_geo)[r1];
    // Reference flux: the volume fluxes cF1, cF2 of each row's node-0 state. A
    // constant flux adds nothing to R (its volume term and its own-side lift
    // cancel exactly), so it is subtracted here and from the surface fluxes and
    // the split products see only the flux's variation over the element (the
    // pressure p'' vanishes at node 0).
    float fr0[6], fr1[6];
    {
      const float d0 = cE0 - cB0, d1 = cE1 - cB1;
      const float i0 = d0 > hvel ? recip(d0) : 0.f, i1v = d1 > hvel ? recip(d1) : 0.f;
      const float u0 = c0[1] * i0, v0 = c0[2] * i0, u1 = c1[1] * i1v, v1 = c1[2] * i1v;
      const float a0r = ge0.x * c0[1] + ge0.y * c0[2], b0r = ge0.z * c0[1] + ge0.w * c0[2];
      const float a1r = ge1.x * c1[1] + ge1.y * c1[2], b1r = ge1.z * c1[1] + ge1.w * c1[2];
      fr0[0] = a0r; fr0[1] = u0 * a0r; fr0[2] = v0 * a0r; fr0[3] = b0r; fr0[4] = u0 * b0r; fr0[5] = v0 * b0r;
      fr1[0] = a1r; fr1[1] = u1 * a1r; fr1[2] = v1 * a1r; fr1[3] = b1r; fr1[4] = u1 * b1r; fr1[5] = v1 * b1r;
    }
    float Racc[3][NT][4];
#pragma unroll
    for (int f = 0; f < 3; ++f)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int c = 0; c < 4; ++c) Racc[f][nt][c] = 0.f;

    // interpolation fragments of the first cubature tile
    uint2 ibh[3][KSTEP], ibl[3][KSTEP];
#pragma unroll
    for (int op = 0; op < 3; ++op)
#pragma unroll
      for (int ks = 0; ks < KSTEP; ++ks) {
        const uint32_t* fb = stc + TL::INTERP + (((op * CT + 0) * KSTEP + ks) * 2) * 64 + lane * 2;
        ibh[op][ks] = __ldg(reinterpret_cast<const uint2*>(fb));
        ibl[op][ks] = __ldg(reinterpret_cast<const uint2*>(fb + 64));
      }
#pragma unroll 1
    for (int ct = 0; ct < CT; ++ct) {
      // projection fragments of this tile: in flight during the interpolation and flux
      uint32_t pbh[3][NT], pbl[3][NT];
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int op = 0; op < 3; ++op) {
          const uint32_t* fb = stc + TL::PROJ + (((op * CT + ct) * NT + nt) * 2) * 32 + lane;
          pbh[op][nt] = __ldg(fb);
          pbl[op][nt] = __ldg(fb + 32);
        }
      // interpolation: acc[0..3] = (eta, hu, hv, B) * Ic, acc[4] = B * Icr, acc[5] = B * Ics
      float acc[6][4];
#pragma unroll
      for (int o = 0; o < 6; ++o)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[o][c] = 0.f;
#pragma unroll
      for (int ks = 0; ks < KSTEP; ++ks) {
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          mma_k16(acc[f], al[f][ks], ibh[0][ks].x, ibh[0][ks].y);
          mma_k16(acc[f], ah[f][ks], ibl[0][ks].x, ibl[0][ks].y);
          mma_k16(acc[f], ah[f][ks], ibh[0][ks].x, ibh[0][ks].y);
        }
#pragma unroll
        for (int op = 1; op < 3; ++op) {
          mma_k16(acc[3 + op], al[3][ks], ibh[op][ks].x, ibh[op][ks].y);
          mma_k16(acc[3 + op], ah[3][ks], ibl[op][ks].x, ibl[op][ks].y);
          mma_k16(acc[3 + op], ah[3][ks], ibh[op][ks].x, ibh[op][ks].y);
        }
      }
      // interpolation fragments of the next tile: in flight during the flux and projection
      if (ct + 1 < CT) {
#pragma unroll
        for (int op = 0; op < 3; ++op)
#pragma unroll
          for (int ks = 0; ks < KSTEP; ++ks) {
            const uint32_t* fb = stc + TL::INTERP + (((op * CT + ct + 1) * KSTEP + ks) * 2) * 64 + lane * 2;
            ibh[op][ks] = __ldg(reinterpret_cast<const uint2*>(fb));
            ibl[op][ks] = __ldg(reinterpret_cast<const uint2*>(fb + 64));
          }
      }
      // flux and source at the lane's four points: (r0, 2t), (r0, 2t+1), (r1, 2t), (r1, 2t+1)
      float fl[8][4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float4 ge = c < 2 ? ge0 : ge1;
        const float rx = ge.x, ry = ge.y, sx = ge.z, sy = ge.w;
        // eta - eta0 and B - B0 at the point (element reference split)
        const float ec = acc[0][c];
        const float huc = (c < 2 ? c0[1] : c1[1]) + acc[1][c], hvc = (c < 2 ? c0[2] : c1[2]) + acc[2][c];
        const float bpc = acc[3][c];
        const float brc = acc[4][c], bsc = acc[5][c];
        const float hc = (c < 2 ? cE0 - cB0 : cE1 - cB1) + (ec - bpc);
        const float ih = hc > hvel ? recip(hc) : 0.f;
        const float u = huc * ih, v = hvc * ih;
        // momentum rows of cF1, cF2 written through the mass row; p'' (the
        // reference part is added in strong form before the commit)
        const float md = c < 2 ? s_md[r0] : s_md[r1];
        const float ep = ec - md * bpc;
        const float pr = hg * ep * (ec - (2.f - md) * bpc);
        const float a0 = rx * huc + ry * hvc, b0 = sx * huc + sy * hvc;
        const float* fr = c < 2 ? fr0 : fr1;
        fl[0][c] = a0 - fr[0];
        fl[1][c] = (u * a0 + rx * pr) - fr[1];
        fl[2][c] = (v * a0 + ry * pr) - fr[2];
        fl[3][c] = b0 - fr[3];
        fl[4][c] = (u * b0 + sx * pr) - fr[4];
        fl[5][c] = (v * b0 + sy * pr) - fr[5];
        const float gm = -gg * ep;
        fl[6][c] = gm * (rx * brc + sx * bsc);
        fl[7][c] = gm * (ry * brc + sy * bsc);
      }
      // A fragments (m16n8k8): reg0 = row r0 (points 2t, 2t+1), reg1 = row r1
      uint32_t fh[8][2], flo[8][2];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        split2(fl[q][0], fl[q][1], fh[q][0], flo[q][0]);
        split2(fl[q][2], fl[q][3], fh[q][1], flo[q][1]);
      }
      // projection: R_h += cF1_h Pr + cF2_h Ps; R_m += cF1_m Pr + cF2_m Ps + cS_m P
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const uint32_t bh[3] = {pbh[0][nt], pbh[1][nt], pbh[2][nt]};
        const uint32_t bl[3] = {pbl[0][nt], pbl[1][nt], pbl[2][nt]};
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          // cF1 (quantity f) with Pr, cF2 (3+f) with Ps, source (5+f, f>0) with P
          mma_k8(Racc[f][nt], flo[f][0], flo[f][1], bh[0]);
          mma_k8(Racc[f][nt], fh[f][0], fh[f][1], bl[0]);
          mma_k8(Racc[f][nt], fh[f][0], fh[f][1], bh[0]);
          mma_k8(Racc[f][nt], flo[3 + f][0], flo[3 + f][1], bh[1]);
          mma_k8(Racc[f][nt], fh[3 + f][0], fh[3 + f][1], bl[1]);
          mma_k8(Racc[f][nt], fh[3 + f][0], fh[3 + f][1], bh[1]);
          if (f > 0) {
            mma_k8(Racc[f][nt], flo[5 + f][0], flo[5 + f][1], bh[2]);
            mma_k8(Racc[f][nt], fh[5 + f][0], fh[5 + f][1], bl[2]);
            mma_k8(Racc[f][nt], fh[5 + f][0], fh[5 + f][1], bh[2]);
          }
        }
      }
    }
    // lift: R -= Flux * L^g^T over the face points, k8 tiles of 8 points; the
    // fluxes of rows r0, r1 at points 8kt + 2t, 2t + 1 form the A fragments
#pragma unroll
    for (int kt = 0; kt < KT; ++kt) {
      uint32_t lbh[NT], lbl[NT];
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const uint32_t* fb = stc + TL::LIFT + ((kt * NT + nt) * 2) * 32 + lane;
        lbh[nt] = __ldg(fb);
        lbl[nt] = __ldg(fb + 32);
      }
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        const float* fq = s_FR + (f * FR + 8 * kt + 2 * t) * LS;
        uint32_t ah0, al0, ah1, al1;
        split2(fq[r0], fq[LS + r0], ah0, al0);
        split2(fq[r1], fq[LS + r1], ah1, al1);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          mma_k8(Racc[f][nt], al0, al1, lbh[nt]);
          mma_k8(Racc[f][nt], ah0, ah1, lbl[nt]);
          mma_k8(Racc[f][nt], ah0, ah1, lbh[nt]);
        }
      }
    }
    // strong-form reference pressure (element reference split, see kernels.cuh):
    // R_hu -= g h0 (rx Dr + sx Ds)(eta - eta0), R_hv -= g h0 (ry Dr + sy Ds)(eta - eta0).
    // The leading term of R at depth, so TF32 split products (2^-21 per product).
    {
      float Dacc[2][NT][4];
#pragma unroll
      for (int op = 0; op < 2; ++op)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
          for (int c = 0; c < 4; ++c) Dacc[op][nt][c] = 0.f;
#pragma unroll
      for (int kk = 0; kk < KP / 8; ++kk) {
        const float* sn = s_state + (8 * kk + t) * LS;   // eta at node 8kk + t
        uint32_t eh[4], el[4];
        split_tf32(sn[r0] - cE0, eh[0], el[0]);
        split_tf32(sn[r1] - cE1, eh[1], el[1]);
        split_tf32(sn[4 * LS + r0] - cE0, eh[2], el[2]);
        split_tf32(sn[4 * LS + r1] - cE1, eh[3], el[3]);
#pragma unroll
        for (int op = 0; op < 2; ++op)
#pragma unroll
          for (int nt = 0; nt < NT; ++nt) {
            const uint32_t* fb = stc + TL::DIFF + (((op * (KP / 8) + kk) * NT + nt) * 2) * 64 + lane * 2;
            const uint2 bh = __ldg(reinterpret_cast<const uint2*>(fb));
            const uint2 bl = __ldg(reinterpret_cast<const uint2*>(fb + 64));
            mma_tf32(Dacc[op][nt], el, bh.x, bh.y);
            mma_tf32(Dacc[op][nt], eh, bl.x, bl.y);
            mma_tf32(Dacc[op][nt], eh, bh.x, bh.y);
          }
      }
      const float gh0 = -gg * (cE0 - cB0), gh1 = -gg * (cE1 - cB1);
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float4 ge = c < 2 ? ge0 : ge1;
          const float gh = c < 2 ? gh0 : gh1;
          Racc[1][nt][c] += gh * (ge.x * Dacc[0][nt][c] + ge.z * Dacc[1][nt][c]);
          Racc[2][nt][c] += gh * (ge.y * Dacc[0][nt][c] + ge.w * Dacc[1][nt][c]);
        }
    }
    // every lane has read this m-tile's flux columns before R overwrites them
    __syncwarp();
    // R of this m-tile to shared memory: rows r0, r1, nodes 8nt + {2t, 2t+1}
#pragma unroll
    for (int f = 0; f < 3; ++f)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        float* rn = s_FR + (f * FR + 8 * nt + 2 * t) * LS;
        rn[r0] = Racc[f][nt][0];
        rn[LS + r0] = Racc[f][nt][1];
        rn[r1] = Racc[f][nt][2];
        rn[LS + r1] = Racc[f][nt][3];
      }
  }
  __syncwarp();

  // ---- one thread per element: commit, positivity ----
  if (valid) {
    float R0[NP], R1[NP], R2[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      R0[i] = s_FR[(0 * FR + i) * LS + lane];
      R1[i] = s_FR[(1 * FR + i) * LS + lane];
      R2[i] = s_FR[(2 * FR + i) * LS + lane];
    }
    const float4 ge = reinterpret_cast<const float4*>(s_geo)[lane];
    // the per-element operators were staged at the start of shared memory with the
    // OpLayout offsets, so the shared epilogue indexes them directly
    const float* my = s_state + lane;
    float eta[NPP], hu[NPP], hv[NPP], bb[NPP];
#pragma unroll
    for (int i = 0; i < NPP; ++i) {
      eta[i] = my[(0 * KP + i) * LS];
      hu[i] = my[(1 * KP + i) * LS];
      hv[i] = my[(2 * KP + i) * LS];
      bb[i] = my[(3 * KP + i) * LS];
    }
    commit_and_limit<float, N, kComp>(p, sops, e, lev, a, eta, hu, hv, bb, ge.x, ge.y, ge.z, ge.w, R0, R1, R2,
                               injected);
  }
  __syncwarp();
}

// Warp-tiles t0, t0 + step, ... below t1 (each warp calls it for its own tiles;
// with prefetch the planes of the warp's next tile are prefetched to L2); returns
// the mass the positivity limiter's dry resets injected. The separate launch and
// the persistent batch kernel both inline it (out of line the body ran 1.5 times
// slower: its parameters become memory loads).
template <int N, bool kComp = false>
__device__ __forceinline__ double stage_tc_range(const StageParams<float>& __restrict__ p, long long k,
                                              int nactive, const float* __restrict__ sops, float* sw, int t0,
                                              int step, int t1, bool prefetch) {
  double injected = 0.0;
  for (int tile = t0; tile < t1; tile += step)
    stage_tc_warp<N, kComp>(p, k, nactive, sops, sw, tile, prefetch ? tile + step : -1, &injected);
  return injected;
}

// CTA: blockDim.x / 32 warps (1 to kTcMaxWarps), each with its own shared tiles after
// the CTA's operator copy. kComp: compensated state update (p.s.comp).
template <int N, bool kComp = false>
__global__ void __launch_bounds__(kTcMaxBlock, 1) k_stage_tc(const __grid_constant__ StageParams<float> p) {
  using SM = TcSmem<N>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sops = reinterpret_cast<float*>(smem_raw);                       // [0, OPS)
  {
    const float4* src = reinterpret_cast<const float4*>(p.s.ops);
    float4* dst = reinterpret_cast<float4*>(sops);
    for (int i = threadIdx.x; i < SM::OPS / 4; i += blockDim.x) dst[i] = __ldg(src + i);
    __syncthreads();
  }
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float* sw = sops + SM::OPS + warp * SM::WARP;
  const long long k = (*p.s.macro) * (1LL << (p.sc.L - 1)) + p.j;
  const int ntiles = (p.nactive + 31) / 32;
  const double injected =
      stage_tc_range<N, kComp>(p, k, p.nactive, sops, sw, blockIdx.x * nw + warp, gridDim.x * nw, ntiles, true);
  if (injected != 0.0) atomicAdd(p.s.acc, injected);
}


}  // namespace swe
