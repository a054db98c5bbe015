// The kernel split of Section 7 as an ablation of the fused stage kernel: the
// traces at the face Gauss points are computed by one kernel and stored in global
// memory (the Q^g of the update kernel, Section 7.3), the volume term by a second
// (Section 7.1) and the surface term by a third that reads the stored traces of
// both sides of every face (Section 7.2). R only, level-synchronous state, output
// in the caller's layout (as swe_rhs). The arithmetic is the fused SIMT kernel's:
// the same traces relative to the same face references, the same flux and lift;
// only the volume and surface sums are added in the other order.
#pragma once

#include "kernels.cuh"

namespace swe {

// Scratch of the split path, planes of stride KS:
//   qg  [3 faces][NG][4] traces (e, hu, hv, b) relative to the face reference,
//       then [3 faces][2] the face reference (Ef, Bf)
//   rg  [3][NP] the volume term
template <typename T>
struct SplitBufs {
  T* qg;
  T* rg;
};

template <int N>
struct SplitLayout {
  static constexpr int TRACES = 3 * Dims<N>::NG * 4;
  static constexpr int PLANES = TRACES + 6;
};

// Q^g: own-side traces at the 3 NG face Gauss points.
template <typename T, int N>
__global__ void __launch_bounds__(kBlock) k_split_traces(StageParams<T> p, SplitBufs<T> sb) {
  using D = Dims<N>;
  using O = OpLayout<N>;
  constexpr int NP = D::NP, NFP = D::NFP, NG = D::NG;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sops = reinterpret_cast<T*>(smem_raw);
  stage_ops<T, N, O::TAIL>(sops, p.s.ops);
  const Sched& sc = p.sc;
  const long long k = (*p.s.macro) * (1LL << (sc.L - 1)) + p.j;
  const size_t ks = (size_t)sc.KS, fstride = (size_t)NP * ks, bstride = 3 * fstride;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p.nactive; e += gridDim.x * blockDim.x) {
    const T* q = p.s.q + (size_t)((k >> (level_of(sc, e) - 1)) & 1) * bstride + e;
    const int4 cn = __ldg(p.s.conn + e);
    const T E0 = __ldg(q), B0 = __ldg(p.s.B + e);
#pragma unroll 1
    for (int f = 0; f < 3; ++f) {
      T Ef = E0, Bf = B0;   // node 0 of the lower-numbered element of the pair
      const int nb = f == 0 ? cn.x : (f == 1 ? cn.y : cn.z);
      if (nb >= 0 && nb < e) {
        Ef = __ldg(p.s.q + (size_t)((k >> (level_of(sc, nb) - 1)) & 1) * bstride + nb);
        Bf = __ldg(p.s.B + nb);
      }
      T oe[NFP], ou[NFP], ov[NFP], oB[NFP];
#pragma unroll
      for (int m = 0; m < NFP; ++m) {
        const size_t idx = (size_t)face_node_rt(Dims<N>::N, f, m) * ks;
        oe[m] = __ldg(q + idx) - Ef;
        ou[m] = __ldg(q + fstride + idx);
        ov[m] = __ldg(q + 2 * fstride + idx);
        oB[m] = __ldg(p.s.B + e + idx) - Bf;
      }
#pragma unroll 1
      for (int gq = 0; gq < NG; ++gq) {
        T i1[D::NFPP];
        load_row<T, D::NFPP>(sops + O::I1D + gq * D::NFPP, i1);
        T te = 0, tu = 0, tv = 0, tb = 0;
#pragma unroll
        for (int m = 0; m < NFP; ++m) {
          te += i1[m] * oe[m];
          tu += i1[m] * ou[m];
          tv += i1[m] * ov[m];
          tb += i1[m] * oB[m];
        }
        T* o = sb.qg + (size_t)((f * NG + gq) * 4) * ks + e;
        o[0] = te;
        o[ks] = tu;
        o[2 * ks] = tv;
        o[3 * ks] = tb;
      }
      sb.qg[(size_t)(SplitLayout<N>::TRACES + 2 * f) * ks + e] = Ef;
      sb.qg[(size_t)(SplitLayout<N>::TRACES + 2 * f + 1) * ks + e] = Bf;
    }
  }
}

// Volume term and the strong-form reference pressure, stored as planes.
template <typename T, int N>
__global__ void __launch_bounds__(kBlock) k_split_volume(StageParams<T> p, SplitBufs<T> sb) {
  using D = Dims<N>;
  constexpr int NP = D::NP, NPP = D::NPP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sops = reinterpret_cast<T*>(smem_raw);
  stage_ops<T, N>(sops, p.s.ops);
  const Sched& sc = p.sc;
  const long long k = (*p.s.macro) * (1LL << (sc.L - 1)) + p.j;
  const T g = (T)p.ph.g, hvel = (T)p.ph.hvel;
  const size_t ks = (size_t)sc.KS, fstride = (size_t)NP * ks, bstride = 3 * fstride;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p.nactive; e += gridDim.x * blockDim.x) {
    const T* q = p.s.q + (size_t)((k >> (level_of(sc, e) - 1)) & 1) * bstride + e;
    T eta[NPP], hu[NPP], hv[NPP], bb[NPP];
    load_nodes<T, NP, NPP>(q, ks, eta);
    load_nodes<T, NP, NPP>(q + fstride, ks, hu);
    load_nodes<T, NP, NPP>(q + 2 * fstride, ks, hv);
    load_nodes<T, NP, NPP>(p.s.B + e, ks, bb);
    T gm[4];
    load_row_global<T, 4>(p.s.geo + 4 * (size_t)e, gm);
    const T md = (Dims<N>::EXACT && p.s.dry[e]) ? T(1) : T(0);
    T R0[NP], R1[NP], R2[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) { R0[i] = 0; R1[i] = 0; R2[i] = 0; }
    volume_term<T, N>(sops, eta, hu, hv, bb, gm[0], gm[1], gm[2], gm[3], md, g, hvel, R0, R1, R2);
    add_reference_pressure<T, N>(sops, eta, bb, g, gm[0], gm[1], gm[2], gm[3], R1, R2);
    store_nodes<T, NP, NP>(sb.rg + e, ks, R0);
    store_nodes<T, NP, NP>(sb.rg + fstride + e, ks, R1);
    store_nodes<T, NP, NP>(sb.rg + 2 * fstride + e, ks, R2);
  }
}

// Surface term from the stored traces of both sides, lifted onto the volume term;
// R written in the caller's layout.
template <typename T, int N>
__global__ void __launch_bounds__(kBlock) k_split_surface(StageParams<T> p, SplitBufs<T> sb) {
  using D = Dims<N>;
  using O = OpLayout<N>;
  constexpr int NP = D::NP, NPP = D::NPP, NG = D::NG;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sops = reinterpret_cast<T*>(smem_raw);
  stage_ops<T, N, O::TAIL>(sops, p.s.ops);
  const Sched& sc = p.sc;
  const long long k = (*p.s.macro) * (1LL << (sc.L - 1)) + p.j;
  const T g = (T)p.ph.g, hvel = (T)p.ph.hvel, hg = T(0.5) * g, qg = T(0.25) * g;
  const size_t ks = (size_t)sc.KS, fstride = (size_t)NP * ks, bstride = 3 * fstride;
  const int K = sc.K;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p.nactive; e += gridDim.x * blockDim.x) {
    T R0[NPP], R1[NPP], R2[NPP];
    load_nodes<T, NP, NPP>(sb.rg + e, ks, R0);
    load_nodes<T, NP, NPP>(sb.rg + fstride + e, ks, R1);
    load_nodes<T, NP, NPP>(sb.rg + 2 * fstride + e, ks, R2);
    T gm[4];
    load_row_global<T, 4>(p.s.geo + 4 * (size_t)e, gm);
    const T rx = gm[0], ry = gm[1], sx = gm[2], sy = gm[3];
    const T md = (Dims<N>::EXACT && p.s.dry[e]) ? T(1) : T(0);
    const T E0 = __ldg(p.s.q + (size_t)((k >> (level_of(sc, e) - 1)) & 1) * bstride + e);
    const T B0 = __ldg(p.s.B + e);
    const int4 cn = __ldg(p.s.conn + e);
#pragma unroll 1
    for (int f = 0; f < 3; ++f) {
      const T vxn = f == 0 ? -sx : (f == 1 ? rx + sx : -rx);
      const T vyn = f == 0 ? -sy : (f == 1 ? ry + sy : -ry);
      const T v2 = vxn * vxn + vyn * vyn;
      const T iv = rsqrt_t(v2);
      const T nx = vxn * iv, ny = vyn * iv, hs = T(0.5) * v2 * iv;
      const int nb = f == 0 ? cn.x : (f == 1 ? cn.y : cn.z);
      const int fn = (cn.w >> (2 * f)) & 3;
      const T Ef = sb.qg[(size_t)(SplitLayout<N>::TRACES + 2 * f) * ks + e];
      const T Bf = sb.qg[(size_t)(SplitLayout<N>::TRACES + 2 * f + 1) * ks + e];
      const T hf = Ef - Bf, dE = Ef - E0, dB = Bf - B0;
#pragma unroll 1
      for (int gq = 0; gq < NG; ++gq) {
        const T* om = sb.qg + (size_t)((f * NG + gq) * 4) * ks + e;
        const Trace<T> tm = {om[0], om[ks], om[2 * ks], om[3 * ks]};
        Trace<T> tp;
        if (nb >= 0) {   // the neighbour's own point NG-1-gq of its face fn
          const T* op = sb.qg + (size_t)((fn * NG + NG - 1 - gq) * 4) * ks + nb;
          tp = {op[0], op[ks], op[2 * ks], op[3 * ks]};
        } else if (nb == kFarField) {   // far field over the continued bed
          tp = {(T)p.ph.ff_h - hf + tm.b, (T)p.ph.ff_hu, (T)p.ph.ff_hv, tm.b};
        } else {         // reflecting wall: mirror the normal momentum
          const T mn = tm.hu * nx + tm.hv * ny;
          tp = {tm.e, tm.hu - T(2) * mn * nx, tm.hv - T(2) * mn * ny, tm.b};
        }
        T f0, f1, f2;
        wb_flux<T>(tm, tp, hf, tm.e + dE, tm.b + dB, md, nx, ny, vxn, vyn, hs, g, hg, qg, hvel, f0, f1, f2);
        T lg[NPP];
        load_row<T, NPP>(sops + O::LGT + (f * NG + gq) * NPP, lg);
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          R0[i] -= lg[i] * f0;
          R1[i] -= lg[i] * f1;
          R2[i] -= lg[i] * f2;
        }
      }
    }
    const int ce = p.perm[e];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      p.out[((size_t)0 * K + ce) * NP + i] = R0[i];
      p.out[((size_t)1 * K + ce) * NP + i] = R1[i];
      p.out[((size_t)2 * K + ce) * NP + i] = R2[i];
    }
  }
}

}  // namespace swe
