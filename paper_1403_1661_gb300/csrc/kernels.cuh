// Device kernels of the DG shallow-water right-hand side, the multirate
// Adams-Bashforth update and the limiters (CUDA, sm_103a).
//
// One thread owns one element (element-blocked SIMT): the element's nodal state
// stays in registers from the loads to the committed, limited result, and the
// reference operators are staged once per CTA in shared memory, where every warp
// reads them as broadcasts. Nodal arrays are node-major planes (node i of element
// e at plane[i * KS + e]), so a warp's loads and stores of one node cover
// consecutive elements: whole lines, and nearly so for the neighbour traces of
// a mesh numbered with locality.
//
// Formulation. The state is stored as (eta, hu, hv) with the free surface
// eta = h + B. The momentum fluxes and the source are written about the datum
// eta = 0 ("pre-balanced"): with the cubature exact to degree 3N-1 and the face
// Gauss rule exact to degree 3N, the static parts g B^2/2 of the volume flux,
// g B grad B of the source and g (B^-)^2/2 of the face flux cancel element by
// element (divergence theorem), so dropping them gives the same semi-discrete
// R(Q) as Section 3 / Eq. well_balance in exact arithmetic while avoiding the
// cancellation of g h^2/2 against g h grad B in floating point:
//   volume:  F = (hu, hu u + p, hu v), G = (hv, hv u, hv v + p), p = g/2 eta (h - B),
//            S = (0, -g eta B_x, -g eta B_y);
//   faces:   pressure term of the well-balanced flux (own side "-")
//            g/2 eta^- (h^- - B^-) + g/4 (h*^+ - h*^-)(h*^+ + h*^-),
//            h*^{+-} = max(0, eta^{+-} - max(B^+, B^-)).
// Element reference split. With eta = eta0 + eta' and B = B0 + B' (eta0, B0 the
// element's values at its node 0), the pressure g/2 eta (eta - 2B) is a constant
// plus terms linear in eta' and B' with constant coefficients plus
// p'' = g/2 eta' (eta' - 2B'). For a constant or such a linear term P (a
// polynomial of degree N) the volume term plus the own-side face term is exactly
// the strong derivative -dP/dx (integration by parts, exact integration); with the
// source's -g eta0 grad B' the linear terms sum to -g h0 grad eta, h0 = eta0 - B0.
// So both kernels take p'' in the volume and face pressures, the source
// -g eta' grad B', and add -g h0 (r_x Dr + s_x Ds) eta (and the y analogue) once.
// At ocean depths the pressure is ~1e5 where R is ~1, and on a beach a film of
// millimetres sits on a bed metres above the datum: the rewrite removes both
// cancellations, and a lake at rest at any level gives R = 0 exactly. Where both
// sides of a face are wet the jump h*^+ - h*^- is computed as eta^+ - eta^-,
// which it equals, instead of as a difference of two large depths.
// Dry elements (the positivity pass's flag) take the depth form instead:
// p_d = g/2 h'^2 and source -g h' grad B', h' = eta' - B'. It differs from
// p'', -g eta' grad B' by the static pair -g/2 B'^2, -g B' grad B', whose volume,
// own-side face and source terms cancel exactly; with it a uniform film on a
// slope (h' = 0) has no cancelling terms left, as a lake at rest (eta' = 0) has
// none in the surface form. With md = 1 for the depth form, 0 for the surface
// form: p = g/2 (eta' - md B')(eta' - (2 - md) B'), source -g (eta' - md B') grad B'.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernel_types.hpp"

namespace swe {

// --------------------------------------------------------------------------
// small helpers

__device__ __forceinline__ int level_of(const Sched& sc, int e) {
  int l = 1;
#pragma unroll
  for (int t = 1; t < kMaxLevels; ++t)
    if (t < sc.L && e >= sc.off[t]) l = t + 1;
  return l;
}

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int n = 4;
  __device__ __forceinline__ static void unpack(const float4& v, float* o) {
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
  __device__ __forceinline__ static float4 pack(const float* o) { return make_float4(o[0], o[1], o[2], o[3]); }
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int n = 2;
  __device__ __forceinline__ static void unpack(const double2& v, double* o) { o[0] = v.x; o[1] = v.y; }
  __device__ __forceinline__ static double2 pack(const double* o) { return make_double2(o[0], o[1]); }
};

// Load LEN (multiple of 16 bytes) consecutive values.
template <typename T, int LEN>
__device__ __forceinline__ void load_row(const T* __restrict__ p, T (&o)[LEN]) {
  using V = Vec16<T>;
  const typename V::type* pv = reinterpret_cast<const typename V::type*>(p);
#pragma unroll
  for (int k = 0; k < LEN / V::n; ++k) V::unpack(pv[k], &o[k * V::n]);
}

template <typename T, int LEN>
__device__ __forceinline__ void load_row_global(const T* __restrict__ p, T (&o)[LEN]) {
  using V = Vec16<T>;
  const typename V::type* pv = reinterpret_cast<const typename V::type*>(p);
#pragma unroll
  for (int k = 0; k < LEN / V::n; ++k) V::unpack(__ldg(pv + k), &o[k * V::n]);
}

template <typename T, int LEN>
__device__ __forceinline__ void load_row_m(const T* p, T (&o)[LEN]) {
  using V = Vec16<T>;
  const typename V::type* pv = reinterpret_cast<const typename V::type*>(p);
#pragma unroll
  for (int k = 0; k < LEN / V::n; ++k) V::unpack(pv[k], &o[k * V::n]);
}

template <typename T, int LEN>
__device__ __forceinline__ void store_row_global(T* __restrict__ p, const T (&o)[LEN]) {
  using V = Vec16<T>;
  typename V::type* pv = reinterpret_cast<typename V::type*>(p);
#pragma unroll
  for (int k = 0; k < LEN / V::n; ++k) pv[k] = V::pack(&o[k * V::n]);
}

// Node-major element access: node i of the element at p is p[i * ks]. LEN >= NP
// registers; the padding entries read as zero.
template <typename T, int NP, int LEN>
__device__ __forceinline__ void load_nodes(const T* __restrict__ p, size_t ks, T (&o)[LEN]) {
#pragma unroll
  for (int i = 0; i < LEN; ++i) o[i] = i < NP ? __ldg(p + i * ks) : T(0);
}

template <typename T, int NP, int LEN>
__device__ __forceinline__ void store_nodes(T* __restrict__ p, size_t ks, const T (&o)[LEN]) {
#pragma unroll
  for (int i = 0; i < NP; ++i) p[i * ks] = o[i];
}

// Reciprocal and square root: hardware approximations in FP32 (about 1-2 ulp, no
// slow-path branches), correctly rounded in FP64.
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
// sqrt of x >= 0; the floor keeps x = 0 at 0 (0 * finite) instead of 0 * inf
__device__ __forceinline__ float sqrt_nn(float x) { return x * rsqrtf(fmaxf(x, 1e-30f)); }
__device__ __forceinline__ double sqrt_nn(double x) { return sqrt(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return 1.0 / sqrt(x); }

// Cache hints: start a line's trip from memory early, without holding registers.
// Only addresses inside live buffers are ever passed.
__device__ __forceinline__ void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Loads of the arrays the kernels write (state, Adams-Bashforth history, half-step
// records, means, dry flags, P1 values): ordinary coherent global loads, never the
// read-only data path. Inside the persistent batch kernel other CTAs of the same
// launch wrote these arrays in earlier phases, and an ordinary load after the
// acquire of the phase counter sees their stores. The separate launches use the
// same loads, so both compile the stage and limiter bodies to the same code and a
// scenario's result is the same, bit for bit, alone and in a batch.
template <typename T>
__device__ __forceinline__ T ldm(const T* p) {
  return *p;
}

template <typename T, int NP, int LEN>
__device__ __forceinline__ void load_nodes_m(const T* p, size_t ks, T (&o)[LEN]) {
#pragma unroll
  for (int i = 0; i < LEN; ++i) o[i] = i < NP ? ldm(p + i * ks) : T(0);
}

template <typename T>
__device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }
template <typename T>
__device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }

// Adams-Bashforth weights (equal steps) for R^(0), R^(-1), R^(-2), in the
// kernel's precision (no FP64 work on the FP32 path).
template <typename T>
__device__ __forceinline__ void ab_weights(int depth, T w[3]) {
  if (depth <= 1) { w[0] = T(1); w[1] = T(0); w[2] = T(0); }
  else if (depth == 2) { w[0] = T(1.5); w[1] = T(-0.5); w[2] = T(0); }
  else { w[0] = T(23) / T(12); w[1] = T(-16) / T(12); w[2] = T(5) / T(12); }
}

// Integral over [0, theta] of the Lagrange interpolant of R at tau = 0, -1, -2.
template <typename T>
__device__ __forceinline__ void ab_partial_weights(int depth, T t, T w[3]) {
  if (depth <= 1) { w[0] = t; w[1] = T(0); w[2] = T(0); }
  else if (depth == 2) { w[0] = t + T(0.5) * t * t; w[1] = T(-0.5) * t * t; w[2] = T(0); }
  else {
    const T t2 = t * t, t3 = t2 * t;
    w[0] = t3 / T(6) + T(0.75) * t2 + t;
    w[1] = -(t3 / T(3) + t2);
    w[2] = t3 / T(6) + T(0.25) * t2;
  }
}

__device__ __forceinline__ float level_dt(const Sched& sc, int l, float) { return sc.dtl_f[l - 1]; }
__device__ __forceinline__ double level_dt(const Sched& sc, int l, double) { return sc.dtl_d[l - 1]; }
__device__ __forceinline__ float eps_of(const Phys& ph, float) { return ph.eps_f; }
__device__ __forceinline__ double eps_of(const Phys& ph, double) { return ph.eps; }

__host__ __device__ constexpr int face_node(int N, int f, int m) {
  // node index of position m along face f (from vertex f to f+1), lattice order
  return f == 0 ? m : (f == 1 ? m * (N + 1) - m * (m - 1) / 2 + (N - m)
                               : (N - m) * (N + 1) - (N - m) * (N - m - 1) / 2);
}

__device__ __forceinline__ int face_node_rt(int N, int f, int m) { return face_node(N, f, m); }

// Stage the first S entries of the operator block into shared memory (all threads
// of the CTA): the whole block for the SIMT stage kernel, the per-element
// operators [0, TAIL) for the limiter kernels.
template <typename T, int N, int S = OpLayout<N>::SIZE>
__device__ __forceinline__ void stage_ops(T* sops, const T* __restrict__ gops) {
  using V = Vec16<T>;
  const typename V::type* src = reinterpret_cast<const typename V::type*>(gops);
  typename V::type* dst = reinterpret_cast<typename V::type*>(sops);
  for (int i = threadIdx.x; i < S / V::n; i += blockDim.x) dst[i] = __ldg(src + i);
  __syncthreads();
}

// --------------------------------------------------------------------------
// the well-balanced local Lax-Friedrichs flux (pre-balanced form), own side "-"

// Traces at a face point relative to the face's reference point (Ef, Bf): surface
// e = eta - Ef, bed b = B - Bf, and the momenta.
template <typename T>
struct Trace {
  T e, hu, hv, b;
};

// (nx, ny) unit outward normal, (vx, vy) = (sJ/J) (nx, ny), hs = sJ/J / 2; the
// returned fluxes are already scaled by sJ/J for the lift. hg = g/2, qg = g/4.
// hf = Ef - Bf, the depth at the face's reference point, so depths are
// hf + (e - b) without cancelling two large values. epm, bpm: eta^- and B^-
// relative to the element's own eta0, B0; the own-side pressure is p'' or p_d by
// md (element reference split above).
template <typename T>
__device__ __forceinline__ void wb_flux(const Trace<T>& m, const Trace<T>& p, T hf, T epm, T bpm, T md, T nx,
                                        T ny, T vx, T vy, T hs, T g, T hg, T qg, T hvel, T& f0, T& f1, T& f2) {
  const T hm = hf + (m.e - m.b), hp = hf + (p.e - p.b);
  const T im = hm > hvel ? recip(hm) : T(0), ip = hp > hvel ? recip(hp) : T(0);
  const T um = m.hu * im, vm = m.hv * im;
  const T up = p.hu * ip, vp = p.hv * ip;
  const T bmax = tmax(m.b, p.b);
  // hydrostatically reconstructed depths and the normal mass fluxes they carry
  const T sm = tmax(T(0), hf + (m.e - bmax)), sp = tmax(T(0), hf + (p.e - bmax));
  const T unm = um * nx + vm * ny, unp = up * nx + vp * ny;
  const T lam = tmax(fabs(unm) + sqrt_nn(g * sm), fabs(unp) + sqrt_nn(g * sp));
  const T Fm = sm * unm, Fp = sp * unp;
  const T ds = (sm > T(0) && sp > T(0)) ? p.e - m.e : sp - sm;
  const T pres = hg * (epm - md * bpm) * (epm - (T(2) - md) * bpm) + qg * ds * (sp + sm);
  f0 = hs * ((Fm + Fp) - lam * ds);
  f1 = hs * ((Fm * um + Fp * up) - lam * (sp * up - sm * um)) + pres * vx;
  f2 = hs * ((Fm * vm + Fp * vp) - lam * (sp * vp - sm * vm)) + pres * vy;
}

// --------------------------------------------------------------------------
// positivity-preserving limiter (Algorithm 3) on an element held in registers.
// Trigger test, means and rescale in FP64 when the element needs limiting;
// returns the dry classification and the element means (eta, hu, hv).

template <typename T, int N>
__device__ __forceinline__ int positivity(T (&eta)[Dims<N>::NPP], T (&hu)[Dims<N>::NPP],
                                          T (&hv)[Dims<N>::NPP], const T (&bb)[Dims<N>::NPP],
                                          const T* __restrict__ sops, double Bbar, T rx, T ry, T sx,
                                          T sy, const Phys& ph, double* injected, T mean_out[3]) {
  using D = Dims<N>;
  using O = OpLayout<N>;
  const T* mw = sops + O::MW;
  T hmin = eta[0] - bb[0];
#pragma unroll
  for (int jn = 1; jn < D::NP; ++jn) hmin = tmin(hmin, eta[jn] - bb[jn]);
  const bool trig = ph.pp && (hmin <= eps_of(ph, T(0)));
  if (!trig) {
    T me = 0, mu = 0, mv = 0;
#pragma unroll
    for (int jn = 0; jn < D::NP; ++jn) {
      me += mw[jn] * eta[jn];
      mu += mw[jn] * hu[jn];
      mv += mw[jn] * hv[jn];
    }
    mean_out[0] = me; mean_out[1] = mu; mean_out[2] = mv;
    return 0;
  }
  double hbar = 0.0, hub = 0.0, hvb = 0.0;
#pragma unroll
  for (int jn = 0; jn < D::NP; ++jn) {
    const double w = (double)mw[jn];
    hbar += w * ((double)eta[jn] - (double)bb[jn]);
    hub += w * (double)hu[jn];
    hvb += w * (double)hv[jn];
  }
  const double h0 = ph.h0;
  if (hbar < 1.01 * h0) {  // dry (the 1% margin keeps a reset element dry under rounding)
    const double hn = ph.dry_mode ? hbar : h0;
#pragma unroll
    for (int jn = 0; jn < D::NP; ++jn) {
      eta[jn] = (T)(hn + (double)bb[jn]);
      hu[jn] = T(0);
      hv[jn] = T(0);
    }
    const double area = 2.0 / ((double)rx * (double)sy - (double)ry * (double)sx);
    *injected += area * (hn - hbar);
    mean_out[0] = (T)(hn + Bbar); mean_out[1] = T(0); mean_out[2] = T(0);
    return 1;
  }
  // P1 projection at the vertices (FP64), theta rescale toward the mean
  const T* t1 = sops + O::T1;
  double vh[3], vu[3], vv[3];
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    double a = 0, b = 0, c = 0;
#pragma unroll
    for (int jn = 0; jn < D::NP; ++jn) {
      const double w = (double)t1[v * D::NPP + jn];
      a += w * ((double)eta[jn] - (double)bb[jn]);
      b += w * (double)hu[jn];
      c += w * (double)hv[jn];
    }
    vh[v] = a; vu[v] = b; vv[v] = c;
  }
  const double h1min = fmin(vh[0], fmin(vh[1], vh[2]));
  const double den = hbar - h1min;
  const double theta = den > 0.0 ? fmin(1.0, (hbar - h0) / den) : 1.0;
  const T* bary = sops + O::BARY;
#pragma unroll
  for (int jn = 0; jn < D::NP; ++jn) {
    const double l0 = bary[jn * 4 + 0], l1 = bary[jn * 4 + 1], l2 = bary[jn * 4 + 2];
    const double h1 = l0 * vh[0] + l1 * vh[1] + l2 * vh[2];
    const double u1 = l0 * vu[0] + l1 * vu[1] + l2 * vu[2];
    const double w1 = l0 * vv[0] + l1 * vv[1] + l2 * vv[2];
    eta[jn] = (T)(theta * (h1 - hbar) + hbar + (double)bb[jn]);
    hu[jn] = (T)(theta * (u1 - hub) + hub);
    hv[jn] = (T)(theta * (w1 - hvb) + hvb);
  }
  mean_out[0] = (T)(hbar + Bbar); mean_out[1] = (T)hub; mean_out[2] = (T)hvb;
  return 0;
}

// Vertex values of Pi1 (eta, hu, hv) for the TVB limiter (Section 5.3), stored
// as planes p1[(3 field + vertex) * KS + e] by whoever last committed the state.
template <typename T, int N>
__device__ __forceinline__ void store_p1(T* __restrict__ p1, size_t ks, const T* __restrict__ sops,
                                         const T (&eta)[Dims<N>::NPP], const T (&hu)[Dims<N>::NPP],
                                         const T (&hv)[Dims<N>::NPP]) {
  using D = Dims<N>;
  const T* t1 = sops + OpLayout<N>::T1;
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    T s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
    for (int jn = 0; jn < D::NP; ++jn) {
      const T w = t1[v * D::NPP + jn];
      s0 += w * eta[jn];
      s1 += w * hu[jn];
      s2 += w * hv[jn];
    }
    p1[(0 + v) * ks] = s0;
    p1[(3 + v) * ks] = s1;
    p1[(6 + v) * ks] = s2;
  }
}

// Surface fluxes (Section 7.2) of element e: traces at the Gauss points of its
// three faces and the well-balanced flux, scaled by sJ/J; emit(f, gq, F0, F1, F2,
// vx, vy) receives the flux at Gauss point gq of face f and the face's (sJ/J) n. own(f, j) returns the element's
// own field f (eta, hu, hv, B) at node j, so the caller decides whether the state
// sits in registers or in shared memory. With kRolled the three faces run
// through one copy of the face code (own() must then accept run-time node
// indices); otherwise the face loop is unrolled.
template <typename T, int N, bool kRolled, typename Own, typename Emit>
__device__ __forceinline__ void surface_fluxes(const StageParams<T>& p, const T* __restrict__ sops, int e,
                                               long long k, const Own& own, T rx, T ry, T sx, T sy, T md,
                                               Emit&& emit) {
  using D = Dims<N>;
  using O = OpLayout<N>;
  constexpr int NP = D::NP, NPP = D::NPP, NFP = D::NFP, NG = D::NG;
  const Sched& sc = p.sc;
  const T g = (T)p.ph.g, hvel = (T)p.ph.hvel, hg = T(0.5) * g, qg = T(0.25) * g;
  const size_t ks = (size_t)sc.KS;
  const size_t fstride = (size_t)NP * ks;
  const size_t bstride = 3 * fstride;
  const int4 cn = __ldg(p.s.conn + e);
  const T E0 = own(0, 0), B0 = own(3, 0);
#pragma unroll (kRolled ? 1 : 3)
  for (int f = 0; f < 3; ++f) {
    // outward normal times sJ/J from the affine factors
    const T vxn = f == 0 ? -sx : (f == 1 ? rx + sx : -rx);
    const T vyn = f == 0 ? -sy : (f == 1 ? ry + sy : -ry);
    const T v2 = vxn * vxn + vyn * vyn;
    const T iv = rsqrt_t(v2);
    const T nx = vxn * iv, ny = vyn * iv, hs = T(0.5) * v2 * iv;
    // Neighbour face-node values in the NEIGHBOUR's own order: its trace at this
    // element's Gauss point gq is its own point NG-1-gq, evaluated below with the
    // same operands in the same order as the neighbour evaluates it, relative to
    // the same face reference (node 0 of the lower-numbered element of the pair),
    // so both sides of a face see bit-identical traces and take the same wet/dry
    // and velocity decisions (the mass flux stays exactly antisymmetric).
    T ne[NFP], nu[NFP], nv[NFP], nB[NFP];
    T Ef = E0, Bf = B0;   // face reference: the own node 0 unless the neighbour is lower
    const int nb = f == 0 ? cn.x : (f == 1 ? cn.y : cn.z);
    if (nb >= 0) {
      const int fn = (cn.w >> (2 * f)) & 3;
      const int ln = level_of(sc, nb);
      const long long an = k >> (ln - 1);
      const long long pern = 1LL << (ln - 1);
      const long long phase = k & (pern - 1);
      // A neighbour one level coarser is always half-way through its step here; it
      // wrote that half-step Adams-Bashforth state at its own commit.
      const bool half = 2 * phase == pern;
      const T* qn = half ? p.s.qmid + (size_t)nb * 3 * NPP : p.s.q + (size_t)(an & 1) * bstride + nb;
      const size_t sn = half ? 1 : ks, sf = half ? (size_t)NPP : fstride;   // node, field strides
#pragma unroll
      for (int m = 0; m < NFP; ++m) {
        const int jn = face_node_rt(Dims<N>::N, fn, m);
        const size_t idx = (size_t)jn * sn;
        ne[m] = ldm(qn + idx);
        nu[m] = ldm(qn + sf + idx);
        nv[m] = ldm(qn + 2 * sf + idx);
        nB[m] = __ldg(p.s.B + nb + (size_t)jn * ks);
      }
      if (phase == 0 && nb < e) {   // an active neighbour numbered lower: its node 0
        Ef = ldm(qn);
        Bf = __ldg(p.s.B + nb);
      }
      if (phase != 0 && !half) {  // other fractions: Adams-Bashforth polynomial at t_k
        const int depth = an + 1 < 3 ? (int)(an + 1) : 3;
        T w[3];
        ab_partial_weights<T>(depth, (T)phase / (T)pern, w);
        const T dtn = level_dt(sc, ln, T(0));
        for (int s = 0; s < depth; ++s) {
          const T ws = dtn * w[s];
          const T* rs = p.s.ring + (size_t)((an - s) % 3) * bstride + nb;
#pragma unroll
          for (int m = 0; m < NFP; ++m) {
            const size_t idx = (size_t)face_node_rt(Dims<N>::N, fn, m) * ks;
            ne[m] += ws * ldm(rs + idx);
            nu[m] += ws * ldm(rs + fstride + idx);
            nv[m] += ws * ldm(rs + 2 * fstride + idx);
          }
        }
      }
    }
    // own face-node values relative to the face reference, read once per face
    T oe[NFP], ou[NFP], ov[NFP], oB[NFP];
#pragma unroll
    for (int m = 0; m < NFP; ++m) {
      const int jn = face_node(Dims<N>::N, f, m);
      oe[m] = own(0, jn) - Ef;
      ou[m] = own(1, jn);
      ov[m] = own(2, jn);
      oB[m] = own(3, jn) - Bf;
    }
    if (nb >= 0) {
#pragma unroll
      for (int m = 0; m < NFP; ++m) {
        ne[m] -= Ef;
        nB[m] -= Bf;
      }
    }
    const T hf = Ef - Bf;               // depth at the face reference
    const T dE = Ef - E0, dB = Bf - B0; // face reference relative to the element's own
#pragma unroll 1
    for (int gq = 0; gq < NG; ++gq) {
      T i1[D::NFPP], i1n[D::NFPP];
      load_row<T, D::NFPP>(sops + O::I1D + gq * D::NFPP, i1);
      load_row<T, D::NFPP>(sops + O::I1D + (NG - 1 - gq) * D::NFPP, i1n);
      Trace<T> tm = {0, 0, 0, 0}, tp;
#pragma unroll
      for (int m = 0; m < NFP; ++m) {
        tm.e += i1[m] * oe[m];
        tm.hu += i1[m] * ou[m];
        tm.hv += i1[m] * ov[m];
        tm.b += i1[m] * oB[m];
      }
      if (nb >= 0) {
        tp = {0, 0, 0, 0};
#pragma unroll
        for (int m = 0; m < NFP; ++m) {
          tp.e += i1n[m] * ne[m];
          tp.hu += i1n[m] * nu[m];
          tp.hv += i1n[m] * nv[m];
          tp.b += i1n[m] * nB[m];
        }
      } else if (nb == kFarField) {  // far field: the constant state over the continued bed
        tp = {(T)p.ph.ff_h - hf + tm.b, (T)p.ph.ff_hu, (T)p.ph.ff_hv, tm.b};
      } else {  // reflecting wall: mirror the normal momentum
        const T mn = tm.hu * nx + tm.hv * ny;
        tp = {tm.e, tm.hu - T(2) * mn * nx, tm.hv - T(2) * mn * ny, tm.b};
      }
      T f0, f1, f2;
      wb_flux<T>(tm, tp, hf, tm.e + dE, tm.b + dB, md, nx, ny, vxn, vyn, hs, g, hg, qg, hvel, f0, f1, f2);
      emit(f, gq, f0, f1, f2, vxn, vyn);
    }
  }
}

// Surface term with the lift R -= L^g F (Section 7.2) applied in registers, point
// by point (the SIMT stage kernel).
template <typename T, int N, bool kRolled = false, typename Own>
__device__ __forceinline__ void surface_lift(const StageParams<T>& p, const T* __restrict__ sops, int e,
                                             long long k, const Own& own, T rx, T ry, T sx, T sy, T md,
                                             T (&R0)[Dims<N>::NP], T (&R1)[Dims<N>::NP],
                                             T (&R2)[Dims<N>::NP]) {
  using D = Dims<N>;
  constexpr int NP = D::NP, NPP = D::NPP, NG = D::NG;
  surface_fluxes<T, N, kRolled>(p, sops, e, k, own, rx, ry, sx, sy, md, [&](int f, int gq, T f0, T f1, T f2, T, T) {
    T lg[NPP];
    load_row<T, NPP>(sops + OpLayout<N>::LGT + (f * NG + gq) * NPP, lg);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      R0[i] -= lg[i] * f0;
      R1[i] -= lg[i] * f1;
      R2[i] -= lg[i] * f2;
    }
  });
}

// The reference part of the pressure and source in strong form (element
// reference split above): R_hu -= g h0 (r_x Dr + s_x Ds)(eta - eta0),
// R_hv -= g h0 (r_y Dr + s_y Ds)(eta - eta0), h0 = eta0 - B0 the depth at node 0.
template <typename T, int N>
__device__ __forceinline__ void add_reference_pressure(const T* __restrict__ sops, const T (&eta)[Dims<N>::NPP],
                                                       const T (&bb)[Dims<N>::NPP], T g, T rx, T ry, T sx,
                                                       T sy, T (&R1)[Dims<N>::NP], T (&R2)[Dims<N>::NP]) {
  using D = Dims<N>;
  using O = OpLayout<N>;
  constexpr int NP = D::NP, NPP = D::NPP;
  T d[NPP];
#pragma unroll
  for (int j = 0; j < NPP; ++j) d[j] = j < NP ? eta[j] - eta[0] : T(0);
  const T gb = -g * (eta[0] - bb[0]);
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    T dr[NPP], ds[NPP];
    load_row<T, NPP>(sops + O::DR + i * NPP, dr);
    load_row<T, NPP>(sops + O::DS + i * NPP, ds);
    T er = 0, es = 0;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      er += dr[j] * d[j];
      es += ds[j] * d[j];
    }
    R1[i] += gb * (rx * er + sx * es);
    R2[i] += gb * (ry * er + sy * es);
  }
}

// Adams-Bashforth commit (Algorithm 1) and positivity limiter (Algorithm 3) of
// element e (mode 0), or the R output in the caller's layout (mode 1). kComp: each
// field's increments are summed first and added to the state with the rounding
// error of the previous update taken back (a compensated sum, p.s.comp), so the
// single-precision state neither drifts in total mass nor accumulates its rounding
// step after step.
template <typename T, int N, bool kComp = false>
__device__ __forceinline__ void commit_and_limit(const StageParams<T>& p, const T* __restrict__ sops, int e,
                                                 int lev, long long a, T (&eta)[Dims<N>::NPP],
                                                 T (&hu)[Dims<N>::NPP], T (&hv)[Dims<N>::NPP],
                                                 const T (&bb)[Dims<N>::NPP], T rx, T ry, T sx, T sy,
                                                 const T (&R0)[Dims<N>::NP], const T (&R1)[Dims<N>::NP],
                                                 const T (&R2)[Dims<N>::NP], double* injected_acc) {
  using D = Dims<N>;
  constexpr int NP = D::NP, NPP = D::NPP;
  const Sched& sc = p.sc;
  const int K = sc.K;
  const int dst = (int)((a + 1) & 1);
  const size_t ks = (size_t)sc.KS;
  const size_t fstride = (size_t)NP * ks;
  const size_t bstride = 3 * fstride;
  double& injected = *injected_acc;
  if (p.mode == 1) {  // R only, caller layout
    const int ce = p.perm[e];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      p.out[((size_t)0 * K + ce) * NP + i] = R0[i];
      p.out[((size_t)1 * K + ce) * NP + i] = R1[i];
      p.out[((size_t)2 * K + ce) * NP + i] = R2[i];
    }
    return;
  }

  // ---- Adams-Bashforth commit (Algorithm 1) ----
  const int depth = a + 1 < 3 ? (int)(a + 1) : 3;
  T wab[3];
  ab_weights<T>(depth, wab);
  const T dtl = level_dt(sc, lev, T(0));
  const T c0 = dtl * wab[0], c1 = dtl * wab[1], c2 = dtl * wab[2];
  T* ring = p.s.ring;
  const size_t eo = (size_t)e;
  store_nodes<T, NP, NP>(ring + (size_t)(a % 3) * bstride + 0 * fstride + eo, ks, R0);
  store_nodes<T, NP, NP>(ring + (size_t)(a % 3) * bstride + 1 * fstride + eo, ks, R1);
  store_nodes<T, NP, NP>(ring + (size_t)(a % 3) * bstride + 2 * fstride + eo, ks, R2);
  // The same pass over the older R slots also gives the Adams-Bashforth
  // polynomial of this step at its middle, q(t_a + dt/2) = q + dt sum_s w_s(1/2)
  // R^(a-s) (Section 4), which an element with a finer neighbour stores for that
  // neighbour's next substep.
  T wh[3];
  ab_partial_weights<T>(depth, T(0.5), wh);
  const T m0 = dtl * wh[0], m1 = dtl * wh[1], m2 = dtl * wh[2];
  T x0[NP], x1[NP], x2[NP];
  T d0[kComp ? NP : 1], d1[kComp ? NP : 1], d2[kComp ? NP : 1];   // compensated: the increments
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    x0[i] = eta[i] + m0 * R0[i];
    x1[i] = hu[i] + m0 * R1[i];
    x2[i] = hv[i] + m0 * R2[i];
    if constexpr (kComp) {
      d0[i] = c0 * R0[i];
      d1[i] = c0 * R1[i];
      d2[i] = c0 * R2[i];
    } else {
      eta[i] += c0 * R0[i];
      hu[i] += c0 * R1[i];
      hv[i] += c0 * R2[i];
    }
  }
  for (int s = 1; s < depth; ++s) {
    const T cs = s == 1 ? c1 : c2, ms = s == 1 ? m1 : m2;
    const T* rs = ring + (size_t)((a - s) % 3) * bstride + eo;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      const T r0 = ldm(rs + i * ks), r1 = ldm(rs + fstride + i * ks);
      const T r2 = ldm(rs + 2 * fstride + i * ks);
      if constexpr (kComp) {
        d0[i] += cs * r0;
        d1[i] += cs * r1;
        d2[i] += cs * r2;
      } else {
        eta[i] += cs * r0;
        hu[i] += cs * r1;
        hv[i] += cs * r2;
      }
      x0[i] += ms * r0;
      x1[i] += ms * r1;
      x2[i] += ms * r2;
    }
  }
  if ((__ldg(reinterpret_cast<const int*>(p.s.conn + e) + 3) >> 12) & 1) {
    T* qm = p.s.qmid + eo * 3 * NPP;
    T row[NPP];
#pragma unroll
    for (int i = 0; i < NPP; ++i) row[i] = i < NP ? x0[i] : T(0);
    store_row_global<T, NPP>(qm, row);
#pragma unroll
    for (int i = 0; i < NPP; ++i) row[i] = i < NP ? x1[i] : T(0);
    store_row_global<T, NPP>(qm + NPP, row);
#pragma unroll
    for (int i = 0; i < NPP; ++i) row[i] = i < NP ? x2[i] : T(0);
    store_row_global<T, NPP>(qm + 2 * NPP, row);
  }
  if constexpr (kComp) {
    // q + d with the previous rounding error c taken back: y = d - c, t = q + y, and
    // the new error c = (t - q) - y (exact when |q| >= |y|). All previous errors are
    // read before the first new one is written, so the loads overlap.
    T* cp = p.s.comp + eo;
    T ce[NP], cu[NP], cv[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      ce[i] = ldm(cp + i * ks);
      cu[i] = ldm(cp + fstride + i * ks);
      cv[i] = ldm(cp + 2 * fstride + i * ks);
    }
    auto add = [&](T& q, T d, T c, T* cout) {
      const T y = d - c;
      const T t = q + y;
      *cout = (t - q) - y;
      q = t;
    };
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      add(eta[i], d0[i], ce[i], cp + i * ks);
      add(hu[i], d1[i], cu[i], cp + fstride + i * ks);
      add(hv[i], d2[i], cv[i], cp + 2 * fstride + i * ks);
    }
  }

  // ---- positivity limiter (Algorithm 3) and means ----
  T mean[3];
  const int dryf = positivity<T, N>(eta, hu, hv, bb, sops, __ldg(p.s.Bbar + e), rx, ry, sx, sy, p.ph,
                                    &injected, mean);
  if (!(isfinite((double)mean[0]) && isfinite((double)mean[1]) && isfinite((double)mean[2])))
    atomicOr(p.s.flags, 1);
  store_nodes<T, NP, NPP>(p.s.q + dst * bstride + 0 * fstride + eo, ks, eta);
  store_nodes<T, NP, NPP>(p.s.q + dst * bstride + 1 * fstride + eo, ks, hu);
  store_nodes<T, NP, NPP>(p.s.q + dst * bstride + 2 * fstride + eo, ks, hv);
  p.s.means[4 * (size_t)e + 0] = mean[0];
  p.s.means[4 * (size_t)e + 1] = mean[1];
  p.s.means[4 * (size_t)e + 2] = mean[2];
  p.s.dry[e] = (uint8_t)dryf;
  store_p1<T, N>(p.s.p1 + eo, ks, sops, eta, hu, hv);
}

// --------------------------------------------------------------------------
// the stage kernel: R(Q) for one element (volume + surface + lift), then the
// Adams-Bashforth commit and the positivity limiter (mode 0) or R only (mode 1)

// Volume term N(Q) (Section 7.1) of one element, accumulated into R: interpolate
// to the cubature points, volume flux and source there, project back.
template <typename T, int N>
__device__ __forceinline__ void volume_term(const T* __restrict__ sops, const T (&eta)[Dims<N>::NPP],
                                            const T (&hu)[Dims<N>::NPP], const T (&hv)[Dims<N>::NPP],
                                            const T (&bb)[Dims<N>::NPP], T rx, T ry, T sx, T sy, T md, T g,
                                            T hvel, T (&R0)[Dims<N>::NP], T (&R1)[Dims<N>::NP],
                                            T (&R2)[Dims<N>::NP]) {
  using D = Dims<N>;
  using O = OpLayout<N>;
  constexpr int NP = D::NP, NPP = D::NPP, NCUB = D::NCUB;
  const T hg = T(0.5) * g;
#pragma unroll 1
  for (int c = 0; c < NCUB; ++c) {
    T ic[NPP], icr[NPP], ics[NPP];
    load_row<T, NPP>(sops + O::IC + c * NPP, ic);
    load_row<T, NPP>(sops + O::ICR + c * NPP, icr);
    load_row<T, NPP>(sops + O::ICS + c * NPP, ics);
    // ec, bc, brc, bsc: of eta - eta0 and B - B0 (element reference split)
    T ec = 0, huc = 0, hvc = 0, bc = 0, brc = 0, bsc = 0;
#pragma unroll
    for (int jn = 0; jn < NP; ++jn) {
      const T ep = eta[jn] - eta[0], bp = bb[jn] - bb[0];
      ec += ic[jn] * ep;
      huc += ic[jn] * hu[jn];
      hvc += ic[jn] * hv[jn];
      bc += ic[jn] * bp;
      brc += icr[jn] * bp;
      bsc += ics[jn] * bp;
    }
    const T hc = (eta[0] - bb[0]) + (ec - bc);
    const T ih = hc > hvel ? recip(hc) : T(0);
    const T u = huc * ih, v = hvc * ih;
    // cF1 = rx F + ry G and cF2 = sx F + sy G, with the momentum rows written
    // through the mass row: rx (hu u + p) + ry hv u = u (rx hu + ry hv) + rx p;
    // p = p'' (element reference split)
    const T ep = ec - md * bc;
    const T pr = hg * ep * (ec - (T(2) - md) * bc);
    const T a0 = rx * huc + ry * hvc, b0 = sx * huc + sy * hvc;
    const T a1 = u * a0 + rx * pr, a2 = v * a0 + ry * pr;
    const T b1 = u * b0 + sx * pr, b2 = v * b0 + sy * pr;
    const T gm = -g * ep;
    const T S1 = gm * (rx * brc + sx * bsc), S2 = gm * (ry * brc + sy * bsc);
    T prt[NPP], pst[NPP], pt[NPP];
    load_row<T, NPP>(sops + O::PRT + c * NPP, prt);
    load_row<T, NPP>(sops + O::PST + c * NPP, pst);
    load_row<T, NPP>(sops + O::PT + c * NPP, pt);
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      R0[i] += prt[i] * a0 + pst[i] * b0;
      R1[i] += prt[i] * a1 + pst[i] * b1 + pt[i] * S1;
      R2[i] += prt[i] * a2 + pst[i] * b2 + pt[i] * S2;
    }
  }
}

// One element of the stage: R(Q) (volume + surface + lift), then the
// Adams-Bashforth commit and the positivity limiter (mode 0) or R only (mode 1).
// k is the finest substep count of the schedule; kComp: compensated state update.
template <typename T, int N, bool kComp = false>
__device__ __forceinline__ void stage_element(const StageParams<T>& p, const T* __restrict__ sops, int e,
                                              long long k, double* injected) {
  using D = Dims<N>;
  constexpr int NP = D::NP, NPP = D::NPP;
  const Sched& sc = p.sc;
  const T g = (T)p.ph.g, hvel = (T)p.ph.hvel;
  const size_t ks = (size_t)sc.KS;
  const size_t fstride = (size_t)NP * ks;            // between fields
  const size_t bstride = 3 * fstride;                // between buffers
  const int lev = level_of(sc, e);
  const long long a = k >> (lev - 1);
  const int src = (int)(a & 1);
  T eta[NPP], hu[NPP], hv[NPP], bb[NPP];
  load_nodes_m<T, NP, NPP>(p.s.q + src * bstride + 0 * fstride + e, ks, eta);
  load_nodes_m<T, NP, NPP>(p.s.q + src * bstride + 1 * fstride + e, ks, hu);
  load_nodes_m<T, NP, NPP>(p.s.q + src * bstride + 2 * fstride + e, ks, hv);
  load_nodes<T, NP, NPP>(p.s.B + e, ks, bb);
  const T rx = __ldg(p.s.geo + 4 * (size_t)e + 0), ry = __ldg(p.s.geo + 4 * (size_t)e + 1);
  const T sx = __ldg(p.s.geo + 4 * (size_t)e + 2), sy = __ldg(p.s.geo + 4 * (size_t)e + 3);
  // depth form of the pressure for dry elements; with inexact rules (collocation,
  // order 2N) the pre-balanced form everywhere (the two forms then differ)
  const T md = (Dims<N>::EXACT && ldm(p.s.dry + e)) ? T(1) : T(0);

  T R0[NP], R1[NP], R2[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) { R0[i] = 0; R1[i] = 0; R2[i] = 0; }

  // ---- volume term (Section 7.1): interpolate, flux + source, project ----
  volume_term<T, N>(sops, eta, hu, hv, bb, rx, ry, sx, sy, md, g, hvel, R0, R1, R2);

  auto own = [&](int f, int jn) -> T { return f == 0 ? eta[jn] : (f == 1 ? hu[jn] : (f == 2 ? hv[jn] : bb[jn])); };
  surface_lift<T, N, false>(p, sops, e, k, own, rx, ry, sx, sy, md, R0, R1, R2);
  add_reference_pressure<T, N>(sops, eta, bb, g, rx, ry, sx, sy, R1, R2);
  commit_and_limit<T, N, kComp>(p, sops, e, lev, a, eta, hu, hv, bb, rx, ry, sx, sy, R0, R1, R2, injected);
}

// Elements e0, e0 + step, ... below e1 of the stage; returns the mass the
// positivity limiter's dry resets injected (inlined by the separate launch and the
// persistent batch kernel alike).
template <typename T, int N, bool kComp = false>
__device__ __forceinline__ double stage_range(const StageParams<T>& __restrict__ p, const T* __restrict__ sops,
                                           int e0, int step, int e1, long long k) {
  double injected = 0.0;
  for (int e = e0; e < e1; e += step) stage_element<T, N, kComp>(p, sops, e, k, &injected);
  return injected;
}

// kGlobalOps: the operators are read from global memory (through L1) instead of
// the block's shared-memory copy (the operator-placement comparison of Section 7.4).
// kComp: compensated state update (p.s.comp).
template <typename T, int N, bool kGlobalOps = false, bool kComp = false>
__global__ void __launch_bounds__(kBlock) k_stage(const __grid_constant__ StageParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const T* sops;
  if constexpr (kGlobalOps) {
    sops = p.s.ops;
  } else {
    stage_ops<T, N>(reinterpret_cast<T*>(smem_raw), p.s.ops);
    sops = reinterpret_cast<const T*>(smem_raw);
  }
  const long long k = (*p.s.macro) * (1LL << (p.sc.L - 1)) + p.j;
  double injected;
  if constexpr (kGlobalOps) {
    injected = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p.nactive; e += gridDim.x * blockDim.x)
      stage_element<T, N>(p, sops, e, k, &injected);
  } else {
    injected = stage_range<T, N, kComp>(p, sops, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x,
                                        p.nactive, k);
  }
  if (injected != 0.0) atomicAdd(p.s.acc, injected);
}

// --------------------------------------------------------------------------
// positivity limiter on the current state (initial limiting, swe_limit)

template <typename T, int N>
__global__ void __launch_bounds__(kBlock) k_positivity(LimitParams<T> p) {
  using D = Dims<N>;
  constexpr int NP = D::NP, NPP = D::NPP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sops = reinterpret_cast<T*>(smem_raw);
  stage_ops<T, N, OpLayout<N>::TAIL>(sops, p.s.ops);
  const Sched& sc = p.sc;
  const long long k = (*p.s.macro) * (1LL << (sc.L - 1)) + p.j;
  const size_t ks = (size_t)sc.KS, fstride = (size_t)NP * ks, bstride = 3 * fstride;
  double injected = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p.nactive; e += gridDim.x * blockDim.x) {
    const int lev = level_of(sc, e);
    const long long a = k >> (lev - 1);
    const int cur = (int)((a + p.post_stage) & 1);
    const size_t eo = (size_t)e;
    T* q = p.s.q + cur * bstride;
    T eta[NPP], hu[NPP], hv[NPP], bb[NPP];
    load_nodes<T, NP, NPP>(q + eo, ks, eta);
    load_nodes<T, NP, NPP>(q + fstride + eo, ks, hu);
    load_nodes<T, NP, NPP>(q + 2 * fstride + eo, ks, hv);
    load_nodes<T, NP, NPP>(p.s.B + eo, ks, bb);
    const T rx = p.s.geo[4 * e], ry = p.s.geo[4 * e + 1], sx = p.s.geo[4 * e + 2], sy = p.s.geo[4 * e + 3];
    T mean[3];
    const int dryf = positivity<T, N>(eta, hu, hv, bb, sops, p.s.Bbar[e], rx, ry, sx, sy, p.ph, &injected, mean);
    store_nodes<T, NP, NPP>(q + eo, ks, eta);
    store_nodes<T, NP, NPP>(q + fstride + eo, ks, hu);
    store_nodes<T, NP, NPP>(q + 2 * fstride + eo, ks, hv);
    store_p1<T, N>(p.s.p1 + eo, ks, sops, eta, hu, hv);
    p.s.means[4 * (size_t)e + 0] = mean[0];
    p.s.means[4 * (size_t)e + 1] = mean[1];
    p.s.means[4 * (size_t)e + 2] = mean[2];
    p.s.dry[e] = (uint8_t)dryf;
    if (!(isfinite((double)mean[0]) && isfinite((double)mean[1]) && isfinite((double)mean[2])))
      atomicOr(p.s.flags, 1);
  }
  if (injected != 0.0) atomicAdd(p.s.acc, injected);
}

// --------------------------------------------------------------------------
// TVB limiter with the positivity modification (Section 5.3), P1 part of
// (eta, hu, hv), characteristic variables, midpoint deltas.

template <typename T>
__device__ __forceinline__ T minmod_tvb(T a, T b, T thr, bool& changed) {
  if (fabs(a) <= thr) return a;
  T r;
  if (a > 0 && b > 0) r = a < b ? a : b;
  else if (a < 0 && b < 0) r = a > b ? a : b;
  else r = T(0);
  if (r != a) changed = true;
  return r;
}

// The TVB limiter with the positivity modification on element e (k: the finest
// substep count of the schedule); returns without change for an element that is dry,
// has a dry neighbour or needs no limiting.
template <typename T, int N>
__device__ __forceinline__ void tvb_element(const ScnParams<T>& p, int post_stage, const T* __restrict__ sops,
                                            int e, long long k) {
  using D = Dims<N>;
  using O = OpLayout<N>;
  constexpr int NP = D::NP, NPP = D::NPP;
  const Sched& sc = p.sc;
  const T g = (T)p.ph.g, h0 = (T)p.ph.h0;
  {
    // Every load is issued before the first branch on loaded data (an element that is
    // dry or has a dry neighbour is skipped afterwards), so the latencies overlap:
    // two dependent trips to memory (connectivity, then the neighbours) instead of four.
    const int4 cn = __ldg(p.s.conn + e);
    const int de = ldm(p.s.dry + e);
    const int nbs[3] = {cn.x, cn.y, cn.z};
    const int lev = level_of(sc, e);
    const long long a = k >> (lev - 1);
    const int cur = (int)((a + post_stage) & 1);
    const size_t ks = (size_t)sc.KS, fstride = (size_t)NP * ks, bstride = 3 * fstride, eo = (size_t)e;
    T* q = p.s.q + cur * bstride;
    // 16-byte rows: geometry, element means (eta, hu, hv, -) as stored by the
    // positivity pass, the neighbour-mean weights
    T gm[4], u0[4], tg[8];
    load_row_global<T, 4>(p.s.geo + 4 * eo, gm);
    load_row_m<T, 4>(p.s.means + 4 * eo, u0);
    load_row_global<T, 8>(p.s.tvbg + 8 * eo, tg);
    // P1 part: vertex values of Pi1 q for eta, hu, hv (stored with the committed
    // state) and of Pi1 B (static)
    T vq[3][3], vb[3];
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      vq[0][v] = ldm(p.s.p1 + (0 + v) * ks + eo);
      vq[1][v] = ldm(p.s.p1 + (3 + v) * ks + eo);
      vq[2][v] = ldm(p.s.p1 + (6 + v) * ks + eo);
      vb[v] = __ldg(p.s.vb + v * ks + eo);
    }
    // neighbour means and dry flags
    T un[3][4];
    int dn = 0;
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      const int nb = nbs[f];
      if (nb >= 0) {
        dn |= ldm(p.s.dry + nb);
        load_row_m<T, 4>(p.s.means + 4 * (size_t)nb, un[f]);
      }
    }
    if (de || dn) return;
    const T rx = gm[0], ry = gm[1], sx = gm[2], sy = gm[3];
    // a far-field face sees the far-field state over the own mean bed; a wall face
    // mirrors the normal momentum of the own mean
    const T Bbar_e = (T)p.s.Bbar[e];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      if (nbs[f] == kFarField) {
        un[f][0] = (T)p.ph.ff_h + Bbar_e;
        un[f][1] = (T)p.ph.ff_hu;
        un[f][2] = (T)p.ph.ff_hv;
      } else if (nbs[f] < 0) {
        const T vxn = f == 0 ? -sx : (f == 1 ? rx + sx : -rx);
        const T vyn = f == 0 ? -sy : (f == 1 ? ry + sy : -ry);
        const T sn = sqrt(vxn * vxn + vyn * vyn);
        const T nx = vxn / sn, ny = vyn / sn;
        const T mn = u0[1] * nx + u0[2] * ny;
        un[f][0] = u0[0];
        un[f][1] = u0[1] - T(2) * mn * nx;
        un[f][2] = u0[2] - T(2) * mn * ny;
      }
    }
    // physical midpoint-minus-centroid vectors from the affine map
    const T Jd = T(1) / (rx * sy - ry * sx);
    const T xr = Jd * sy, xs = -Jd * ry, yr = -Jd * sx, ys = Jd * rx;
    const T dr[3] = {T(1) / 3, T(1) / 3, T(-2) / 3}, ds[3] = {T(-2) / 3, T(1) / 3, T(1) / 3};
    const T Bbar = Bbar_e;
    const T hb = u0[0] - Bbar;
    const T cb = sqrt(g * hb);
    const T ub = u0[1] / hb, vb0 = u0[2] / hb;
    const T floor = T(1e-6) * (hb + sqrt(u0[1] * u0[1] + u0[2] * u0[2]) / cb);
    const T M = (T)p.ph.tvb_M, nu = (T)p.ph.tvb_nu;
    bool changed = false;
    T dl[3][3];  // limited deltas, [edge][field]
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int jj = (cn.w >> (6 + 2 * i)) & 3;
      const T al = tg[2 * i], be = tg[2 * i + 1];
      T dt_[3], dn[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        dt_[c] = T(0.5) * (vq[c][i] + vq[c][(i + 1) % 3]) - u0[c];
        const T uj = jj == 0 ? un[0][c] : (jj == 1 ? un[1][c] : un[2][c]);   // selects, no local array
        dn[c] = al * (un[i][c] - u0[c]) + be * (uj - u0[c]);
      }
      const T mx = xr * dr[i] + xs * ds[i], my = yr * dr[i] + ys * ds[i];
      const T dist = sqrt(mx * mx + my * my);
      const T nx = mx / dist, ny = my / dist;
      // right eigenvectors (columns) and their inverse
      const T Rm[3][3] = {{T(1), T(0), T(1)},
                          {ub - cb * nx, -ny, ub + cb * nx},
                          {vb0 - cb * ny, nx, vb0 + cb * ny}};
      const T det = Rm[0][0] * (Rm[1][1] * Rm[2][2] - Rm[1][2] * Rm[2][1]) -
                    Rm[0][1] * (Rm[1][0] * Rm[2][2] - Rm[1][2] * Rm[2][0]) +
                    Rm[0][2] * (Rm[1][0] * Rm[2][1] - Rm[1][1] * Rm[2][0]);
      const T id = T(1) / det;
      T Lm[3][3];
      Lm[0][0] = (Rm[1][1] * Rm[2][2] - Rm[1][2] * Rm[2][1]) * id;
      Lm[0][1] = (Rm[0][2] * Rm[2][1] - Rm[0][1] * Rm[2][2]) * id;
      Lm[0][2] = (Rm[0][1] * Rm[1][2] - Rm[0][2] * Rm[1][1]) * id;
      Lm[1][0] = (Rm[1][2] * Rm[2][0] - Rm[1][0] * Rm[2][2]) * id;
      Lm[1][1] = (Rm[0][0] * Rm[2][2] - Rm[0][2] * Rm[2][0]) * id;
      Lm[1][2] = (Rm[0][2] * Rm[1][0] - Rm[0][0] * Rm[1][2]) * id;
      Lm[2][0] = (Rm[1][0] * Rm[2][1] - Rm[1][1] * Rm[2][0]) * id;
      Lm[2][1] = (Rm[0][1] * Rm[2][0] - Rm[0][0] * Rm[2][1]) * id;
      Lm[2][2] = (Rm[0][0] * Rm[1][1] - Rm[0][1] * Rm[1][0]) * id;
      const T thr0 = M * dist * dist + floor;
      T wl[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T wt = Lm[c][0] * dt_[0] + Lm[c][1] * dt_[1] + Lm[c][2] * dt_[2];
        const T wn = Lm[c][0] * dn[0] + Lm[c][1] * dn[1] + Lm[c][2] * dn[2];
        wl[c] = minmod_tvb<T>(wt, nu * wn, c == 1 ? thr0 * cb : thr0, changed);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) dl[i][c] = Rm[c][0] * wl[0] + Rm[c][1] * wl[1] + Rm[c][2] * wl[2];
    }
    if (!changed) return;
    // redistribution: deltas of each field sum to zero
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T pos = 0, neg = 0;
#pragma unroll
      for (int i = 0; i < 3; ++i) { pos += tmax(dl[i][c], T(0)); neg += tmax(-dl[i][c], T(0)); }
      const T tp = pos > 0 ? tmin(T(1), neg / pos) : T(1);
      const T tn = neg > 0 ? tmin(T(1), pos / neg) : T(1);
#pragma unroll
      for (int i = 0; i < 3; ++i) dl[i][c] = tp * tmax(dl[i][c], T(0)) - tn * tmax(-dl[i][c], T(0));
    }
    // depth deltas = eta deltas minus those of Pi1 B; positivity modification (Eq. modified_TVB)
    T dh[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) dh[i] = dl[i][0] - (T(0.5) * (vb[i] + vb[(i + 1) % 3]) - Bbar);
    T S[3] = {dh[0] + dh[2] - dh[1], dh[1] + dh[0] - dh[2], dh[2] + dh[1] - dh[0]};
    const T smin = tmin(S[0], tmin(S[1], S[2]));
    if (hb + smin < h0) {
      const T dbar = (dh[0] + dh[1] + dh[2]) / T(3);
      const T den = dbar - smin;
      T th = den > 0 ? (hb + dbar - h0) / den : T(1);
      th = tmin(T(1), tmax(T(0), th));
#pragma unroll
      for (int i = 0; i < 3; ++i) dh[i] = dbar + th * (dh[i] - dbar);
    }
    // vertex values and the P1 rebuild at the nodes
    T vh[3], vu[3], vv[3];
    vh[0] = hb + dh[0] + dh[2] - dh[1]; vh[1] = hb + dh[1] + dh[0] - dh[2]; vh[2] = hb + dh[2] + dh[1] - dh[0];
    vu[0] = u0[1] + dl[0][1] + dl[2][1] - dl[1][1];
    vu[1] = u0[1] + dl[1][1] + dl[0][1] - dl[2][1];
    vu[2] = u0[1] + dl[2][1] + dl[1][1] - dl[0][1];
    vv[0] = u0[2] + dl[0][2] + dl[2][2] - dl[1][2];
    vv[1] = u0[2] + dl[1][2] + dl[0][2] - dl[2][2];
    vv[2] = u0[2] + dl[2][2] + dl[1][2] - dl[0][2];
    const T* bary = sops + O::BARY;
    T fld[3][NPP], bb[NPP];
    load_nodes<T, NP, NPP>(p.s.B + eo, ks, bb);
    if constexpr (sizeof(T) == 4) {
      // Single precision: rebuild about the means, eta = eta-bar + sum_v l_v S_v +
      // (B - B-bar) with S_v the vertex deltas. The stored barycentric weights sum to
      // one only to rounding (2^-25 at worst), so sum_v l_v (h-bar + S_v) would scale
      // every rebuilt element's mean by that sum; about the mean the rounding is of
      // the size of the deltas, not of the depth.
      const T Sh[3] = {dh[0] + dh[2] - dh[1], dh[1] + dh[0] - dh[2], dh[2] + dh[1] - dh[0]};
      const T Su[3] = {dl[0][1] + dl[2][1] - dl[1][1], dl[1][1] + dl[0][1] - dl[2][1],
                       dl[2][1] + dl[1][1] - dl[0][1]};
      const T Sv[3] = {dl[0][2] + dl[2][2] - dl[1][2], dl[1][2] + dl[0][2] - dl[2][2],
                       dl[2][2] + dl[1][2] - dl[0][2]};
#pragma unroll
      for (int jn = 0; jn < NP; ++jn) {
        const T l0 = bary[4 * jn], l1 = bary[4 * jn + 1], l2 = bary[4 * jn + 2];
        fld[0][jn] = u0[0] + (l0 * Sh[0] + l1 * Sh[1] + l2 * Sh[2]) + (bb[jn] - Bbar);
        fld[1][jn] = u0[1] + (l0 * Su[0] + l1 * Su[1] + l2 * Su[2]);
        fld[2][jn] = u0[2] + (l0 * Sv[0] + l1 * Sv[1] + l2 * Sv[2]);
      }
    } else {
#pragma unroll
      for (int jn = 0; jn < NP; ++jn) {
        const T l0 = bary[4 * jn], l1 = bary[4 * jn + 1], l2 = bary[4 * jn + 2];
        fld[0][jn] = l0 * vh[0] + l1 * vh[1] + l2 * vh[2] + bb[jn];
        fld[1][jn] = l0 * vu[0] + l1 * vu[1] + l2 * vu[2];
        fld[2][jn] = l0 * vv[0] + l1 * vv[1] + l2 * vv[2];
      }
    }
    store_nodes<T, NP, NPP>(q + eo, ks, fld[0]);
    store_nodes<T, NP, NPP>(q + fstride + eo, ks, fld[1]);
    store_nodes<T, NP, NPP>(q + 2 * fstride + eo, ks, fld[2]);
  }
}

// Elements e0, e0 + step, ... below e1 of the TVB limiter (post_stage: 1 limits the
// just-committed state, 0 the current one). Out of line: the
// separate launch and the persistent batch kernel then run one compiled copy of its
// arithmetic (its many short multiply-add chains were rounded differently when it
// was inlined into the two kernels), at no measured cost.
template <typename T, int N>
__device__ __noinline__ void tvb_range(const ScnParams<T>& __restrict__ p, int post_stage,
                                       const T* __restrict__ sops, int e0, int step, int e1, long long k) {
  for (int e = e0; e < e1; e += step) tvb_element<T, N>(p, post_stage, sops, e, k);
}

template <typename T, int N>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? 6 : 3) k_tvb(const __grid_constant__ LimitParams<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sops = reinterpret_cast<T*>(smem_raw);
  stage_ops<T, N, OpLayout<N>::TAIL>(sops, p.s.ops);
  const long long k = (*p.s.macro) * (1LL << (p.sc.L - 1)) + p.j;
  tvb_range<T, N>(p, p.post_stage, sops, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, p.nactive,
                  k);
}

}  // namespace swe
