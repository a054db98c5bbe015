// Solver state, workspace layout, multirate schedule, CUDA-graph capture and the
// C ABI declared in include/swe.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/swe.h"
#include "launch.hpp"
#include "mesh.hpp"
#include "refelem.hpp"

struct swe_mesh {
  swe::Mesh m;
};

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define SWE_CUDA(call)                                                                        \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(SWE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));             \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// The CFL rule (element_dt) needs a finite nodal state with some positive depth:
// its maxima would pass over a NaN operand, and with no positive depth there is no
// wave speed to bound the step. nonfinite_code: what a non-finite value returns.
int check_cfl_input(const double* h, const double* hu, const double* hv, size_t n, int nonfinite_code) {
  bool wet = false;
  for (size_t i = 0; i < n; ++i) {
    if (!std::isfinite(h[i]) || !std::isfinite(hu[i]) || !std::isfinite(hv[i]))
      return fail(nonfinite_code, "non-finite state: the CFL rule needs finite values");
    wet = wet || h[i] > 0.0;
  }
  if (!wet) return fail(SWE_EINVAL, "no positive depth: the CFL rule has no wave speed");
  return SWE_OK;
}

int npp_of(int N) {
  int np = (N + 1) * (N + 2) / 2;
  return (np + 3) / 4 * 4;
}

int np_of(int N) { return (N + 1) * (N + 2) / 2; }

// element stride of the node-major planes: whole 128-byte lines per 32 elements
int ks_of(int K) { return (K + 31) / 32 * 32; }

struct Layout {
  size_t comp, q, ring, qmid, B, p1, vb, xfer, bcaller, iperm, xflag, geo, conn, tvbg, means, dry, Bbar, ops, tcops, perm, acc, flags, macro, partials, total;
  int nb_stats;
};

int tc_size_of(int N);

// comp: the compensation planes of the state, [3][NP][KS] (single-precision tiers
// with compensated = 1), else empty
Layout make_layout(int K, int N, size_t ts, int op_size, int code, bool comp) {
  Layout L;
  const size_t plane = (size_t)np_of(N) * (size_t)ks_of(K);   // one field, all nodes
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  L.q = take(2 * 3 * plane * ts);
  L.ring = take(3 * 3 * plane * ts);
  L.qmid = take((size_t)K * 3 * npp_of(N) * ts);
  L.B = take(plane * ts);
  L.p1 = take(9 * (size_t)ks_of(K) * ts);
  L.vb = take(3 * (size_t)ks_of(K) * ts);
  L.xfer = take(3 * (size_t)K * np_of(N) * 8);      // caller-layout FP64 staging of the state
  L.bcaller = take((size_t)K * np_of(N) * 8);       // the bed in caller order, FP64
  L.iperm = take((size_t)K * 4);
  L.xflag = take(16);
  L.geo = take((size_t)K * 4 * ts);
  L.conn = take((size_t)K * 16);
  L.tvbg = take((size_t)K * 8 * ts);
  L.means = take((size_t)K * 4 * ts);
  L.dry = take((size_t)K);
  L.Bbar = take((size_t)K * 8);
  L.ops = take((size_t)op_size * ts);
  L.tcops = take((size_t)tc_size_of(code) * 4);
  L.perm = take((size_t)K * 4);
  L.acc = take(8 * 8);
  L.flags = take(4 * 4);
  L.macro = take(8);
  L.comp = take(comp ? 3 * plane * ts : 0);
  L.nb_stats = std::max(1, std::min(1024, (K + 255) / 256));
  L.partials = take((size_t)L.nb_stats * 2 * 8 + 16);
  L.total = off;
  return L;
}

int check_params(const swe_params* p) {
  if (!p) return fail(SWE_EINVAL, "params is NULL");
  if (p->N < 1 || p->N > 5) return fail(SWE_EUNSUPPORTED, "this build supports N = 1..5");
  if (p->N == 1 && p->scheme != SWE_SCHEME_CUBATURE)
    return fail(SWE_EUNSUPPORTED, "N = 1 is built for the default scheme only");
  if (p->precision != SWE_FP64 && p->precision != SWE_FP32 && p->precision != SWE_FP32_TC)
    return fail(SWE_EUNSUPPORTED, "precision must be SWE_FP64, SWE_FP32 or SWE_FP32_TC");
  if (!(p->g > 0) || !(p->h0 > 0) || !(p->cfl > 0)) return fail(SWE_EINVAL, "g, h0 and cfl must be > 0");
  if (p->nlevels_max < 1 || p->nlevels_max > swe::kMaxLevels)
    return fail(SWE_EINVAL, "nlevels_max must be in 1..8");
  if (p->limiter_mask & ~3) return fail(SWE_EINVAL, "unknown limiter bits");
  if (p->scheme != SWE_SCHEME_CUBATURE && p->scheme != SWE_SCHEME_COLLOCATION &&
      p->scheme != SWE_SCHEME_CUBATURE_2N)
    return fail(SWE_EINVAL, "unknown scheme");
  if (p->compensated != 0 && p->compensated != 1) return fail(SWE_EINVAL, "compensated must be 0 or 1");
  return SWE_OK;
}

int scheme_code(const swe_params* p) {
  return p->N + (p->scheme == SWE_SCHEME_COLLOCATION ? swe::kColloc : 0) +
         (p->scheme == SWE_SCHEME_CUBATURE_2N ? swe::kReduced : 0);
}

// Base class so the C handle does not depend on the precision.
struct SolverBase {
  virtual ~SolverBase() {}
};

}  // namespace

struct swe_solver {
  swe::Mesh mesh;
  swe_params prm;
  swe::RefElem ref;
  int N = 0, K = 0, Np = 0, NPP = 0;
  int code = 0;                  // N, plus swe::kColloc for the nodal-collocation scheme
  int KS = 0;                    // element stride of the device node planes
  bool fp64 = false;
  bool tc = false;   // FP32 with tensor-core volume contractions
  bool comp = false; // single precision with a compensated state update
  size_t ts = 4;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  Layout lay;
  swe::KernelCfg cfg;
  int ctas_per_sm = 0;           // cap of swe_set_launch_config (0 = as many as fit)
  const swe::Launchers<float>* lf = nullptr;
  const swe::Launchers<double>* ld = nullptr;
  // host copies
  std::vector<double> B_in;      // caller order, as given
  std::vector<double> B_dev;     // caller order, device-precision values
  bool have_B = false, have_state = false, have_levels = false;
  std::vector<int32_t> level;    // caller order
  std::vector<int32_t> perm;     // device index -> caller index
  std::vector<int32_t> iperm;    // caller index -> device index
  int L = 1;
  std::vector<int> off;          // size L+1
  double dt_min = 0.0;
  int64_t k = 0;                 // finest substeps since the last restart
  double t0 = 0.0;               // time at the last restart
  int64_t dof_updates = 0;
  int64_t launches = 0;
  cudaGraphExec_t graph = nullptr;
  uint64_t sched_version = 0;    // bumped whenever captured launches go stale (levels, order, launch shape)
  double ff[3] = {0.0, 0.0, 0.0};   // far-field state of the open boundary faces
  std::vector<uint8_t> open_face;   // K x 3, caller order: 1 = open (far field), 0 = wall
  int graph_launches = 0;
  int64_t graph_dofs = 0;
  swe::KernelCfg cfg_max;   // occupancy limits (set_launch_config caps below these)
};

// One persistent kernel's scenarios: the same precision tier and scheme code.
struct BatchGroup {
  bool fp64 = false, tc = false;
  int code = 0;
  std::vector<int> idx;              // solvers of the batch in this group
  size_t off_ctl = 0, off_segs = 0, off_cnt = 0, off_release = 0, off_nmacro = 0, off_segof = 0;
  int seg_cap = 0;
  int ticket_cap = 0;
  std::vector<int> seg_of;           // host copy of this call's ticket -> segment table
  int grid = 0;
  cudaStream_t stream = nullptr;     // its branch of the captured graph
  cudaEvent_t join = nullptr;
  std::vector<swe::BatchSeg> segs;   // host copy of this call's ticket segments
};

struct swe_batch {
  std::vector<swe_solver*> solvers;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  int max_macro = 1;
  double wait_s = 10.0;
  std::vector<BatchGroup> groups;
  std::vector<int32_t> hold;          // per solver: withhold its release
  std::vector<int32_t> last_nmacro;   // the segment tables were built for these
  cudaGraphExec_t graph = nullptr;
  cudaEvent_t fork = nullptr, done = nullptr;
  std::vector<cudaEvent_t> join;      // per solver: work queued on its own stream
  std::vector<int64_t> dofs;          // per solver: DOF updates of one macro step
  std::vector<uint64_t> versions;     // each solver's sched_version at creation
  int64_t launches = 0;               // kernels this batch has launched
};

namespace {

template <typename T>
swe::DevState<T> dev_state(swe_solver* s) {
  swe::DevState<T> d;
  char* w = s->ws;
  d.q = reinterpret_cast<T*>(w + s->lay.q);
  d.ring = reinterpret_cast<T*>(w + s->lay.ring);
  d.qmid = reinterpret_cast<T*>(w + s->lay.qmid);
  d.p1 = reinterpret_cast<T*>(w + s->lay.p1);
  d.vb = reinterpret_cast<const T*>(w + s->lay.vb);
  d.B = reinterpret_cast<const T*>(w + s->lay.B);
  d.geo = reinterpret_cast<const T*>(w + s->lay.geo);
  d.conn = reinterpret_cast<const int4*>(w + s->lay.conn);
  d.tvbg = reinterpret_cast<const T*>(w + s->lay.tvbg);
  d.means = reinterpret_cast<T*>(w + s->lay.means);
  d.dry = reinterpret_cast<uint8_t*>(w + s->lay.dry);
  d.Bbar = reinterpret_cast<const double*>(w + s->lay.Bbar);
  d.ops = reinterpret_cast<const T*>(w + s->lay.ops);
  d.tcops = reinterpret_cast<const uint32_t*>(w + s->lay.tcops);
  d.acc = reinterpret_cast<double*>(w + s->lay.acc);
  d.flags = reinterpret_cast<int*>(w + s->lay.flags);
  d.macro = reinterpret_cast<long long*>(w + s->lay.macro);
  d.comp = s->comp ? reinterpret_cast<T*>(w + s->lay.comp) : nullptr;
  return d;
}

swe::Sched sched_of(const swe_solver* s) {
  swe::Sched sc;
  std::memset(&sc, 0, sizeof(sc));
  sc.K = s->K;
  sc.KS = s->KS;
  sc.L = s->L;
  for (int l = 0; l <= s->L; ++l) sc.off[l] = s->off[l];
  for (int l = s->L + 1; l <= swe::kMaxLevels; ++l) sc.off[l] = s->K;
  sc.dt_min = s->dt_min;
  for (int l = 1; l <= swe::kMaxLevels; ++l) {
    sc.dtl_d[l - 1] = s->dt_min * (double)(1LL << (l - 1));
    sc.dtl_f[l - 1] = (float)sc.dtl_d[l - 1];
  }
  return sc;
}

swe::Phys phys_of(const swe_solver* s, int mask) {
  swe::Phys ph;
  ph.g = s->prm.g;
  ph.h0 = s->prm.h0;
  // a depth the limiter leaves exactly at h0 (a vertex of a limited element) takes
  // u = 0 whatever the rounding of eta - B
  ph.hvel = s->prm.h0 * (1.0 + 1e-6);
  ph.eps = s->prm.eps > 0 ? s->prm.eps : s->prm.h0;
  ph.eps_f = (float)ph.eps;
  ph.tvb_M = s->prm.tvb_M;
  ph.tvb_nu = s->prm.tvb_nu > 0 ? s->prm.tvb_nu : 1.5;
  ph.pp = (mask & SWE_LIM_PP) ? 1 : 0;
  ph.dry_mode = s->prm.dry_mode;
  ph.ff_h = s->ff[0];
  ph.ff_hu = s->ff[1];
  ph.ff_hv = s->ff[2];
  return ph;
}

int upload(swe_solver* s, size_t off, const void* host, size_t bytes) {
  SWE_CUDA(cudaMemcpyAsync(s->ws + off, host, bytes, cudaMemcpyHostToDevice, s->stream));
  return SWE_OK;
}

template <typename T>
std::vector<T> to_t(const std::vector<double>& v) {
  std::vector<T> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = (T)v[i];
  return o;
}

// bf16 round-to-nearest-even of a float (host), and its value
uint16_t bf16_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}
float bf16_value(uint16_t b) {
  uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
// hi/lo TF32 split of an operator entry: hi rounded to 10 mantissa bits (to
// nearest, ties away), lo = the single-precision remainder (the tensor core reads
// its top 10 mantissa bits)
void tf32_split(double v, uint32_t& hi, uint32_t& lo) {
  const float vf = (float)v;
  uint32_t u;
  std::memcpy(&u, &vf, 4);
  u = (u + 0x1000u) & 0xFFFFE000u;
  float h;
  std::memcpy(&h, &u, 4);
  const float l = vf - h;
  hi = u;
  std::memcpy(&lo, &l, 4);
}

// hi/lo bf16 split of a single-precision operator entry
void bf16_split(double v, uint16_t& hi, uint16_t& lo) {
  const float vf = (float)v;
  hi = bf16_bits(vf);
  lo = bf16_bits(vf - bf16_value(hi));
}

// Pack the FP64 reference operators into the kernels' operator block (OpLayout)
// and the tensor-core fragment block (TcLayout).
template <int N>
void pack_ops_n(const swe::RefElem& e, std::vector<double>& o, std::vector<uint32_t>& tc) {
  using O = swe::OpLayout<N>;
  using D = swe::Dims<N>;
  using C = swe::TcDims<N>;
  using TL = swe::TcLayout<N>;
  const int np = e.Np, nc = e.Ncub, ng = e.Ng, nfp = e.Nfp, npp = D::NPP, nfpp = D::NFPP;
  o.assign(O::SIZE, 0.0);
  auto put_rows = [&](int off, const std::vector<double>& M, int rows, int cols, bool transpose_src) {
    // destination [rows][npp]; source M is rows x cols (or cols x rows if transposed)
    for (int r = 0; r < rows; ++r)
      for (int c = 0; c < cols; ++c)
        o[off + (size_t)r * npp + c] = transpose_src ? M[(size_t)c * rows + r] : M[(size_t)r * cols + c];
  };
  put_rows(O::LGT, e.Lg, 3 * ng, np, true);  // Lg is np x 3ng
  for (int g = 0; g < ng; ++g)
    for (int m = 0; m < nfp; ++m) o[O::I1D + (size_t)g * nfpp + m] = e.I1d[(size_t)g * nfp + m];
  for (int j = 0; j < np; ++j) o[O::MW + j] = e.mean_w[j];
  for (int v = 0; v < 3; ++v)
    for (int j = 0; j < np; ++j) o[O::T1 + (size_t)v * npp + j] = e.T1[(size_t)v * np + j];
  for (int j = 0; j < np; ++j)
    for (int v = 0; v < 3; ++v) o[O::BARY + (size_t)j * 4 + v] = e.bary[(size_t)j * 3 + v];

  // nodal differentiation: d/dr of the interpolant has degree N-1, so projecting
  // its cubature values back onto P_N (P = M^-1 Ic^T W) recovers it: Dr = P Icr
  for (int i = 0; i < np; ++i)
    for (int j = 0; j < np; ++j) {
      double dr = 0.0, ds = 0.0;
      for (int c = 0; c < nc; ++c) {
        dr += e.P[(size_t)i * nc + c] * e.Icr[(size_t)c * np + j];
        ds += e.P[(size_t)i * nc + c] * e.Ics[(size_t)c * np + j];
      }
      o[O::DR + (size_t)i * npp + j] = dr;
      o[O::DS + (size_t)i * npp + j] = ds;
    }
  put_rows(O::IC, e.Ic, nc, np, false);
  put_rows(O::ICR, e.Icr, nc, np, false);
  put_rows(O::ICS, e.Ics, nc, np, false);
  put_rows(O::PRT, e.Pr, nc, np, true);  // Pr is np x nc -> rows c
  put_rows(O::PST, e.Ps, nc, np, true);
  put_rows(O::PT, e.P, nc, np, true);

  {
  // tensor-core fragments (mma.sync m16n8k16 / m16n8k8 bf16 B operands)
  tc.assign(TL::SIZE, 0u);
  const std::vector<double>* interp[3] = {&e.Ic, &e.Icr, &e.Ics};   // nc x np
  const std::vector<double>* proj[3] = {&e.Pr, &e.Ps, &e.P};        // np x nc
  auto pack2 = [](uint16_t lo16, uint16_t hi16) { return (uint32_t)lo16 | ((uint32_t)hi16 << 16); };
  for (int op = 0; op < 3; ++op)
    for (int ct = 0; ct < C::CT; ++ct)
      for (int ks = 0; ks < C::KSTEP; ++ks)
        for (int lane = 0; lane < 32; ++lane) {
          const int g = lane / 4, t = lane % 4;
          // B[k][n] = Op[c = 8ct + n][j = 16ks + k]
          auto Bv = [&](int kk, int nn) {
            const int c = 8 * ct + nn, j = 16 * ks + kk;
            return (c < nc && j < np) ? (*interp[op])[(size_t)c * np + j] : 0.0;
          };
          const int kk[4] = {2 * t, 2 * t + 1, 2 * t + 8, 2 * t + 9};
          uint16_t h[4], l[4];
          for (int q = 0; q < 4; ++q) bf16_split(Bv(kk[q], g), h[q], l[q]);
          const size_t base = (((size_t)(op * C::CT + ct) * C::KSTEP + ks) * 2) * 64;
          tc[TL::INTERP + base + 0 * 64 + lane * 2 + 0] = pack2(h[0], h[1]);
          tc[TL::INTERP + base + 0 * 64 + lane * 2 + 1] = pack2(h[2], h[3]);
          tc[TL::INTERP + base + 1 * 64 + lane * 2 + 0] = pack2(l[0], l[1]);
          tc[TL::INTERP + base + 1 * 64 + lane * 2 + 1] = pack2(l[2], l[3]);
        }
  for (int op = 0; op < 3; ++op)
    for (int ct = 0; ct < C::CT; ++ct)
      for (int nt = 0; nt < C::NT; ++nt)
        for (int lane = 0; lane < 32; ++lane) {
          const int g = lane / 4, t = lane % 4;
          // B[k][n] = Op[i = 8nt + n][c = 8ct + k]
          auto Bv = [&](int kk, int nn) {
            const int i = 8 * nt + nn, c = 8 * ct + kk;
            return (i < np && c < nc) ? (*proj[op])[(size_t)i * nc + c] : 0.0;
          };
          uint16_t h0, l0, h1, l1;
          bf16_split(Bv(2 * t, g), h0, l0);
          bf16_split(Bv(2 * t + 1, g), h1, l1);
          const size_t base = (((size_t)(op * C::CT + ct) * C::NT + nt) * 2) * 32;
          tc[TL::PROJ + base + 0 * 32 + lane] = pack2(h0, h1);
          tc[TL::PROJ + base + 1 * 32 + lane] = pack2(l0, l1);
        }
  // nodal differentiation for the strong-form pressure term: TF32 m16n8k8 B
  // operands, B[k][n] = D[i = 8nt + n][j = 8kk + k]; lane (g, t) holds k = t, t + 4
  for (int op = 0; op < 2; ++op)
    for (int kk = 0; kk < C::KP / 8; ++kk)
      for (int nt = 0; nt < C::NT; ++nt)
        for (int lane = 0; lane < 32; ++lane) {
          const int g = lane / 4, t = lane % 4;
          auto Bv = [&](int k, int n) {
            const int i = 8 * nt + n, j = 8 * kk + k;
            return (i < np && j < np) ? o[(op == 0 ? O::DR : O::DS) + (size_t)i * npp + j] : 0.0;
          };
          uint32_t h0, l0, h1, l1;
          tf32_split(Bv(t, g), h0, l0);
          tf32_split(Bv(t + 4, g), h1, l1);
          const size_t base = TL::DIFF + ((((size_t)op * (C::KP / 8) + kk) * C::NT + nt) * 2) * 64;
          tc[base + 0 * 64 + lane * 2 + 0] = h0;
          tc[base + 0 * 64 + lane * 2 + 1] = h1;
          tc[base + 1 * 64 + lane * 2 + 0] = l0;
          tc[base + 1 * 64 + lane * 2 + 1] = l1;
        }
  // lift: B[k][n] = -Lg[i = 8nt + n][q = 8kt + k], q = 3 Ng face points (Lg is np x 3ng)
  for (int kt = 0; kt < C::KT; ++kt)
    for (int nt = 0; nt < C::NT; ++nt)
      for (int lane = 0; lane < 32; ++lane) {
        const int g = lane / 4, t = lane % 4;
        auto Bv = [&](int kk, int nn) {
          const int i = 8 * nt + nn, q = 8 * kt + kk;
          return (i < np && q < 3 * ng) ? -e.Lg[(size_t)i * 3 * ng + q] : 0.0;
        };
        uint16_t h0, l0, h1, l1;
        bf16_split(Bv(2 * t, g), h0, l0);
        bf16_split(Bv(2 * t + 1, g), h1, l1);
        const size_t base = ((size_t)(kt * C::NT + nt) * 2) * 32;
        tc[TL::LIFT + base + 0 * 32 + lane] = pack2(h0, h1);
        tc[TL::LIFT + base + 1 * 32 + lane] = pack2(l0, l1);
      }
  }
}

// The operators of the nodal-collocation scheme in the cubature scheme's slots:
// "cubature points" = the nodes (Ic = I, Icr = Dr, Ics = Ds, Pr = M^-1 Dr^T M,
// Ps = M^-1 Ds^T M, P = I) and "Gauss points" = the face nodes (I1d = I, lift of
// face f = Lg_f I1d = M^-1 E_f, exact for the degree-N interpolant along the face).
swe::RefElem collocation_of(const swe::RefElem& e) {
  const int np = e.Np, nc = e.Ncub, ng = e.Ng, nfp = e.Nfp;
  swe::RefElem c = e;
  std::vector<double> Dr((size_t)np * np, 0.0), Ds((size_t)np * np, 0.0);
  for (int i = 0; i < np; ++i)
    for (int j = 0; j < np; ++j)
      for (int q = 0; q < nc; ++q) {
        Dr[(size_t)i * np + j] += e.P[(size_t)i * nc + q] * e.Icr[(size_t)q * np + j];
        Ds[(size_t)i * np + j] += e.P[(size_t)i * nc + q] * e.Ics[(size_t)q * np + j];
      }
  // M = invV^T invV, M^-1 = V V^T
  std::vector<double> M((size_t)np * np, 0.0), Mi((size_t)np * np, 0.0);
  for (int i = 0; i < np; ++i)
    for (int j = 0; j < np; ++j)
      for (int q = 0; q < np; ++q) {
        M[(size_t)i * np + j] += e.invV[(size_t)q * np + i] * e.invV[(size_t)q * np + j];
        Mi[(size_t)i * np + j] += e.V[(size_t)i * np + q] * e.V[(size_t)j * np + q];
      }
  auto weak = [&](const std::vector<double>& D) {   // M^-1 D^T M
    std::vector<double> t((size_t)np * np, 0.0), o((size_t)np * np, 0.0);
    for (int i = 0; i < np; ++i)
      for (int j = 0; j < np; ++j)
        for (int q = 0; q < np; ++q) t[(size_t)i * np + j] += D[(size_t)q * np + i] * M[(size_t)q * np + j];
    for (int i = 0; i < np; ++i)
      for (int j = 0; j < np; ++j)
        for (int q = 0; q < np; ++q) o[(size_t)i * np + j] += Mi[(size_t)i * np + q] * t[(size_t)q * np + j];
    return o;
  };
  c.Ncub = np;
  c.Ic.assign((size_t)np * np, 0.0);
  for (int i = 0; i < np; ++i) c.Ic[(size_t)i * np + i] = 1.0;
  c.P = c.Ic;
  c.Icr = Dr;
  c.Ics = Ds;
  c.Pr = weak(Dr);
  c.Ps = weak(Ds);
  c.Ng = nfp;
  c.Lg.assign((size_t)np * 3 * nfp, 0.0);
  for (int f = 0; f < 3; ++f)
    for (int i = 0; i < np; ++i)
      for (int m = 0; m < nfp; ++m) {
        double v = 0.0;
        for (int g = 0; g < ng; ++g) v += e.Lg[(size_t)i * 3 * ng + f * ng + g] * e.I1d[(size_t)g * nfp + m];
        c.Lg[(size_t)i * 3 * nfp + f * nfp + m] = v;
      }
  c.I1d.assign((size_t)nfp * nfp, 0.0);
  for (int m = 0; m < nfp; ++m) c.I1d[(size_t)m * nfp + m] = 1.0;
  return c;
}

void pack_ops(int code, const swe::RefElem& e, std::vector<double>& o, std::vector<uint32_t>& tc) {
  constexpr int C = swe::kColloc, R = swe::kReduced;
  switch (code) {
    case 1: pack_ops_n<1>(e, o, tc); break;
    case 2: pack_ops_n<2>(e, o, tc); break;
    case 3: pack_ops_n<3>(e, o, tc); break;
    case 4: pack_ops_n<4>(e, o, tc); break;
    case 5: pack_ops_n<5>(e, o, tc); break;
    case C + 2: pack_ops_n<C + 2>(collocation_of(e), o, tc); break;
    case C + 3: pack_ops_n<C + 3>(collocation_of(e), o, tc); break;
    case C + 4: pack_ops_n<C + 4>(collocation_of(e), o, tc); break;
    case C + 5: pack_ops_n<C + 5>(collocation_of(e), o, tc); break;
    case R + 2: pack_ops_n<R + 2>(e, o, tc); break;   // e holds the order-2N rules
    case R + 3: pack_ops_n<R + 3>(e, o, tc); break;
    case R + 4: pack_ops_n<R + 4>(e, o, tc); break;
    case R + 5: pack_ops_n<R + 5>(e, o, tc); break;
    default: break;
  }
}

int tc_size_of(int N) {
  switch (N) {
    case 1: return swe::TcLayout<1>::SIZE;
    case 2: return swe::TcLayout<2>::SIZE;
    case 3: return swe::TcLayout<3>::SIZE;
    case 4: return swe::TcLayout<4>::SIZE;
    case 5: return swe::TcLayout<5>::SIZE;
    case swe::kColloc + 2: return swe::TcLayout<swe::kColloc + 2>::SIZE;
    case swe::kColloc + 3: return swe::TcLayout<swe::kColloc + 3>::SIZE;
    case swe::kColloc + 4: return swe::TcLayout<swe::kColloc + 4>::SIZE;
    case swe::kColloc + 5: return swe::TcLayout<swe::kColloc + 5>::SIZE;
    case swe::kReduced + 2: return swe::TcLayout<swe::kReduced + 2>::SIZE;
    case swe::kReduced + 3: return swe::TcLayout<swe::kReduced + 3>::SIZE;
    case swe::kReduced + 4: return swe::TcLayout<swe::kReduced + 4>::SIZE;
    case swe::kReduced + 5: return swe::TcLayout<swe::kReduced + 5>::SIZE;
    default: return 0;
  }
}

template <typename T>
int upload_ops_t(swe_solver* s) {
  std::vector<double> o;
  std::vector<uint32_t> tc;
  pack_ops(s->code, s->ref, o, tc);
  const int opsz = s->fp64 ? s->ld->op_size : s->lf->op_size;
  if ((int)o.size() != opsz) return fail(SWE_EINVAL, "internal: operator block size mismatch");
  std::vector<T> ot = to_t<T>(o);
  int rc = upload(s, s->lay.ops, ot.data(), ot.size() * sizeof(T));
  if (rc) return rc;
  rc = upload(s, s->lay.tcops, tc.data(), tc.size() * sizeof(uint32_t));
  if (rc) return rc;
  SWE_CUDA(cudaStreamSynchronize(s->stream));
  return SWE_OK;
}

// Upload everything that depends on the element order (geometry, connectivity,
// stencil, bathymetry, permutation).
template <typename T>
int upload_mesh_t(swe_solver* s) {
  const int K = s->K, KS = s->KS;
  const swe::Mesh& m = s->mesh;
  std::vector<double> alpha, beta;
  std::vector<int32_t> jsel;
  swe::tvb_stencil(m, alpha, beta, jsel);
  std::vector<T> geo((size_t)K * 4), tvbg((size_t)K * 8, T(0));
  std::vector<int32_t> conn((size_t)K * 4);
  for (int e = 0; e < K; ++e) {
    const int c = s->perm[e];
    geo[4 * (size_t)e + 0] = (T)m.rx[c];
    geo[4 * (size_t)e + 1] = (T)m.ry[c];
    geo[4 * (size_t)e + 2] = (T)m.sx[c];
    geo[4 * (size_t)e + 3] = (T)m.sy[c];
    int w = 0;
    for (int f = 0; f < 3; ++f) {
      const int nb = m.EToE[3 * (size_t)c + f];
      if (nb >= 0 && s->level[nb] < s->level[c]) w |= 1 << 12;   // a finer neighbour reads qmid
      conn[4 * (size_t)e + f] = nb >= 0 ? s->iperm[nb] : (s->open_face[3 * (size_t)c + f] ? swe::kFarField : swe::kWall);
      const int fn = nb >= 0 ? m.EToF[3 * (size_t)c + f] : 0;
      w |= (fn & 3) << (2 * f);
      w |= (jsel[3 * (size_t)c + f] & 3) << (6 + 2 * f);
      tvbg[8 * (size_t)e + 2 * f] = (T)alpha[3 * (size_t)c + f];
      tvbg[8 * (size_t)e + 2 * f + 1] = (T)beta[3 * (size_t)c + f];
    }
    conn[4 * (size_t)e + 3] = w;
  }
  int rc;
  if ((rc = upload(s, s->lay.geo, geo.data(), geo.size() * sizeof(T)))) return rc;
  if ((rc = upload(s, s->lay.conn, conn.data(), conn.size() * 4))) return rc;
  if ((rc = upload(s, s->lay.tvbg, tvbg.data(), tvbg.size() * sizeof(T)))) return rc;
  if ((rc = upload(s, s->lay.perm, s->perm.data(), (size_t)K * 4))) return rc;
  if ((rc = upload(s, s->lay.iperm, s->iperm.data(), (size_t)K * 4))) return rc;
  if (s->have_B) {
    std::vector<T> b((size_t)s->Np * KS, T(0)), vb(3 * (size_t)KS, T(0));
    std::vector<double> bbar(K, 0.0);
    for (int e = 0; e < K; ++e) {
      const int c = s->perm[e];
      double acc = 0.0, v1[3] = {0.0, 0.0, 0.0};
      for (int j = 0; j < s->Np; ++j) {
        const T v = (T)s->B_in[(size_t)c * s->Np + j];
        b[(size_t)j * KS + e] = v;
        acc += s->ref.mean_w[j] * (double)v;
        for (int t = 0; t < 3; ++t) v1[t] += s->ref.T1[(size_t)t * s->Np + j] * (double)v;
      }
      bbar[e] = acc;
      for (int t = 0; t < 3; ++t) vb[(size_t)t * KS + e] = (T)v1[t];
    }
    if ((rc = upload(s, s->lay.B, b.data(), b.size() * sizeof(T)))) return rc;
    if ((rc = upload(s, s->lay.vb, vb.data(), vb.size() * sizeof(T)))) return rc;
    if ((rc = upload(s, s->lay.bcaller, s->B_in.data(), s->B_in.size() * 8))) return rc;
    if ((rc = upload(s, s->lay.Bbar, bbar.data(), bbar.size() * 8))) return rc;
    SWE_CUDA(cudaStreamSynchronize(s->stream));
  }
  SWE_CUDA(cudaStreamSynchronize(s->stream));
  return SWE_OK;
}

int upload_mesh(swe_solver* s) { return s->fp64 ? upload_mesh_t<double>(s) : upload_mesh_t<float>(s); }

// level-sorted permutation (finest level first, caller order kept inside a level)
void build_order(swe_solver* s) {
  const int K = s->K;
  s->perm.resize(K);
  s->iperm.resize(K);
  int L = 1;
  for (int v : s->level) L = std::max(L, v);
  s->L = L;
  s->off.assign(L + 1, 0);
  std::vector<int> cnt(L + 1, 0);
  for (int c = 0; c < K; ++c) cnt[s->level[c]]++;
  for (int l = 1; l <= L; ++l) s->off[l] = s->off[l - 1] + cnt[l];
  std::vector<int> pos(s->off.begin(), s->off.end());
  for (int c = 0; c < K; ++c) {
    const int e = pos[s->level[c] - 1]++;
    s->perm[e] = c;
    s->iperm[c] = e;
  }
}

int invalidate_graph(swe_solver* s) {
  s->sched_version++;
  if (s->graph) {
    cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
  }
  return SWE_OK;
}

// The compensation planes start at zero whenever the state is set or re-ordered
// from the host (they hold at most one rounding of each node's state).
int clear_comp(swe_solver* s) {
  if (s->comp) SWE_CUDA(cudaMemsetAsync(s->ws + s->lay.comp, 0, 3 * (size_t)s->Np * s->KS * s->ts, s->stream));
  return SWE_OK;
}

int reset_counters(swe_solver* s) {
  s->k = 0;
  SWE_CUDA(cudaMemsetAsync(s->ws + s->lay.macro, 0, 8, s->stream));
  return SWE_OK;
}

// limiter launches on the current (post_stage = 0) or just-committed state
template <typename T>
int launch_limit_t(swe_solver* s, int mask, int post_stage, int j, int nactive) {
  const swe::Launchers<T>* lt;
  if constexpr (sizeof(T) == 8) lt = s->ld; else lt = s->lf;
  swe::LimitParams<T> p;
  p.s = dev_state<T>(s);
  p.sc = sched_of(s);
  p.ph = phys_of(s, mask);
  p.j = j;
  p.nactive = nactive;
  p.post_stage = post_stage;
  if ((mask & SWE_LIM_PP) && !post_stage) {
    SWE_CUDA(lt->positivity(p, s->cfg, s->stream));
    s->launches++;
  } else if (!post_stage) {
    // means and dry flags are still needed by the TVB limiter: positivity pass without limiting
    p.ph.pp = 0;
    SWE_CUDA(lt->positivity(p, s->cfg, s->stream));
    s->launches++;
    p.ph.pp = (mask & SWE_LIM_PP) ? 1 : 0;
  }
  if (mask & SWE_LIM_TVB) {
    SWE_CUDA(lt->tvb(p, s->cfg, s->stream));
    s->launches++;
  }
  return SWE_OK;
}

int launch_limit(swe_solver* s, int mask, int post_stage, int j, int nactive) {
  return s->fp64 ? launch_limit_t<double>(s, mask, post_stage, j, nactive)
                 : launch_limit_t<float>(s, mask, post_stage, j, nactive);
}

int active_levels(const swe_solver* s, int j) {
  if (j == 0) return s->L;
  int m = 1;
  while (m < s->L && (j % (1 << m)) == 0) ++m;
  return m;
}

// enqueue one finest substep j of the current macro step
struct KernelTimer {
  std::vector<cudaEvent_t> ev;   // pairs (start, stop)
  std::vector<int> kind;         // 0 stage, 1 tvb, 2 other
  std::vector<int64_t> elems;
};

int timer_mark(swe_solver* s, KernelTimer* t, bool start, int kind, int64_t elems) {
  if (!t) return SWE_OK;
  cudaEvent_t e;
  SWE_CUDA(cudaEventCreate(&e));
  SWE_CUDA(cudaEventRecord(e, s->stream));
  t->ev.push_back(e);
  if (start) {
    t->kind.push_back(kind);
    t->elems.push_back(elems);
  }
  return SWE_OK;
}

template <typename T>
int enqueue_substep_t(swe_solver* s, int j, KernelTimer* tm = nullptr) {
  const swe::Launchers<T>* lt;
  if constexpr (sizeof(T) == 8) lt = s->ld; else lt = s->lf;
  const int m = active_levels(s, j);
  const int nactive = s->off[m];
  swe::StageParams<T> p;
  p.s = dev_state<T>(s);
  p.sc = sched_of(s);
  p.ph = phys_of(s, s->prm.limiter_mask);
  p.j = j;
  p.nactive = nactive;
  p.mode = 0;
  p.out = nullptr;
  p.perm = nullptr;
  int rc;
  if ((rc = timer_mark(s, tm, true, 0, nactive))) return rc;
  if (s->tc) {
    SWE_CUDA(lt->stage_tc(p, s->cfg, s->stream));
  } else {
    SWE_CUDA(lt->stage(p, s->cfg, s->stream));
  }
  if ((rc = timer_mark(s, tm, false, 0, 0))) return rc;
  int nl = 1;
  if (s->prm.limiter_mask & SWE_LIM_TVB) {
    swe::LimitParams<T> lp;
    lp.s = p.s;
    lp.sc = p.sc;
    lp.ph = p.ph;
    lp.j = j;
    lp.nactive = nactive;
    lp.post_stage = 1;
    if ((rc = timer_mark(s, tm, true, 1, nactive))) return rc;
    SWE_CUDA(lt->tvb(lp, s->cfg, s->stream));
    if ((rc = timer_mark(s, tm, false, 1, 0))) return rc;
    ++nl;
  }
  const int period = 1 << (s->L - 1);
  if (j == period - 1) {
    if ((rc = timer_mark(s, tm, true, 2, 0))) return rc;
    SWE_CUDA(swe::launch_advance(p.s.macro, s->stream));
    if ((rc = timer_mark(s, tm, false, 2, 0))) return rc;
    ++nl;
  }
  return nl;
}

int enqueue_substep(swe_solver* s, int j, KernelTimer* tm = nullptr) {
  return s->fp64 ? enqueue_substep_t<double>(s, j, tm) : enqueue_substep_t<float>(s, j, tm);
}

int64_t substep_dofs(const swe_solver* s, int j) {
  return (int64_t)s->off[active_levels(s, j)] * s->Np * 3;
}

bool synchronous(const swe_solver* s) { return (s->k % (1LL << (s->L - 1))) == 0; }

// Current state in the caller's layout ([K][Np] FP64 arrays, depth h): unpacked
// on the device into the staging region, then one copy per array (any of h, hu,
// hv may be NULL).
int download_state(const swe_solver* cs, double* h, double* hu, double* hv) {
  swe_solver* s = const_cast<swe_solver*>(cs);
  const size_t n = (size_t)s->K * s->Np;
  double* x = reinterpret_cast<double*>(s->ws + s->lay.xfer);
  const double* bc = reinterpret_cast<const double*>(s->ws + s->lay.bcaller);
  const int* ip = reinterpret_cast<const int*>(s->ws + s->lay.iperm);
  const swe::Sched sc = sched_of(s);
  cudaError_t ce = s->fp64
      ? swe::launch_unpack_state<double>(reinterpret_cast<const double*>(s->ws + s->lay.q), bc, ip, sc, s->k,
                                         s->Np, x, s->stream)
      : swe::launch_unpack_state<float>(reinterpret_cast<const float*>(s->ws + s->lay.q), bc, ip, sc, s->k,
                                        s->Np, x, s->stream);
  if (ce != cudaSuccess) return fail(SWE_ECUDA, std::string("state unpack: ") + cudaGetErrorString(ce));
  s->launches++;
  if (h) SWE_CUDA(cudaMemcpyAsync(h, x, n * 8, cudaMemcpyDeviceToHost, s->stream));
  if (hu) SWE_CUDA(cudaMemcpyAsync(hu, x + n, n * 8, cudaMemcpyDeviceToHost, s->stream));
  if (hv) SWE_CUDA(cudaMemcpyAsync(hv, x + 2 * n, n * 8, cudaMemcpyDeviceToHost, s->stream));
  SWE_CUDA(cudaStreamSynchronize(s->stream));
  return SWE_OK;
}

// current state in device precision, caller order, [3][K][Np] (no conversion)
template <typename T>
int download_raw_t(const swe_solver* s, std::vector<char>& raw) {
  const int K = s->K, KS = s->KS, np = s->Np;
  const size_t fs = (size_t)np * KS, bs = 3 * fs, cs = (size_t)K * np;
  std::vector<T> q(2 * bs);
  SWE_CUDA(cudaMemcpyAsync(q.data(), s->ws + s->lay.q, q.size() * sizeof(T), cudaMemcpyDeviceToHost,
                           s->stream));
  SWE_CUDA(cudaStreamSynchronize(s->stream));
  raw.assign(3 * cs * sizeof(T), 0);
  T* out = reinterpret_cast<T*>(raw.data());
  for (int e = 0; e < K; ++e) {
    const int c = s->perm[e];
    int l = 1;
    while (l < s->L && e >= s->off[l]) ++l;
    const int cur = (int)((s->k >> (l - 1)) & 1);
    for (int f = 0; f < 3; ++f)
      for (int j = 0; j < np; ++j)
        out[f * cs + (size_t)c * np + j] = q[cur * bs + f * fs + (size_t)j * KS + e];
  }
  return SWE_OK;
}

template <typename T>
int upload_raw_t(swe_solver* s, const std::vector<char>& raw) {
  const int K = s->K, KS = s->KS, np = s->Np;
  const T* in = reinterpret_cast<const T*>(raw.data());
  const size_t fs = (size_t)np * KS, cs = (size_t)K * np;
  std::vector<T> q(3 * fs, T(0));
  for (int e = 0; e < K; ++e) {
    const int c = s->perm[e];
    for (int f = 0; f < 3; ++f)
      for (int j = 0; j < np; ++j) q[f * fs + (size_t)j * KS + e] = in[f * cs + (size_t)c * np + j];
  }
  int rc = upload(s, s->lay.q, q.data(), q.size() * sizeof(T));
  if (rc) return rc;
  SWE_CUDA(cudaStreamSynchronize(s->stream));
  return SWE_OK;
}

int apply_levels(swe_solver* s, const std::vector<int32_t>& level, double dt_min) {
  // keep the current state (bit for bit, in device precision) across a re-ordering
  std::vector<char> raw;
  std::vector<uint8_t> dry_dev, dry_caller;
  const bool had_state = s->have_state;
  if (had_state) {
    if (!synchronous(s)) return fail(SWE_EINVAL, "levels can change only at a level-synchronous state");
    int rc = s->fp64 ? download_raw_t<double>(s, raw) : download_raw_t<float>(s, raw);
    if (rc) return rc;
    dry_dev.resize(s->K);
    dry_caller.resize(s->K);
    SWE_CUDA(cudaMemcpy(dry_dev.data(), s->ws + s->lay.dry, s->K, cudaMemcpyDeviceToHost));
    for (int e = 0; e < s->K; ++e) dry_caller[s->perm[e]] = dry_dev[e];
    s->t0 += (double)s->k * s->dt_min;
  }
  s->level = level;
  s->dt_min = dt_min;
  build_order(s);
  s->have_levels = true;
  invalidate_graph(s);
  int rc = upload_mesh(s);
  if (rc) return rc;
  if (had_state) {
    rc = s->fp64 ? upload_raw_t<double>(s, raw) : upload_raw_t<float>(s, raw);
    if (rc) return rc;
    if ((rc = reset_counters(s))) return rc;
    if ((rc = clear_comp(s))) return rc;
    // recompute the means of the re-ordered state (positivity pass, no limiting),
    // then restore the dry flags of the latest positivity pass
    if ((rc = launch_limit(s, 0, 0, 0, s->K))) return rc;
    for (int e = 0; e < s->K; ++e) dry_dev[e] = dry_caller[s->perm[e]];
    SWE_CUDA(cudaMemcpyAsync(s->ws + s->lay.dry, dry_dev.data(), s->K, cudaMemcpyHostToDevice, s->stream));
    SWE_CUDA(cudaStreamSynchronize(s->stream));
  }
  return SWE_OK;
}

// Regroup at a level-synchronous substep k with dt_min, k and the Adams-Bashforth
// history kept (reading in the swe_regroup contract), on the device: the history of
// moved elements is re-interpolated in place (ring slot of activation a = a mod 3,
// a = k >> (level - 1)), then every per-element array is gathered into the new
// level order through the FP64 staging buffer. Only index arrays cross the bus.
template <typename T>
int regroup_t(swe_solver* s, const std::vector<int32_t>& lev_new) {
  const int K = s->K, KS = s->KS, np = s->Np;
  const int64_t k = s->k;
  cudaStream_t st = s->stream;
  const std::vector<int32_t> perm_old = s->perm, iperm_old = s->iperm, lev_old = s->level;
  s->level = lev_new;
  build_order(s);
  invalidate_graph(s);
  // pi: new index -> old index; sigma: old -> new; levels by old and new index
  std::vector<int32_t> pi(K), sigma(K);
  std::vector<uint8_t> lo(K), ln_old(K), ln_new(K);
  for (int e = 0; e < K; ++e) {
    pi[e] = iperm_old[s->perm[e]];
    ln_new[e] = (uint8_t)lev_new[s->perm[e]];
    const int c = perm_old[e];
    sigma[e] = s->iperm[c];
    lo[e] = (uint8_t)lev_old[c];
    ln_old[e] = (uint8_t)lev_new[c];
  }
  char* x = s->ws + s->lay.xfer;
  const size_t xbytes = 3 * (size_t)K * np * 8;
  int* d_pi = reinterpret_cast<int*>(x);
  int* d_sigma = d_pi + K;
  uint8_t* d_lo = reinterpret_cast<uint8_t*>(d_sigma + K);
  uint8_t* d_lno = d_lo + K;
  uint8_t* d_lnn = d_lno + K;
  const size_t idx = ((size_t)K * 11 + 255) / 256 * 256;
  char* scr = x + idx;
  const size_t scr_bytes = xbytes > idx ? xbytes - idx : 0;
  const size_t plane = (size_t)KS * sizeof(T);
  const int chunk = (int)std::min<size_t>(scr_bytes / plane, (size_t)1 << 20);
  if (chunk < 1 || scr_bytes < (size_t)K * 8 * sizeof(T) || scr_bytes < (size_t)K * 16)
    return fail(SWE_ENOMEM, "mesh too small for the regroup staging");
  SWE_CUDA(cudaMemcpyAsync(d_pi, pi.data(), (size_t)K * 4, cudaMemcpyHostToDevice, st));
  SWE_CUDA(cudaMemcpyAsync(d_sigma, sigma.data(), (size_t)K * 4, cudaMemcpyHostToDevice, st));
  SWE_CUDA(cudaMemcpyAsync(d_lo, lo.data(), K, cudaMemcpyHostToDevice, st));
  SWE_CUDA(cudaMemcpyAsync(d_lno, ln_old.data(), K, cudaMemcpyHostToDevice, st));
  SWE_CUDA(cudaMemcpyAsync(d_lnn, ln_new.data(), K, cudaMemcpyHostToDevice, st));
  T* ring = reinterpret_cast<T*>(s->ws + s->lay.ring);
  T* sT = reinterpret_cast<T*>(scr);
  SWE_CUDA(swe::launch_ring_reinterp<T>(ring, K, KS, np, d_lo, d_lno, (long long)k, st));
  // the state: each element's current buffer into both halves, new order
  T* q = reinterpret_cast<T*>(s->ws + s->lay.q);
  const size_t bs = (size_t)3 * np * KS;
  for (int p0 = 0; p0 < 3 * np; p0 += chunk) {
    const int P = std::min(chunk, 3 * np - p0);
    SWE_CUDA(swe::launch_gather_state<T>(q, sT, p0, P, KS, K, np, d_pi, d_lo, (long long)k, st));
    SWE_CUDA(cudaMemcpyAsync(q + (size_t)p0 * KS, sT, P * plane, cudaMemcpyDeviceToDevice, st));
    SWE_CUDA(cudaMemcpyAsync(q + bs + (size_t)p0 * KS, sT, P * plane, cudaMemcpyDeviceToDevice, st));
  }
  // plane arrays
  auto planes = [&](T* a, int P) -> int {
    for (int p0 = 0; p0 < P; p0 += chunk) {
      const int n = std::min(chunk, P - p0);
      SWE_CUDA(swe::launch_gather_planes<T>(a + (size_t)p0 * KS, sT, n, KS, K, d_pi, st));
      SWE_CUDA(cudaMemcpyAsync(a + (size_t)p0 * KS, sT, n * plane, cudaMemcpyDeviceToDevice, st));
    }
    return SWE_OK;
  };
  int rc;
  if ((rc = planes(ring, 9 * np))) return rc;
  if (s->comp && (rc = planes(reinterpret_cast<T*>(s->ws + s->lay.comp), 3 * np))) return rc;
  if ((rc = planes(reinterpret_cast<T*>(s->ws + s->lay.B), np))) return rc;
  if ((rc = planes(reinterpret_cast<T*>(s->ws + s->lay.vb), 3))) return rc;
  if ((rc = planes(reinterpret_cast<T*>(s->ws + s->lay.p1), 9))) return rc;
  // per-element records
  auto rows_t = [&](size_t off, int W) -> int {
    T* a = reinterpret_cast<T*>(s->ws + off);
    SWE_CUDA(swe::launch_gather_rows<T>(a, sT, W, K, d_pi, st));
    SWE_CUDA(cudaMemcpyAsync(a, sT, (size_t)K * W * sizeof(T), cudaMemcpyDeviceToDevice, st));
    return SWE_OK;
  };
  if ((rc = rows_t(s->lay.geo, 4))) return rc;
  if ((rc = rows_t(s->lay.tvbg, 8))) return rc;
  if ((rc = rows_t(s->lay.means, 4))) return rc;
  double* bbar = reinterpret_cast<double*>(s->ws + s->lay.Bbar);
  SWE_CUDA(swe::launch_gather_rows<double>(bbar, reinterpret_cast<double*>(scr), 1, K, d_pi, st));
  SWE_CUDA(cudaMemcpyAsync(bbar, scr, (size_t)K * 8, cudaMemcpyDeviceToDevice, st));
  uint8_t* dry = reinterpret_cast<uint8_t*>(s->ws + s->lay.dry);
  SWE_CUDA(swe::launch_gather_rows<uint8_t>(dry, reinterpret_cast<uint8_t*>(scr), 1, K, d_pi, st));
  SWE_CUDA(cudaMemcpyAsync(dry, scr, (size_t)K, cudaMemcpyDeviceToDevice, st));
  int4* conn = reinterpret_cast<int4*>(s->ws + s->lay.conn);
  SWE_CUDA(swe::launch_remap_conn(conn, reinterpret_cast<int4*>(scr), K, d_pi, d_sigma, d_lnn, st));
  SWE_CUDA(cudaMemcpyAsync(conn, scr, (size_t)K * 16, cudaMemcpyDeviceToDevice, st));
  if ((rc = upload(s, s->lay.perm, s->perm.data(), (size_t)K * 4))) return rc;
  if ((rc = upload(s, s->lay.iperm, s->iperm.data(), (size_t)K * 4))) return rc;
  const long long macro = (long long)(k >> (s->L - 1));
  SWE_CUDA(cudaMemcpyAsync(s->ws + s->lay.macro, &macro, 8, cudaMemcpyHostToDevice, st));
  SWE_CUDA(cudaStreamSynchronize(st));
  return SWE_OK;
}

// Eq. cfl's per-element step (caller order) computed on the device from the
// current state; the same arithmetic as swe::element_dt on downloaded depths.
int device_element_dt(swe_solver* s, std::vector<double>& dt) {
  const int K = s->K;
  const swe::Mesh& m = s->mesh;
  std::vector<double> H(K);
  for (int e = 0; e < K; ++e) {
    const int c = s->perm[e];
    const double* L = &m.flen[3 * (size_t)c];
    H[e] = 2.0 * (2.0 * m.J[c]) / (L[0] + L[1] + L[2]);   // inradius
  }
  char* x = s->ws + s->lay.xfer;   // staging: [max depth][H (K)][dt (K)]
  unsigned long long* hm = reinterpret_cast<unsigned long long*>(x);
  double* dH = reinterpret_cast<double*>(x + 256);
  double* ddt = dH + K;
  SWE_CUDA(cudaMemcpyAsync(dH, H.data(), (size_t)K * 8, cudaMemcpyHostToDevice, s->stream));
  const double C = s->prm.cfl / ((s->N + 1.0) * (s->N + 1.0));
  const swe::Sched sc = sched_of(s);
  cudaError_t ce = s->fp64 ? swe::launch_element_dt<double>(reinterpret_cast<const double*>(s->ws + s->lay.q),
                                                              reinterpret_cast<const double*>(s->ws + s->lay.B),
                                                              sc, (long long)s->k, s->Np, dH, s->prm.g, C, hm,
                                                              ddt, s->stream)
                           : swe::launch_element_dt<float>(reinterpret_cast<const float*>(s->ws + s->lay.q),
                                                             reinterpret_cast<const float*>(s->ws + s->lay.B), sc,
                                                             (long long)s->k, s->Np, dH, s->prm.g, C, hm, ddt,
                                                             s->stream);
  if (ce != cudaSuccess) return fail(SWE_ECUDA, std::string("element dt: ") + cudaGetErrorString(ce));
  std::vector<double> dd(K);
  SWE_CUDA(cudaMemcpyAsync(dd.data(), ddt, (size_t)K * 8, cudaMemcpyDeviceToHost, s->stream));
  SWE_CUDA(cudaStreamSynchronize(s->stream));
  dt.resize(K);
  for (int e = 0; e < K; ++e) dt[s->perm[e]] = dd[e];
  return SWE_OK;
}

}  // namespace

namespace swe {
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace swe

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

int swe_version(void) { return 100; }

const char* swe_strerror(int code) {
  switch (code) {
    case SWE_OK: return "ok";
    case SWE_EINVAL: return "invalid argument";
    case SWE_ENOMEM: return "not enough memory";
    case SWE_ECUDA: return "CUDA error";
    case SWE_ENAN: return "non-finite state";
    case SWE_ETIMEOUT: return "device wait timed out";
    case SWE_EUNSUPPORTED: return "unsupported";
    default: return "unknown error";
  }
}

const char* swe_last_error(void) { return g_last_error.c_str(); }

int swe_ref_sizes(int32_t N, int32_t* Np, int32_t* Ncub, int32_t* Ng) {
  if (N < 1 || N > 7) return fail(SWE_EINVAL, "N out of range");
  if (Np) *Np = (N + 1) * (N + 2) / 2;
  if (Ncub) *Ncub = swe::ref_num_cubature(N);
  if (Ng) *Ng = swe::ref_num_gauss(N);
  return SWE_OK;
}

int swe_ref_nodes(int32_t N, double* r, double* s) {
  if (N < 1 || N > 7 || !r || !s) return fail(SWE_EINVAL, "bad arguments");
  swe::RefElem e = swe::RefElem::build(N);
  std::copy(e.r.begin(), e.r.end(), r);
  std::copy(e.s.begin(), e.s.end(), s);
  return SWE_OK;
}

int swe_ref_operator(int32_t N, int32_t which, double* out, size_t count) {
  if (N < 1 || N > 7 || !out) return fail(SWE_EINVAL, "bad arguments");
  swe::RefElem e = swe::RefElem::build(N);
  const std::vector<double>* src = nullptr;
  switch (which) {
    case 0: src = &e.Ic; break;
    case 1: src = &e.Icr; break;
    case 2: src = &e.Ics; break;
    case 3: src = &e.Pr; break;
    case 4: src = &e.Ps; break;
    case 5: src = &e.P; break;
    case 6: src = &e.Lg; break;
    case 7: src = &e.I1d; break;
    case 8: src = &e.mean_w; break;
    case 9: src = &e.T1; break;
    case 10: src = &e.wc; break;
    case 11: src = &e.wg; break;
    default: return fail(SWE_EINVAL, "unknown operator id");
  }
  if (count < src->size()) return fail(SWE_EINVAL, "output buffer too small");
  std::copy(src->begin(), src->end(), out);
  return SWE_OK;
}

int swe_mesh_create(const double* vx, const double* vy, int32_t nv, const int32_t* EToV, int32_t K,
                    swe_mesh** out) {
  if (!out) return fail(SWE_EINVAL, "out is NULL");
  *out = nullptr;
  std::unique_ptr<swe_mesh> m(new (std::nothrow) swe_mesh);
  if (!m) return fail(SWE_ENOMEM, "host allocation failed");
  std::string err = swe::Mesh::create(vx, vy, nv, EToV, K, m->m);
  if (!err.empty()) return fail(SWE_EINVAL, err);
  *out = m.release();
  return SWE_OK;
}

void swe_mesh_destroy(swe_mesh* mesh) { delete mesh; }

int swe_mesh_num_elements(const swe_mesh* mesh, int32_t* K) {
  if (!mesh || !K) return fail(SWE_EINVAL, "NULL argument");
  *K = mesh->m.K;
  return SWE_OK;
}

int swe_mesh_connectivity(const swe_mesh* mesh, int32_t* EToE, int32_t* EToF) {
  if (!mesh || !EToE || !EToF) return fail(SWE_EINVAL, "NULL argument");
  std::copy(mesh->m.EToE.begin(), mesh->m.EToE.end(), EToE);
  std::copy(mesh->m.EToF.begin(), mesh->m.EToF.end(), EToF);
  return SWE_OK;
}

int swe_mesh_node_coords(const swe_mesh* mesh, int32_t N, double* x, double* y) {
  if (!mesh || !x || !y || N < 1 || N > 7) return fail(SWE_EINVAL, "bad arguments");
  swe::RefElem e = swe::RefElem::build(N);
  const swe::Mesh& m = mesh->m;
  for (int k = 0; k < m.K; ++k) {
    const int32_t* v = &m.EToV[3 * (size_t)k];
    for (int j = 0; j < e.Np; ++j) {
      const double l0 = -(e.r[j] + e.s[j]) / 2, l1 = (1 + e.r[j]) / 2, l2 = (1 + e.s[j]) / 2;
      x[(size_t)k * e.Np + j] = l0 * m.vx[v[0]] + l1 * m.vx[v[1]] + l2 * m.vx[v[2]];
      y[(size_t)k * e.Np + j] = l0 * m.vy[v[0]] + l1 * m.vy[v[1]] + l2 * m.vy[v[2]];
    }
  }
  return SWE_OK;
}

int swe_mesh_levels(const swe_mesh* mesh, int32_t N, const double* h, const double* hu, const double* hv,
                    double g, double cfl, int32_t nlevels_max, int32_t* level_out, double* dt_min_out) {
  if (!mesh || !h || !hu || !hv || !level_out) return fail(SWE_EINVAL, "NULL argument");
  if (N < 1 || N > 7 || !(g > 0) || !(cfl > 0) || nlevels_max < 1 || nlevels_max > swe::kMaxLevels)
    return fail(SWE_EINVAL, "bad arguments");
  const size_t np = (size_t)(N + 1) * (N + 2) / 2;
  if (int rc = check_cfl_input(h, hu, hv, (size_t)mesh->m.K * np, SWE_EINVAL)) return rc;
  std::vector<double> dt;
  swe::element_dt(mesh->m, N, h, hu, hv, g, cfl, dt);
  std::vector<int32_t> lev;
  double dtmin = swe::assign_levels(dt, nlevels_max, lev);
  std::copy(lev.begin(), lev.end(), level_out);
  if (dt_min_out) *dt_min_out = dtmin;
  return SWE_OK;
}

int swe_regroup_rule(const double* dt, const int32_t* level, int32_t K, double dt_min, int64_t k,
                     int32_t nlevels_max, int32_t* level_out, double* margin_out) {
  if (!dt || !level || !level_out || K < 0) return fail(SWE_EINVAL, "bad arguments");
  if (!(dt_min > 0) || !std::isfinite(dt_min) || nlevels_max < 1 || nlevels_max > swe::kMaxLevels || k < 0)
    return fail(SWE_EINVAL, "bad arguments");
  for (int32_t i = 0; i < K; ++i) {
    if (!(dt[i] > 0) || !std::isfinite(dt[i])) return fail(SWE_EINVAL, "element steps must be finite and > 0");
    if (level[i] < 1 || level[i] > nlevels_max) return fail(SWE_EINVAL, "level out of 1..nlevels_max");
  }
  std::vector<double> d(dt, dt + K);
  std::vector<int32_t> old(level, level + K), lev;
  const double margin = swe::regroup_levels(d, dt_min, old, k, nlevels_max, lev);
  std::copy(lev.begin(), lev.end(), level_out);
  if (margin_out) *margin_out = margin;
  return SWE_OK;
}

int swe_workspace_bytes(const swe_mesh* mesh, const swe_params* params, size_t* bytes) {
  if (!mesh || !bytes) return fail(SWE_EINVAL, "NULL argument");
  int rc = check_params(params);
  if (rc) return rc;
  const bool fp64 = params->precision == SWE_FP64;
  int opsz = fp64 ? swe::launchers_for<double>(scheme_code(params))->op_size
                  : swe::launchers_for<float>(scheme_code(params))->op_size;
  *bytes = make_layout(mesh->m.K, params->N, fp64 ? 8 : 4, opsz, scheme_code(params),
                       !fp64 && params->compensated).total;
  return SWE_OK;
}

int swe_solver_create(const swe_mesh* mesh, const swe_params* params, void* dev_workspace, size_t bytes,
                      void* stream, swe_solver** out) {
  if (!mesh || !out || !dev_workspace) return fail(SWE_EINVAL, "NULL argument");
  *out = nullptr;
  int rc = check_params(params);
  if (rc) return rc;
  if (((uintptr_t)dev_workspace & 255) != 0) return fail(SWE_EINVAL, "workspace must be 256-byte aligned");
  std::unique_ptr<swe_solver> s(new (std::nothrow) swe_solver);
  if (!s) return fail(SWE_ENOMEM, "host allocation failed");
  s->mesh = mesh->m;
  s->prm = *params;
  s->N = params->N;
  s->code = scheme_code(params);
  s->K = mesh->m.K;
  s->ref = params->scheme == SWE_SCHEME_CUBATURE_2N ? swe::RefElem::build(s->N, s->N + 1, s->N + 1)
                                                      : swe::RefElem::build(s->N);
  s->Np = s->ref.Np;
  s->NPP = npp_of(s->N);
  s->KS = ks_of(s->K);
  s->fp64 = params->precision == SWE_FP64;
  s->tc = params->precision == SWE_FP32_TC;
  s->comp = !s->fp64 && params->compensated;
  s->ts = s->fp64 ? 8 : 4;
  s->stream = reinterpret_cast<cudaStream_t>(stream);
  s->ws = reinterpret_cast<char*>(dev_workspace);
  s->ws_bytes = bytes;
  if (s->fp64) {
    s->ld = swe::launchers_for<double>(s->code);
    if (!s->ld) return fail(SWE_EUNSUPPORTED, "order not built");
  } else {
    s->lf = swe::launchers_for<float>(s->code);
    if (!s->lf) return fail(SWE_EUNSUPPORTED, "order not built");
  }
  s->lay = make_layout(s->K, s->N, s->ts, s->fp64 ? s->ld->op_size : s->lf->op_size, s->code, s->comp);
  if (bytes < s->lay.total) return fail(SWE_ENOMEM, "workspace smaller than swe_workspace_bytes()");
  cudaError_t ce = s->fp64 ? s->ld->prepare(&s->cfg) : s->lf->prepare(&s->cfg);
  if (ce != cudaSuccess) return fail(SWE_ECUDA, std::string("kernel setup: ") + cudaGetErrorString(ce));
  s->cfg_max = s->cfg;
  // single level until levels are set up
  s->level.assign(s->K, 1);
  s->open_face.assign((size_t)3 * s->K, 0);
  s->dt_min = 0.0;
  build_order(s.get());
  SWE_CUDA(cudaMemsetAsync(s->ws, 0, s->lay.total, s->stream));
  rc = s->fp64 ? upload_ops_t<double>(s.get()) : upload_ops_t<float>(s.get());
  if (rc) return rc;
  rc = upload_mesh(s.get());
  if (rc) return rc;
  SWE_CUDA(cudaStreamSynchronize(s->stream));
  *out = s.release();
  return SWE_OK;
}

void swe_solver_destroy(swe_solver* solver) {
  if (!solver) return;
  cudaStreamSynchronize(solver->stream);
  invalidate_graph(solver);
  delete solver;
}

int swe_stream_create(void** out) {
  if (!out) return fail(SWE_EINVAL, "NULL argument");
  *out = nullptr;
  cudaStream_t st = nullptr;
  SWE_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  *out = st;
  return SWE_OK;
}

int swe_stream_destroy(void* stream) {
  if (!stream) return fail(SWE_EINVAL, "NULL stream");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  SWE_CUDA(cudaStreamSynchronize(st));
  SWE_CUDA(cudaStreamDestroy(st));
  return SWE_OK;
}

int swe_set_bathymetry(swe_solver* s, const double* B) {
  if (!s || !B) return fail(SWE_EINVAL, "NULL argument");
  const size_t n = (size_t)s->K * s->Np;
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(B[i])) return fail(SWE_EINVAL, "non-finite bathymetry");
  s->B_in.assign(B, B + n);
  s->B_dev.resize(n);
  for (size_t i = 0; i < n; ++i) s->B_dev[i] = s->fp64 ? B[i] : (double)(float)B[i];
  s->have_B = true;
  s->have_state = false;
  return upload_mesh(s);
}

int swe_set_state(swe_solver* s, const double* h, const double* hu, const double* hv) {
  if (!s || !h || !hu || !hv) return fail(SWE_EINVAL, "NULL argument");
  if (!s->have_B) return fail(SWE_EINVAL, "swe_set_bathymetry must come first");
  // the caller's arrays go to the device as they are; the finiteness check, the
  // level-order permutation, eta = h + B and the precision conversion run there
  const size_t n = (size_t)s->K * s->Np;
  double* x = reinterpret_cast<double*>(s->ws + s->lay.xfer);
  int* flag = reinterpret_cast<int*>(s->ws + s->lay.xflag);
  SWE_CUDA(cudaMemcpyAsync(x, h, n * 8, cudaMemcpyHostToDevice, s->stream));
  SWE_CUDA(cudaMemcpyAsync(x + n, hu, n * 8, cudaMemcpyHostToDevice, s->stream));
  SWE_CUDA(cudaMemcpyAsync(x + 2 * n, hv, n * 8, cudaMemcpyHostToDevice, s->stream));
  SWE_CUDA(cudaMemsetAsync(flag, 0, 4, s->stream));
  SWE_CUDA(swe::launch_check_finite(x, 3 * n, flag, s->stream));
  int bad = 0;
  SWE_CUDA(cudaMemcpyAsync(&bad, flag, 4, cudaMemcpyDeviceToHost, s->stream));
  SWE_CUDA(cudaStreamSynchronize(s->stream));
  s->launches++;
  if (bad) return fail(SWE_EINVAL, "non-finite state");
  const double* bc = reinterpret_cast<const double*>(s->ws + s->lay.bcaller);
  const int* ip = reinterpret_cast<const int*>(s->ws + s->lay.iperm);
  cudaError_t ce = s->fp64
      ? swe::launch_pack_state<double>(x, bc, ip, s->K, s->KS, s->Np, reinterpret_cast<double*>(s->ws + s->lay.q),
                                       s->stream)
      : swe::launch_pack_state<float>(x, bc, ip, s->K, s->KS, s->Np, reinterpret_cast<float*>(s->ws + s->lay.q),
                                      s->stream);
  if (ce != cudaSuccess) return fail(SWE_ECUDA, std::string("state pack: ") + cudaGetErrorString(ce));
  s->launches++;
  int rc;
  if ((rc = reset_counters(s))) return rc;
  if ((rc = clear_comp(s))) return rc;
  s->t0 = 0.0;
  s->dof_updates = 0;
  SWE_CUDA(cudaMemsetAsync(s->ws + s->lay.acc, 0, 64, s->stream));
  SWE_CUDA(cudaMemsetAsync(s->ws + s->lay.flags, 0, 16, s->stream));
  s->have_state = true;
  // Algorithm 2, first line: limit the initial state
  if ((rc = launch_limit(s, s->prm.limiter_mask, 0, 0, s->K))) return rc;
  SWE_CUDA(cudaStreamSynchronize(s->stream));
  return SWE_OK;
}

int swe_setup_levels(swe_solver* s, int32_t* level_out, double* dt_min_out) {
  if (!s) return fail(SWE_EINVAL, "NULL argument");
  if (!s->have_state) return fail(SWE_EINVAL, "swe_set_state must come first");
  if (!synchronous(s)) return fail(SWE_EINVAL, "state is not level-synchronous");
  const size_t n = (size_t)s->K * s->Np;
  std::vector<double> h(n), hu(n), hv(n), dt;
  int rc = download_state(s, h.data(), hu.data(), hv.data());
  if (rc) return rc;
  if ((rc = check_cfl_input(h.data(), hu.data(), hv.data(), n, SWE_ENAN))) return rc;
  swe::element_dt(s->mesh, s->N, h.data(), hu.data(), hv.data(), s->prm.g, s->prm.cfl, dt);
  std::vector<int32_t> lev;
  double dtmin = swe::assign_levels(dt, s->prm.nlevels_max, lev);
  if ((rc = apply_levels(s, lev, dtmin))) return rc;
  if (level_out) std::copy(lev.begin(), lev.end(), level_out);
  if (dt_min_out) *dt_min_out = dtmin;
  return SWE_OK;
}

int swe_regroup(swe_solver* s, const int32_t* level, int32_t* level_out, double* cfl_margin_out) {
  if (!s) return fail(SWE_EINVAL, "NULL argument");
  if (!s->have_state || !s->have_levels) return fail(SWE_EINVAL, "state and levels must come first");
  if (!synchronous(s)) return fail(SWE_EINVAL, "state is not level-synchronous");
  if (s->k < 3 * (1LL << (s->L - 1))) return fail(SWE_EINVAL, "regroup needs three activations of every level");
  std::vector<double> dt;
  int rc = device_element_dt(s, dt);
  if (rc) return rc;
  std::vector<int32_t> lev;
  double margin = swe::regroup_levels(dt, s->dt_min, s->level, s->k, s->prm.nlevels_max, lev);
  if (level) {
    lev.assign(level, level + s->K);
    int lmax = 1;
    for (int32_t v : lev) {
      if (v < 1 || v > s->prm.nlevels_max) return fail(SWE_EINVAL, "level out of 1..nlevels_max");
      lmax = std::max(lmax, (int)v);
    }
    if (s->k % (1LL << (lmax - 1))) return fail(SWE_EINVAL, "2^(max level - 1) must divide the substep count");
    margin = 1e300;
    for (int c = 0; c < s->K; ++c) margin = std::min(margin, dt[c] / std::ldexp(s->dt_min, lev[c] - 1));
  }
  rc = s->fp64 ? regroup_t<double>(s, lev) : regroup_t<float>(s, lev);
  if (rc) return rc;
  if (level_out) std::copy(lev.begin(), lev.end(), level_out);
  if (cfl_margin_out) *cfl_margin_out = margin;
  return SWE_OK;
}

int swe_set_levels(swe_solver* s, const int32_t* level, double dt_min) {
  if (!s || !level) return fail(SWE_EINVAL, "NULL argument");
  if (!(dt_min > 0) || !std::isfinite(dt_min)) return fail(SWE_EINVAL, "dt_min must be finite and > 0");
  std::vector<int32_t> lev(level, level + s->K);
  for (int32_t v : lev)
    if (v < 1 || v > s->prm.nlevels_max) return fail(SWE_EINVAL, "level out of 1..nlevels_max");
  return apply_levels(s, lev, dt_min);
}

int swe_rhs(swe_solver* s, void* dev_R) {
  if (!s || !dev_R) return fail(SWE_EINVAL, "NULL argument");
  if (!s->have_state) return fail(SWE_EINVAL, "no state");
  if (!synchronous(s)) return fail(SWE_EINVAL, "state is not level-synchronous");
  const int period = 1 << (s->L - 1);
  (void)period;
  if (s->fp64) {
    swe::StageParams<double> p;
    p.s = dev_state<double>(s);
    p.sc = sched_of(s);
    p.ph = phys_of(s, s->prm.limiter_mask);
    p.j = 0;
    p.nactive = s->K;
    p.mode = 1;
    p.out = reinterpret_cast<double*>(dev_R);
    p.perm = reinterpret_cast<const int*>(s->ws + s->lay.perm);
    SWE_CUDA(s->ld->stage(p, s->cfg, s->stream));
  } else {
    swe::StageParams<float> p;
    p.s = dev_state<float>(s);
    p.sc = sched_of(s);
    p.ph = phys_of(s, s->prm.limiter_mask);
    p.j = 0;
    p.nactive = s->K;
    p.mode = 1;
    p.out = reinterpret_cast<float*>(dev_R);
    p.perm = reinterpret_cast<const int*>(s->ws + s->lay.perm);
    if (s->tc) {
      SWE_CUDA(s->lf->stage_tc(p, s->cfg, s->stream));
    } else {
      SWE_CUDA(s->lf->stage(p, s->cfg, s->stream));
    }
  }
  s->launches++;
  return SWE_OK;
}

int swe_rhs_scratch_bytes(const swe_solver* s, int variant, size_t* bytes) {
  if (!s || !bytes) return fail(SWE_EINVAL, "NULL argument");
  if (variant < SWE_RHS_FUSED || variant > SWE_RHS_SPLIT) return fail(SWE_EINVAL, "unknown variant");
  *bytes = 0;
  if (variant == SWE_RHS_SPLIT) {
    const int planes = s->fp64 ? s->ld->split_planes : s->lf->split_planes;
    const size_t plane = (size_t)s->KS * s->ts;
    *bytes = ((plane * planes + 255) / 256) * 256 + plane * 3 * s->Np;
  }
  return SWE_OK;
}

extern "C++" {
namespace {

template <typename T>
int rhs_variant_t(swe_solver* s, const swe::Launchers<T>* lt, int variant, T* R, char* scratch) {
  swe::StageParams<T> p;
  p.s = dev_state<T>(s);
  p.sc = sched_of(s);
  p.ph = phys_of(s, s->prm.limiter_mask);
  p.j = 0;
  p.nactive = s->K;
  p.mode = 1;
  p.out = R;
  p.perm = reinterpret_cast<const int*>(s->ws + s->lay.perm);
  if (variant == SWE_RHS_FUSED) {
    if (s->tc) {
      SWE_CUDA(lt->stage_tc(p, s->cfg, s->stream));
    } else {
      SWE_CUDA(lt->stage(p, s->cfg, s->stream));
    }
    s->launches += 1;
  } else if (variant == SWE_RHS_FUSED_SIMT) {
    SWE_CUDA(lt->stage(p, s->cfg, s->stream));
    s->launches += 1;
  } else if (variant == SWE_RHS_GLOBAL_OPS) {
    SWE_CUDA(lt->stage_global_ops(p, s->cfg, s->stream));
    s->launches += 1;
  } else {
    const size_t plane = (size_t)s->KS * sizeof(T);
    T* qg = reinterpret_cast<T*>(scratch);
    T* rg = reinterpret_cast<T*>(scratch + ((plane * lt->split_planes + 255) / 256) * 256);
    SWE_CUDA(lt->split_rhs(p, qg, rg, s->cfg, s->stream));
    s->launches += 3;
  }
  return SWE_OK;
}

}  // namespace
}  // extern "C++"

int swe_rhs_variant(swe_solver* s, int variant, void* dev_R, void* dev_scratch, size_t scratch_bytes) {
  if (!s || !dev_R) return fail(SWE_EINVAL, "NULL argument");
  size_t need = 0;
  int rc = swe_rhs_scratch_bytes(s, variant, &need);
  if (rc) return rc;
  if (need > 0 && (!dev_scratch || scratch_bytes < need)) return fail(SWE_ENOMEM, "scratch too small");
  if (need > 0 && (reinterpret_cast<uintptr_t>(dev_scratch) & 255))
    return fail(SWE_EINVAL, "scratch must be 256-byte aligned");
  if (!s->have_state) return fail(SWE_EINVAL, "no state");
  if (!synchronous(s)) return fail(SWE_EINVAL, "state is not level-synchronous");
  if (s->fp64) return rhs_variant_t<double>(s, s->ld, variant, reinterpret_cast<double*>(dev_R),
                                            reinterpret_cast<char*>(dev_scratch));
  return rhs_variant_t<float>(s, s->lf, variant, reinterpret_cast<float*>(dev_R),
                              reinterpret_cast<char*>(dev_scratch));
}

int swe_substep(swe_solver* s, int32_t n) {
  if (!s || n < 0) return fail(SWE_EINVAL, "bad arguments");
  if (!s->have_state) return fail(SWE_EINVAL, "no state");
  if (!(s->dt_min > 0)) return fail(SWE_EINVAL, "levels / dt_min not set up");
  const int64_t period = 1LL << (s->L - 1);
  for (int32_t i = 0; i < n; ++i) {
    const int j = (int)(s->k % period);
    int nl = enqueue_substep(s, j);
    if (nl < 0) return nl;
    s->launches += nl;
    s->dof_updates += substep_dofs(s, j);
    s->k++;
  }
  return SWE_OK;
}

int swe_step(swe_solver* s, int32_t n_macro) {
  if (!s || n_macro < 0) return fail(SWE_EINVAL, "bad arguments");
  if (!s->have_state) return fail(SWE_EINVAL, "no state");
  if (!(s->dt_min > 0)) return fail(SWE_EINVAL, "levels / dt_min not set up");
  if (!synchronous(s)) return fail(SWE_EINVAL, "state is not level-synchronous");
  if (n_macro == 0) return SWE_OK;
  const int period = 1 << (s->L - 1);
  if (!s->graph) {
    cudaGraph_t g = nullptr;
    SWE_CUDA(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    int total = 0;
    int64_t dofs = 0;
    for (int j = 0; j < period; ++j) {
      int nl = enqueue_substep(s, j);
      if (nl < 0) {
        cudaStreamEndCapture(s->stream, &g);
        if (g) cudaGraphDestroy(g);
        return nl;
      }
      total += nl;
      dofs += substep_dofs(s, j);
    }
    SWE_CUDA(cudaStreamEndCapture(s->stream, &g));
    cudaError_t ce = cudaGraphInstantiate(&s->graph, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) {
      s->graph = nullptr;
      return fail(SWE_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ce));
    }
    s->graph_launches = total;
    s->graph_dofs = dofs;
  }
  for (int32_t i = 0; i < n_macro; ++i) {
    SWE_CUDA(cudaGraphLaunch(s->graph, s->stream));
    s->launches += s->graph_launches;
    s->dof_updates += s->graph_dofs;
    s->k += period;
  }
  return SWE_OK;
}

int swe_limit(swe_solver* s, int32_t mask) {
  if (!s) return fail(SWE_EINVAL, "NULL argument");
  if (!s->have_state) return fail(SWE_EINVAL, "no state");
  if (!synchronous(s)) return fail(SWE_EINVAL, "state is not level-synchronous");
  if (mask & ~3) return fail(SWE_EINVAL, "unknown limiter bits");
  return launch_limit(s, mask, 0, 0, s->K);
}

int swe_get_state(const swe_solver* s, double* h, double* hu, double* hv, double* t) {
  if (!s) return fail(SWE_EINVAL, "NULL argument");
  if (!s->have_state) return fail(SWE_EINVAL, "no state");
  if (!synchronous(s)) return fail(SWE_EINVAL, "state is not level-synchronous");
  int rc = download_state(s, h, hu, hv);
  if (rc) return rc;
  if (t) *t = s->t0 + (double)s->k * s->dt_min;
  return SWE_OK;
}

int swe_stats(const swe_solver* cs, double* mass, double* injected_mass, double* hmin, int64_t* dof_updates) {
  swe_solver* s = const_cast<swe_solver*>(cs);
  if (!s) return fail(SWE_EINVAL, "NULL argument");
  if (!s->have_state) return fail(SWE_EINVAL, "no state");
  if (!synchronous(s)) return fail(SWE_EINVAL, "state is not level-synchronous");
  double* partials = reinterpret_cast<double*>(s->ws + s->lay.partials);
  double* outd = partials + 2 * (size_t)s->lay.nb_stats;
  cudaError_t ce = s->fp64 ? s->ld->stats(dev_state<double>(s), sched_of(s), s->lay.nb_stats, partials, s->stream)
                           : s->lf->stats(dev_state<float>(s), sched_of(s), s->lay.nb_stats, partials, s->stream);
  if (ce != cudaSuccess) return fail(SWE_ECUDA, std::string("stats: ") + cudaGetErrorString(ce));
  SWE_CUDA(swe::launch_stats_finalize(partials, s->lay.nb_stats, outd, s->stream));
  s->launches += 2;
  double res[2], acc[1];
  int flags = 0;
  SWE_CUDA(cudaMemcpyAsync(res, outd, 16, cudaMemcpyDeviceToHost, s->stream));
  SWE_CUDA(cudaMemcpyAsync(acc, s->ws + s->lay.acc, 8, cudaMemcpyDeviceToHost, s->stream));
  SWE_CUDA(cudaMemcpyAsync(&flags, s->ws + s->lay.flags, 4, cudaMemcpyDeviceToHost, s->stream));
  SWE_CUDA(cudaStreamSynchronize(s->stream));
  if (mass) *mass = res[0];
  if (hmin) *hmin = res[1];
  if (injected_mass) *injected_mass = acc[0];
  if (dof_updates) *dof_updates = s->dof_updates;
  if (flags & 1) return fail(SWE_ENAN, "non-finite values in the state");
  return SWE_OK;
}

// checkpoint: header + level array + raw device regions [q, ring) .. [means, dry], acc, macro and,
// for a compensated solver, the compensation planes
namespace {
struct CkptHeader {
  char magic[8];
  int32_t K, N, precision, L, scheme, pad;
  int64_t k, dof_updates;
  double t0, dt_min;
  uint64_t bytes_q, bytes_ring, bytes_qmid, bytes_means, bytes_dry;
  uint64_t bytes_comp;   // the compensation planes (compensated solvers), else 0
};

size_t comp_bytes(const swe_solver* s) { return s->comp ? 3 * (size_t)s->Np * s->KS * s->ts : 0; }
}  // namespace

int swe_full_state_bytes(const swe_solver* s, size_t* bytes) {
  if (!s || !bytes) return fail(SWE_EINVAL, "NULL argument");
  const size_t qb = 2 * 3 * (size_t)s->Np * s->KS * s->ts, rb = 3 * qb / 2;
  const size_t mb = (size_t)s->K * 3 * s->NPP * s->ts;
  *bytes = sizeof(CkptHeader) + (size_t)s->K * 4 + qb + rb + mb + (size_t)s->K * 4 * s->ts + s->K + 64 + 8 +
           comp_bytes(s);
  return SWE_OK;
}

int swe_get_full_state(const swe_solver* s, void* host_buf, size_t bytes) {
  size_t need;
  int rc = swe_full_state_bytes(s, &need);
  if (rc) return rc;
  if (!host_buf || bytes < need) return fail(SWE_EINVAL, "buffer too small");
  if (!s->have_state) return fail(SWE_EINVAL, "no state");
  CkptHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "SWEGB300", 8);
  h.K = s->K; h.N = s->N; h.precision = s->prm.precision; h.L = s->L;
  h.scheme = s->prm.scheme; h.pad = 0;
  h.k = s->k; h.dof_updates = s->dof_updates; h.t0 = s->t0; h.dt_min = s->dt_min;
  h.bytes_q = 2 * 3 * (uint64_t)s->Np * s->KS * s->ts;
  h.bytes_ring = 3 * h.bytes_q / 2;
  h.bytes_qmid = (uint64_t)s->K * 3 * s->NPP * s->ts;
  h.bytes_means = (uint64_t)s->K * 4 * s->ts;
  h.bytes_dry = s->K;
  h.bytes_comp = comp_bytes(s);
  char* p = reinterpret_cast<char*>(host_buf);
  std::memcpy(p, &h, sizeof(h)); p += sizeof(h);
  std::memcpy(p, s->level.data(), (size_t)s->K * 4); p += (size_t)s->K * 4;
  cudaStream_t st = s->stream;
  SWE_CUDA(cudaMemcpyAsync(p, s->ws + s->lay.q, h.bytes_q, cudaMemcpyDeviceToHost, st)); p += h.bytes_q;
  SWE_CUDA(cudaMemcpyAsync(p, s->ws + s->lay.ring, h.bytes_ring, cudaMemcpyDeviceToHost, st)); p += h.bytes_ring;
  SWE_CUDA(cudaMemcpyAsync(p, s->ws + s->lay.qmid, h.bytes_qmid, cudaMemcpyDeviceToHost, st)); p += h.bytes_qmid;
  SWE_CUDA(cudaMemcpyAsync(p, s->ws + s->lay.means, h.bytes_means, cudaMemcpyDeviceToHost, st)); p += h.bytes_means;
  SWE_CUDA(cudaMemcpyAsync(p, s->ws + s->lay.dry, h.bytes_dry, cudaMemcpyDeviceToHost, st)); p += h.bytes_dry;
  SWE_CUDA(cudaMemcpyAsync(p, s->ws + s->lay.acc, 64, cudaMemcpyDeviceToHost, st)); p += 64;
  SWE_CUDA(cudaMemcpyAsync(p, s->ws + s->lay.macro, 8, cudaMemcpyDeviceToHost, st)); p += 8;
  if (h.bytes_comp) SWE_CUDA(cudaMemcpyAsync(p, s->ws + s->lay.comp, h.bytes_comp, cudaMemcpyDeviceToHost, st));
  SWE_CUDA(cudaStreamSynchronize(st));
  return SWE_OK;
}

int swe_set_full_state(swe_solver* s, const void* host_buf, size_t bytes) {
  size_t need;
  int rc = swe_full_state_bytes(s, &need);
  if (rc) return rc;
  if (!host_buf || bytes < need) return fail(SWE_EINVAL, "buffer too small");
  if (!s->have_B) return fail(SWE_EINVAL, "swe_set_bathymetry must come first");
  CkptHeader h;
  const char* p = reinterpret_cast<const char*>(host_buf);
  std::memcpy(&h, p, sizeof(h)); p += sizeof(h);
  if (std::memcmp(h.magic, "SWEGB300", 8) != 0 || h.K != s->K || h.N != s->N || h.precision != s->prm.precision ||
      h.scheme != s->prm.scheme || h.bytes_comp != comp_bytes(s))
    return fail(SWE_EINVAL, "checkpoint does not match this solver");
  // every size and value taken from the buffer is checked before it is used: the
  // sections must have this solver's layout (a corrupted header must not steer a
  // copy past a workspace region or past the caller's buffer)
  const uint64_t bq = 2 * 3 * (uint64_t)s->Np * s->KS * s->ts;
  if (h.bytes_q != bq || h.bytes_ring != 3 * bq / 2 || h.bytes_qmid != (uint64_t)s->K * 3 * s->NPP * s->ts ||
      h.bytes_means != (uint64_t)s->K * 4 * s->ts || h.bytes_dry != (uint64_t)s->K)
    return fail(SWE_EINVAL, "checkpoint section sizes do not match this solver");
  if (!(h.dt_min > 0) || !std::isfinite(h.dt_min) || !std::isfinite(h.t0) || h.k < 0 || h.dof_updates < 0)
    return fail(SWE_EINVAL, "checkpoint holds an invalid time, step count or dt_min");
  std::vector<int32_t> lev(s->K);
  std::memcpy(lev.data(), p, (size_t)s->K * 4); p += (size_t)s->K * 4;
  for (int32_t v : lev)
    if (v < 1 || v > s->prm.nlevels_max) return fail(SWE_EINVAL, "checkpoint level out of 1..nlevels_max");
  s->have_state = false;  // no state to carry across the re-ordering
  if ((rc = apply_levels(s, lev, h.dt_min))) return rc;
  cudaStream_t st = s->stream;
  SWE_CUDA(cudaMemcpyAsync(s->ws + s->lay.q, p, h.bytes_q, cudaMemcpyHostToDevice, st)); p += h.bytes_q;
  SWE_CUDA(cudaMemcpyAsync(s->ws + s->lay.ring, p, h.bytes_ring, cudaMemcpyHostToDevice, st)); p += h.bytes_ring;
  SWE_CUDA(cudaMemcpyAsync(s->ws + s->lay.qmid, p, h.bytes_qmid, cudaMemcpyHostToDevice, st)); p += h.bytes_qmid;
  SWE_CUDA(cudaMemcpyAsync(s->ws + s->lay.means, p, h.bytes_means, cudaMemcpyHostToDevice, st)); p += h.bytes_means;
  SWE_CUDA(cudaMemcpyAsync(s->ws + s->lay.dry, p, h.bytes_dry, cudaMemcpyHostToDevice, st)); p += h.bytes_dry;
  SWE_CUDA(cudaMemcpyAsync(s->ws + s->lay.acc, p, 64, cudaMemcpyHostToDevice, st)); p += 64;
  SWE_CUDA(cudaMemcpyAsync(s->ws + s->lay.macro, p, 8, cudaMemcpyHostToDevice, st)); p += 8;
  if (h.bytes_comp) SWE_CUDA(cudaMemcpyAsync(s->ws + s->lay.comp, p, h.bytes_comp, cudaMemcpyHostToDevice, st));
  SWE_CUDA(cudaMemsetAsync(s->ws + s->lay.flags, 0, 16, st));
  SWE_CUDA(cudaStreamSynchronize(st));
  s->k = h.k;
  s->t0 = h.t0;
  s->dof_updates = h.dof_updates;
  s->have_state = true;
  return SWE_OK;
}

int swe_level_info(const swe_solver* s, int32_t* L, int32_t* counts, double* dt_min) {
  if (!s) return fail(SWE_EINVAL, "NULL argument");
  if (L) *L = s->L;
  if (counts)
    for (int l = 1; l <= s->L; ++l) counts[l - 1] = s->off[l] - s->off[l - 1];
  if (dt_min) *dt_min = s->dt_min;
  return SWE_OK;
}

namespace {
// s->cfg from the occupancy limits in s->cfg_max and the solver's CTA cap
int apply_launch_config(swe_solver* s) {
  int dev = 0, nsm = 0;
  SWE_CUDA(cudaGetDevice(&dev));
  SWE_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  auto cap = [&](int maxgrid) {
    if (s->ctas_per_sm == 0) return maxgrid;
    const int g = nsm * s->ctas_per_sm;
    return g < maxgrid ? g : maxgrid;
  };
  s->cfg = s->cfg_max;
  s->cfg.grid_stage = cap(s->cfg_max.grid_stage);
  s->cfg.grid_tc = cap(s->cfg_max.grid_tc);
  s->cfg.grid_tvb = cap(s->cfg_max.grid_tvb);
  s->cfg.grid_pos = cap(s->cfg_max.grid_pos);
  invalidate_graph(s);
  return SWE_OK;
}
}  // namespace

int swe_set_launch_config(swe_solver* s, int32_t ctas_per_sm) {
  if (!s || ctas_per_sm < 0) return fail(SWE_EINVAL, "bad arguments");
  s->ctas_per_sm = ctas_per_sm;
  return apply_launch_config(s);
}

int swe_set_tc_warps(swe_solver* s, int32_t warps) {
  if (!s) return fail(SWE_EINVAL, "bad arguments");
  if (!s->tc) return fail(SWE_EUNSUPPORTED, "warps per CTA apply to the FP32 tensor-core tier only");
  swe::KernelCfg c = s->cfg_max;
  const cudaError_t e = s->lf->tc_config(&c, warps);
  if (e == cudaErrorInvalidValue) return fail(SWE_EINVAL, "that many warps per CTA do not fit on an SM (1..8)");
  if (e != cudaSuccess) return fail(SWE_ECUDA, std::string("tc_config: ") + cudaGetErrorString(e));
  s->cfg_max = c;
  return apply_launch_config(s);
}

int swe_set_farfield(swe_solver* s, int32_t enable, double h, double hu, double hv) {
  if (!s || (enable != 0 && enable != 1)) return fail(SWE_EINVAL, "bad arguments");
  if (enable && !(std::isfinite(h) && std::isfinite(hu) && std::isfinite(hv) && h >= 0.0))
    return fail(SWE_EINVAL, "far-field state must be finite with h >= 0");
  s->ff[0] = enable ? h : 0.0;
  s->ff[1] = enable ? hu : 0.0;
  s->ff[2] = enable ? hv : 0.0;
  s->open_face.assign((size_t)3 * s->K, enable ? 1 : 0);
  invalidate_graph(s);
  return upload_mesh(s);
}

int swe_set_open_faces(swe_solver* s, const uint8_t* open) {
  if (!s || !open) return fail(SWE_EINVAL, "NULL argument");
  for (size_t i = 0; i < (size_t)3 * s->K; ++i)
    if (open[i] > 1) return fail(SWE_EINVAL, "open-face flags must be 0 or 1");
  s->open_face.assign(open, open + (size_t)3 * s->K);
  invalidate_graph(s);
  return upload_mesh(s);
}

// ---- persistent batched launch --------------------------------------------

extern "C++" {
namespace {

int batch_period(const swe_solver* s) { return 1 << (s->L - 1); }

bool batch_tvb(const swe_solver* s) { return (s->prm.limiter_mask & SWE_LIM_TVB) != 0; }

// tickets of one phase: tiles of kBatchStageTile elements (stage) or kBatchTvbTile (TVB)
int batch_tiles(int nactive, int kind) {
  const int t = kind == 0 ? swe::kBatchStageTile : swe::kBatchTvbTile;
  return (nactive + t - 1) / t;
}

// tickets of one macro step of a solver
int batch_tickets_per_macro(const swe_solver* s) {
  int n = 0;
  for (int j = 0; j < batch_period(s); ++j) {
    const int na = s->off[active_levels(s, j)];
    n += batch_tiles(na, 0) + (batch_tvb(s) ? batch_tiles(na, 1) : 0);
  }
  return n;
}

// Group the solvers by precision tier and scheme code, at most kBatchMaxScn per group.
std::vector<BatchGroup> batch_groups(swe_solver* const* solvers, int n) {
  std::vector<BatchGroup> gs;
  for (int i = 0; i < n; ++i) {
    const swe_solver* s = solvers[i];
    BatchGroup* g = nullptr;
    for (BatchGroup& c : gs)
      if (c.fp64 == s->fp64 && c.tc == s->tc && c.code == s->code && (int)c.idx.size() < swe::kBatchMaxScn) g = &c;
    if (!g) {
      gs.emplace_back();
      g = &gs.back();
      g->fp64 = s->fp64;
      g->tc = s->tc;
      g->code = s->code;
    }
    g->idx.push_back(i);
  }
  return gs;
}

// Workspace layout of the batch (each section 256-byte aligned): per group the
// control block, the ticket segments (capacity for max_macro macro steps of every
// scenario), the counters done / ran / status (one int each per scenario), the
// release flags and the macro steps of the call.
size_t batch_layout(std::vector<BatchGroup>& gs, swe_solver* const* solvers, int max_macro) {
  size_t off = 0;
  for (BatchGroup& g : gs) {
    int cap = 0, tcap = 0;
    for (int i : g.idx) {
      cap += max_macro * batch_period(solvers[i]) * (batch_tvb(solvers[i]) ? 2 : 1);
      tcap += max_macro * batch_tickets_per_macro(solvers[i]);
    }
    g.seg_cap = cap;
    g.ticket_cap = tcap;
    const size_t n = g.idx.size();
    g.off_ctl = off;
    off = align256(off + sizeof(swe::BatchCtl));
    g.off_segs = off;
    off = align256(off + (size_t)cap * sizeof(swe::BatchSeg));
    g.off_cnt = off;
    off = align256(off + 3 * n * sizeof(int));
    g.off_release = off;
    off = align256(off + n * sizeof(int));
    g.off_nmacro = off;
    off = align256(off + n * sizeof(int));
    g.off_segof = off;
    off = align256(off + (size_t)tcap * sizeof(int));
  }
  return off;
}

// Ticket segments of one call: the phases of every scenario (per macro step and
// finest substep: the stage kernel, then the TVB limiter), ordered phase by phase,
// round-robin over the scenarios, each after the tickets of its scenario's earlier
// phases.
void batch_segments(BatchGroup& g, const std::vector<swe_solver*>& solvers, const int32_t* nmacro) {
  g.segs.clear();
  const int n = (int)g.idx.size();
  std::vector<int> nph(n), need(n, 0);
  int maxp = 0;
  for (int a = 0; a < n; ++a) {
    const swe_solver* s = solvers[g.idx[a]];
    nph[a] = nmacro[g.idx[a]] * batch_period(s) * (batch_tvb(s) ? 2 : 1);
    maxp = std::max(maxp, nph[a]);
  }
  int t0 = 0;
  for (int ph = 0; ph < maxp; ++ph)
    for (int a = 0; a < n; ++a) {
      if (ph >= nph[a]) continue;
      const swe_solver* s = solvers[g.idx[a]];
      const int per = batch_period(s), kinds = batch_tvb(s) ? 2 : 1;
      const int step = ph / kinds;   // substeps since the start of the call
      const int j = step % per;
      swe::BatchSeg sg;
      std::memset(&sg, 0, sizeof(sg));
      sg.t0 = t0;
      sg.nactive = s->off[active_levels(s, j)];
      sg.kind = ph % kinds;
      sg.ntiles = batch_tiles(sg.nactive, sg.kind);
      sg.need = need[a];
      sg.scn = a;
      sg.j = j;
      sg.kofs = step;
      sg.first = ph == 0 ? 1 : 0;
      need[a] += sg.ntiles;
      t0 += sg.ntiles;
      g.segs.push_back(sg);
    }
  g.seg_of.resize(t0);
  for (size_t q = 0; q < g.segs.size(); ++q)
    for (int t = 0; t < g.segs[q].ntiles; ++t) g.seg_of[g.segs[q].t0 + t] = (int)q;
}

template <typename T>
swe::BatchLaunch<T> batch_params(const swe_batch* b, const BatchGroup& g) {
  swe::BatchLaunch<T> bl;
  std::memset(&bl, 0, sizeof(bl));
  for (size_t a = 0; a < g.idx.size(); ++a) {
    swe_solver* s = b->solvers[g.idx[a]];
    bl.scn[a].s = dev_state<T>(s);
    bl.scn[a].sc = sched_of(s);
    bl.scn[a].ph = phys_of(s, s->prm.limiter_mask);
    bl.scn[a].j = 0;
    bl.scn[a].nactive = s->K;
    bl.scn[a].mode = 0;
    bl.period[a] = batch_period(s);
  }
  const size_t n = g.idx.size();
  bl.segs = reinterpret_cast<const swe::BatchSeg*>(b->ws + g.off_segs);
  bl.seg_of = reinterpret_cast<const int*>(b->ws + g.off_segof);
  bl.ctl = reinterpret_cast<swe::BatchCtl*>(b->ws + g.off_ctl);
  bl.done = reinterpret_cast<int*>(b->ws + g.off_cnt);
  bl.ran = bl.done + n;
  bl.status = bl.done + 2 * n;
  bl.release = reinterpret_cast<const int*>(b->ws + g.off_release);
  bl.nscn = (int)n;
  return bl;
}

template <typename T>
cudaError_t batch_enqueue_group(swe_batch* b, const BatchGroup& g) {
  const swe_solver* s0 = b->solvers[g.idx[0]];
  const swe::Launchers<T>* lt;
  if constexpr (sizeof(T) == 8) lt = s0->ld; else lt = s0->lf;
  const swe::BatchLaunch<T> bl = batch_params<T>(b, g);
  cudaError_t e;
  // a fresh queue: head and the per-scenario counters start at zero
  if ((e = cudaMemsetAsync(b->ws + g.off_ctl, 0, sizeof(int), g.stream))) return e;
  if ((e = cudaMemsetAsync(b->ws + g.off_cnt, 0, 3 * g.idx.size() * sizeof(int), g.stream))) return e;
  if ((e = lt->batch(bl, g.tc, g.grid, s0->cfg, g.stream))) return e;
  return swe::launch_batch_finish<T>(bl, reinterpret_cast<const int*>(b->ws + g.off_nmacro), g.stream);
}

}  // namespace
}  // extern "C++"

int swe_batch_workspace_bytes(swe_solver* const* solvers, int32_t n, int32_t max_macro, size_t* bytes) {
  if (!solvers || n < 1 || max_macro < 1 || !bytes) return fail(SWE_EINVAL, "bad arguments");
  for (int i = 0; i < n; ++i)
    if (!solvers[i] || !solvers[i]->have_state || !(solvers[i]->dt_min > 0))
      return fail(SWE_EINVAL, "every solver needs state and levels");
  std::vector<BatchGroup> gs = batch_groups(solvers, n);
  *bytes = batch_layout(gs, solvers, max_macro);
  return SWE_OK;
}

int swe_batch_create(swe_solver* const* solvers, int32_t n, int32_t max_macro, void* dev_workspace, size_t bytes,
                     void* stream, swe_batch** out) {
  if (!solvers || n < 1 || max_macro < 1 || !out) return fail(SWE_EINVAL, "bad arguments");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    swe_solver* s = solvers[i];
    if (!s || !s->have_state || !(s->dt_min > 0)) return fail(SWE_EINVAL, "every solver needs state and levels");
    if (!synchronous(s)) return fail(SWE_EINVAL, "every solver must be level-synchronous");
    if (s->comp) return fail(SWE_EUNSUPPORTED, "a compensated solver cannot join a batch");
    if (!s->stream) return fail(SWE_EINVAL, "batched solvers need their own (non-default) streams");
    for (int j = 0; j < i; ++j)
      if (solvers[j] == s) return fail(SWE_EINVAL, "a solver appears twice in the batch");
  }
  if (!stream) return fail(SWE_EINVAL, "the batch needs a non-default stream");
  if (!dev_workspace || (reinterpret_cast<uintptr_t>(dev_workspace) & 255))
    return fail(SWE_EINVAL, "the batch workspace must be 256-byte aligned device memory");
  // every return before the end releases what was created so far (streams, events)
  std::unique_ptr<swe_batch, void (*)(swe_batch*)> b(new (std::nothrow) swe_batch, swe_batch_destroy);
  if (!b) return fail(SWE_ENOMEM, "host allocation failed");
  b->solvers.assign(solvers, solvers + n);
  b->stream = reinterpret_cast<cudaStream_t>(stream);
  b->max_macro = max_macro;
  b->groups = batch_groups(solvers, n);
  const size_t need = batch_layout(b->groups, solvers, max_macro);
  if (bytes < need) return fail(SWE_ENOMEM, "batch workspace smaller than swe_batch_workspace_bytes");
  b->ws = static_cast<char*>(dev_workspace);
  b->ws_bytes = bytes;
  b->hold.assign(n, 0);
  b->dofs.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    swe_solver* s = solvers[i];
    for (int j = 0; j < batch_period(s); ++j) b->dofs[i] += substep_dofs(s, j);
    b->versions.push_back(s->sched_version);
  }
  // grids: every group's kernel is given as many CTAs as fit on the GPU; the groups
  // run side by side and the hardware places their CTAs as room frees up. A CTA takes
  // tickets only while it is resident, so one that starts late takes fewer, and no
  // group is held to a share that leaves SMs idle once the others are done.
  int dev = 0, nsm = 0;
  SWE_CUDA(cudaGetDevice(&dev));
  SWE_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    BatchGroup& g = b->groups[gi];
    const swe_solver* s0 = solvers[g.idx[0]];
    const int occ = g.tc ? s0->cfg_max.occ_batch_tc : s0->cfg_max.occ_batch;
    if (occ < 1) return fail(SWE_ECUDA, "the batch kernel does not fit on an SM");
    g.grid = occ * nsm;
    SWE_CUDA(cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking));
    SWE_CUDA(cudaEventCreateWithFlags(&g.join, cudaEventDisableTiming));
  }
  SWE_CUDA(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  SWE_CUDA(cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming));
  b->join.resize(n, nullptr);
  for (int i = 0; i < n; ++i) SWE_CUDA(cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming));
  // the captured step: per group (a parallel branch) fresh counters, the persistent
  // kernel and the macro-counter update
  cudaGraph_t graph = nullptr;
  SWE_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t ce = cudaEventRecord(b->fork, b->stream);
  for (size_t gi = 0; gi < b->groups.size() && ce == cudaSuccess; ++gi) {
    BatchGroup& g = b->groups[gi];
    ce = cudaStreamWaitEvent(g.stream, b->fork, 0);
    if (ce == cudaSuccess) ce = g.fp64 ? batch_enqueue_group<double>(b.get(), g) : batch_enqueue_group<float>(b.get(), g);
    if (ce == cudaSuccess) ce = cudaEventRecord(g.join, g.stream);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(b->stream, g.join, 0);
  }
  cudaError_t ce2 = cudaStreamEndCapture(b->stream, &graph);
  if (ce != cudaSuccess || ce2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(SWE_ECUDA, std::string("batch capture: ") + cudaGetErrorString(ce != cudaSuccess ? ce : ce2));
  }
  ce = cudaGraphInstantiate(&b->graph, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) {
    b->graph = nullptr;
    return fail(SWE_ECUDA, std::string("batch instantiate: ") + cudaGetErrorString(ce));
  }
  *out = b.release();
  return SWE_OK;
}

int swe_batch_set_wait_limit(swe_batch* b, double seconds) {
  if (!b || !(seconds > 0.0) || !(seconds < 3600.0)) return fail(SWE_EINVAL, "wait limit must be in (0, 3600) s");
  b->wait_s = seconds;
  return SWE_OK;
}

int swe_batch_hold(swe_batch* b, int32_t i, int32_t hold) {
  if (!b || i < 0 || i >= (int32_t)b->solvers.size()) return fail(SWE_EINVAL, "bad scenario index");
  b->hold[i] = hold ? 1 : 0;
  return SWE_OK;
}

int swe_batch_step(swe_batch* b, const int32_t* n_macro_each, int32_t* status_each) {
  if (!b || !n_macro_each || !status_each) return fail(SWE_EINVAL, "bad arguments");
  const int n = (int)b->solvers.size();
  for (int i = 0; i < n; ++i) {
    if (n_macro_each[i] < 0 || n_macro_each[i] > b->max_macro)
      return fail(SWE_EINVAL, "n_macro_each outside 0..max_macro");
    const swe_solver* s = b->solvers[i];
    if (s->sched_version != b->versions[i])
      return fail(SWE_EINVAL, "a solver's levels, order or boundary faces changed since swe_batch_create");
    if (!s->have_state || !synchronous(s)) return fail(SWE_EINVAL, "a solver has no valid level-synchronous state");
  }
  const bool rebuild = b->last_nmacro.size() != (size_t)n ||
                       !std::equal(b->last_nmacro.begin(), b->last_nmacro.end(), n_macro_each);
  // this call's tables: ticket segments (when the macro steps changed), the control
  // block, the release flags and the macro steps, uploaded on the batch stream
  for (BatchGroup& g : b->groups) {
    if (rebuild) {
      batch_segments(g, b->solvers, n_macro_each);
      if ((int)g.segs.size() > g.seg_cap || (int)g.seg_of.size() > g.ticket_cap)
        return fail(SWE_EINVAL, "internal: ticket table overflow");
      if (!g.segs.empty()) {
        SWE_CUDA(cudaMemcpyAsync(b->ws + g.off_segs, g.segs.data(), g.segs.size() * sizeof(swe::BatchSeg),
                                 cudaMemcpyHostToDevice, b->stream));
        SWE_CUDA(cudaMemcpyAsync(b->ws + g.off_segof, g.seg_of.data(), g.seg_of.size() * sizeof(int),
                                 cudaMemcpyHostToDevice, b->stream));
      }
    }
    swe::BatchCtl ctl;
    std::memset(&ctl, 0, sizeof(ctl));
    ctl.total = g.segs.empty() ? 0 : g.segs.back().t0 + g.segs.back().ntiles;
    ctl.nseg = (int)g.segs.size();
    ctl.wait_ns = (long long)(b->wait_s * 1e9);
    SWE_CUDA(cudaMemcpyAsync(b->ws + g.off_ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice, b->stream));
    std::vector<int> rel(g.idx.size()), nm(g.idx.size());
    for (size_t a = 0; a < g.idx.size(); ++a) {
      rel[a] = b->hold[g.idx[a]] ? 0 : 1;
      nm[a] = n_macro_each[g.idx[a]];
    }
    SWE_CUDA(cudaMemcpyAsync(b->ws + g.off_release, rel.data(), rel.size() * sizeof(int), cudaMemcpyHostToDevice,
                             b->stream));
    SWE_CUDA(cudaMemcpyAsync(b->ws + g.off_nmacro, nm.data(), nm.size() * sizeof(int), cudaMemcpyHostToDevice,
                             b->stream));
  }
  b->last_nmacro.assign(n_macro_each, n_macro_each + n);
  // the batch stream waits for work already queued on the solvers' own streams
  for (int i = 0; i < n; ++i) {
    SWE_CUDA(cudaEventRecord(b->join[i], b->solvers[i]->stream));
    SWE_CUDA(cudaStreamWaitEvent(b->stream, b->join[i], 0));
  }
  SWE_CUDA(cudaGraphLaunch(b->graph, b->stream));
  b->launches += 2 * (int64_t)b->groups.size();
  // per scenario: status and tiles run, read back when the step is over
  std::vector<std::vector<int>> host(b->groups.size());
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    host[gi].resize(3 * b->groups[gi].idx.size());
    SWE_CUDA(cudaMemcpyAsync(host[gi].data(), b->ws + b->groups[gi].off_cnt, host[gi].size() * sizeof(int),
                             cudaMemcpyDeviceToHost, b->stream));
  }
  SWE_CUDA(cudaEventRecord(b->done, b->stream));
  SWE_CUDA(cudaStreamSynchronize(b->stream));
  int rc = SWE_OK;
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    const BatchGroup& g = b->groups[gi];
    const size_t m = g.idx.size();
    for (size_t a = 0; a < m; ++a) {
      const int i = g.idx[a];
      swe_solver* s = b->solvers[i];
      const int st = host[gi][2 * m + a], ran = host[gi][m + a];
      status_each[i] = st;
      if (st == SWE_OK) {
        s->k += (int64_t)n_macro_each[i] << (s->L - 1);
        s->dof_updates += b->dofs[i] * n_macro_each[i];
      } else {
        rc = st;
        // gave up before any of its tiles ran: its state is as before the call;
        // otherwise part of a macro step ran and the state must be set again
        if (ran > 0) s->have_state = false;
      }
    }
  }
  for (int i = 0; i < n; ++i) SWE_CUDA(cudaStreamWaitEvent(b->solvers[i]->stream, b->done, 0));
  if (rc != SWE_OK) return fail(rc, "a scenario's bounded wait gave up (status_each)");
  return SWE_OK;
}

int swe_batch_launches(const swe_batch* b, int64_t* launches) {
  if (!b || !launches) return fail(SWE_EINVAL, "NULL argument");
  *launches = b->launches;
  return SWE_OK;
}

void swe_batch_destroy(swe_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->done) cudaEventDestroy(b->done);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  for (BatchGroup& g : b->groups) {
    if (g.stream) {
      cudaStreamSynchronize(g.stream);
      cudaStreamDestroy(g.stream);
    }
    if (g.join) cudaEventDestroy(g.join);
  }
  delete b;
}

int swe_profile_substeps(swe_solver* s, int32_t n, double* out) {
  if (!s || n < 0 || !out) return fail(SWE_EINVAL, "bad arguments");
  if (!s->have_state) return fail(SWE_EINVAL, "no state");
  if (!(s->dt_min > 0)) return fail(SWE_EINVAL, "levels / dt_min not set up");
  KernelTimer tm;
  const int64_t period = 1LL << (s->L - 1);
  int rc = SWE_OK;
  for (int32_t i = 0; i < n && rc == SWE_OK; ++i) {
    const int j = (int)(s->k % period);
    int nl = enqueue_substep(s, j, &tm);
    if (nl < 0) { rc = nl; break; }
    s->launches += nl;
    s->dof_updates += substep_dofs(s, j);
    s->k++;
  }
  cudaError_t ce = cudaStreamSynchronize(s->stream);
  for (int i = 0; i < 6; ++i) out[i] = 0.0;
  for (size_t i = 0; 2 * i + 1 < tm.ev.size(); ++i) {
    float ms = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, tm.ev[2 * i], tm.ev[2 * i + 1]);
    const int kind = tm.kind[i];
    out[kind] += ms;
    if (kind == 0) { out[3] += 1; out[4] += (double)tm.elems[i]; }
    if (kind == 1) out[5] += (double)tm.elems[i];
  }
  for (cudaEvent_t e : tm.ev) cudaEventDestroy(e);
  if (rc) return rc;
  if (ce != cudaSuccess) return fail(SWE_ECUDA, std::string("profile: ") + cudaGetErrorString(ce));
  return SWE_OK;
}

int swe_kernel_launches(const swe_solver* s, int64_t* launches) {
  if (!s || !launches) return fail(SWE_EINVAL, "NULL argument");
  *launches = s->launches;
  return SWE_OK;
}

}  // extern "C"
