// Plain data shared by the host launch code and the device kernels (no device
// code, so host-only translation units can include it).
#pragma once

#include <stdint.h>
#include <vector_types.h>

namespace swe {

constexpr int kMaxLevels = 8;
constexpr int kBlock = 128;

// Scheme code: the polynomial order N (bits 0-3), plus
//   kColloc   the nodal-collocation variant (volume and face integrals of the nodal
//             interpolants: the "cubature points" are the Np nodes and the "Gauss
//             points" the Nfp face nodes, so the same kernels run with other operators)
//   kReduced  the rules of integration order 2N (a conical product of (N+1)^2 points,
//             N + 1 Gauss points per face) instead of 3N - 1 and 3N
constexpr int kColloc = 16;

// Boundary faces in the connectivity: a neighbour index below zero.
constexpr int kWall = -1;      // reflecting wall
constexpr int kFarField = -2;  // open: the far-field state of Phys
constexpr int kReduced = 32;

template <int NN>
struct Dims {
  static constexpr int N = NN & 15;
  static constexpr bool COLLOC = (NN & kColloc) != 0;
  static constexpr bool REDUCED = (NN & kReduced) != 0;
  // rules exact to degrees 3N - 1 and 3N: only then is the depth form of the
  // pressure for dry elements the same discretisation as the pre-balanced form
  static constexpr bool EXACT = !COLLOC && !REDUCED;
  static constexpr int NP = (N + 1) * (N + 2) / 2;
  static constexpr int NPP = (NP + 3) / 4 * 4;
  static constexpr int NFP = N + 1;
  static constexpr int NFPP = (NFP + 3) / 4 * 4;
  static constexpr int Q = REDUCED ? N + 1 : (3 * N + 1) / 2;
  static constexpr int NCUB = COLLOC ? NP : Q * Q;
  static constexpr int NG = COLLOC ? NFP : (REDUCED ? N + 1 : (3 * N + 2) / 2);
};

// Operator block (element type T), packed by the host, staged in shared memory.
// The per-element (surface, limiter) operators come first so a kernel that does
// its volume contractions elsewhere can stage only [0, TAIL).
template <int N>
struct OpLayout {
  using D = Dims<N>;
  static constexpr int LGT = 0;                                // [3 NG][NPP], Lg^T
  static constexpr int I1D = LGT + 3 * D::NG * D::NPP;         // [NG][NFPP]
  static constexpr int MW = I1D + D::NG * D::NFPP;             // [NPP] mean weights
  static constexpr int T1 = MW + D::NPP;                       // [3][NPP] P1 vertex map
  static constexpr int BARY = T1 + 3 * D::NPP;                 // [NPP][4] barycentric
  static constexpr int TAIL = BARY + 4 * D::NPP;
  static constexpr int IC = TAIL;                              // [NCUB][NPP]
  static constexpr int ICR = IC + D::NCUB * D::NPP;            // [NCUB][NPP]
  static constexpr int ICS = ICR + D::NCUB * D::NPP;           // [NCUB][NPP]
  static constexpr int PRT = ICS + D::NCUB * D::NPP;           // [NCUB][NPP], Pr^T
  static constexpr int PST = PRT + D::NCUB * D::NPP;           // [NCUB][NPP], Ps^T
  static constexpr int PT = PST + D::NCUB * D::NPP;            // [NCUB][NPP], P^T
  static constexpr int DR = PT + D::NCUB * D::NPP;             // [NP][NPP] nodal d/dr
  static constexpr int DS = DR + D::NP * D::NPP;               // [NP][NPP] nodal d/ds
  static constexpr int SIZE = DS + D::NP * D::NPP;
};

// Tensor-core tiling of the volume contractions (mma.sync, bf16 operands).
//   KP   node dimension padded to the k16 step of the interpolation
//   CT   cubature points in tiles of 8 (n of the interpolation, k of the projection)
//   NT   nodes in tiles of 8 (n of the projection and of the lift)
//   KF   the 3 Ng face Gauss points padded to the k8 step of the lift; KT = KF / 8
//   FR   rows per field of the shared flux / R tile, max(KF, NPT)
template <int N>
struct TcDims {
  using D = Dims<N>;
  static constexpr int KP = (D::NP + 15) / 16 * 16;
  static constexpr int KSTEP = KP / 16;
  static constexpr int CT = (D::NCUB + 7) / 8;
  static constexpr int NT = (D::NP + 7) / 8;
  static constexpr int NPT = 8 * NT;
  static constexpr int KF = (3 * D::NG + 7) / 8 * 8;
  static constexpr int KT = KF / 8;
  static constexpr int FR = KF > NPT ? KF : NPT;
};

// Operator fragments in register order (uint32 = two bf16), hi and lo parts.
//   INTERP [3 ops Ic,Icr,Ics][CT][KSTEP][2 parts][32 lanes][2 regs]
//   PROJ   [3 ops Pr,Ps,P][CT][NT][2 parts][32 lanes]
//   LIFT   [KT][NT][2 parts][32 lanes], the B operand -L^g^T (face points x nodes)
//   DIFF   [2 ops Dr,Ds][KP/8][NT][2 parts][32 lanes][2 regs], TF32 B operands
//          Dr^T, Ds^T (nodes x nodes) of m16n8k8.tf32
template <int N>
struct TcLayout {
  using C = TcDims<N>;
  static constexpr int INTERP = 0;
  static constexpr int PROJ = INTERP + 3 * C::CT * C::KSTEP * 2 * 64;
  static constexpr int LIFT = PROJ + 3 * C::CT * C::NT * 2 * 32;
  static constexpr int DIFF = LIFT + C::KT * C::NT * 2 * 32;
  static constexpr int SIZE = DIFF + 2 * (C::KP / 8) * C::NT * 2 * 64;
};

// Pointers into the caller-owned workspace. Nodal arrays are node-major
// ("planes"): node i of element e is at plane[i * KS + e], KS = K rounded up to
// a multiple of 32, so the threads of a warp, one element each, read and write
// whole 128-byte lines.
template <typename T>
struct DevState {
  T* q;                 // [2][3][NP][KS] double-buffered (eta, hu, hv)
  T* ring;              // [3][3][NP][KS] Adams-Bashforth history of R
  T* qmid;              // [K][3][NPP] state at the middle of the element's current step,
                        // element-major records (written only by elements with a finer
                        // neighbour, so each writer fills whole sectors)
  const T* B;           // [NP][KS]
  T* p1;                // [3][3][KS] vertex values of Pi1 (eta, hu, hv) after each commit
  const T* vb;          // [3][KS] vertex values of Pi1 B (static)
  const T* geo;         // [K][4] rx, ry, sx, sy
  const int4* conn;     // [K] neighbour across faces 0,1,2 (kWall, kFarField); .w packs neighbour faces
                        // (bits 0-5), TVB stencil (6-11) and "has a finer neighbour" (12)
  const T* tvbg;        // [K][8] alpha_i, beta_i (i = 0..2)
  T* means;             // [K][4] element means (eta, hu, hv)
  uint8_t* dry;         // [K] dry flag of the latest positivity pass
  const double* Bbar;   // [K] mean of B (FP64)
  const T* ops;         // operator block
  const uint32_t* tcops; // tensor-core operator fragments (FP32 tensor-core tier)
  double* acc;          // accumulators: [0] injected mass
  int* flags;           // [0] non-finite state detected
  long long* macro;     // macro-step counter (advanced on the device)
  T* comp;              // [3][NP][KS] rounding error of the last state update, or nullptr
                        // (not compensated)
};

struct Sched {
  int K;                     // elements
  int KS;                    // element stride of the node planes (K rounded up to 32)
  int L;                     // levels in use
  int off[kMaxLevels + 1];   // level l (1-based) occupies [off[l-1], off[l])
  double dt_min;
  double dtl_d[kMaxLevels];  // step of level l = 2^{l-1} dt_min, in both precisions
  float dtl_f[kMaxLevels];
};

struct Phys {
  double g, h0, eps, tvb_M, tvb_nu;
  double hvel;   // velocity u = hu/h only where h > hvel = h0 (1 + 1e-6), else 0
  double ff_h, ff_hu, ff_hv;   // far-field state of the open boundary faces (kFarField)
  float eps_f;
  int pp, dry_mode;
};

// One scenario: its device arrays, schedule and physics. The limiter bodies read
// only this part, so the separate launch and the batch kernel pass them the same type.
template <typename T>
struct ScnParams {
  DevState<T> s;
  Sched sc;
  Phys ph;
};

template <typename T>
struct StageParams : ScnParams<T> {
  int j;          // substep within the macro step
  int nactive;    // elements [0, nactive) are active
  int mode;       // 0: R + commit + positivity; 1: R only, written to out
  T* out;         // mode 1: [3][K][NP], caller order
  const int* perm;
};

template <typename T>
struct LimitParams : ScnParams<T> {
  int j;
  int nactive;
  int post_stage;  // 1: limit the just-committed state of active elements; 0: current state
};

// ---- persistent batched launch ------------------------------------------
// Many scenarios advance in one persistent kernel per (tier, scheme and order)
// group. The work is a queue of tickets; a ticket is one tile of elements of one
// phase (the stage kernel or the TVB limiter of one finest substep) of one
// scenario, taken by one warp. Tickets are ordered phase by phase, round-robin over the scenarios, so a
// ticket depends only on tickets handed out before it (its scenario's earlier
// phases): the lowest outstanding ticket can always run, with or without every CTA
// resident.

constexpr int kBatchTile = 128;       // threads per CTA of the SIMT body (four warps, each taking its own
                                      // tickets); the tensor-core body runs the solvers' warps per CTA
constexpr int kBatchStageTile = 64;   // elements per stage ticket: two warp-tiles
constexpr int kBatchTvbTile = 128;    // elements per TVB ticket: four per lane
constexpr int kBatchMaxScn = 48;    // scenarios per group launch (kernel-parameter space)

struct alignas(16) BatchSeg {   // one phase of one scenario: tickets [t0, t0 + ntiles)
  int t0;
  int ntiles;
  int need;         // tiles of this scenario that must be complete first
  int scn;          // scenario (index in the group)
  int nactive;      // active elements
  int kind;         // 0: stage kernel, 1: TVB limiter
  int j;            // substep within the macro step
  int kofs;         // k of this phase minus k at the start of the call
  int first;        // the scenario's first phase in this call: waits for its release
  int pad[3];
};
static_assert(sizeof(BatchSeg) == 48, "a segment is three 16-byte words");

struct BatchCtl {   // per group, in the batch workspace
  int head;         // next ticket
  int total;        // tickets of this call
  int nseg;         // segments of this call
  int pad;
  long long wait_ns;  // bound of every wait
};

template <typename T>
struct BatchLaunch {
  // the parameters of each scenario (j = 0, nactive = K, mode 0; a segment supplies
  // the substep and the active count, and the limiter runs on the just-committed
  // state). They stay in the kernel-parameter space: the stage and limiter bodies
  // read them through the constant cache, which the streaming node data never evicts
  StageParams<T> scn[kBatchMaxScn];
  const BatchSeg* segs;
  const int* seg_of;  // [tickets] the segment of each ticket
  BatchCtl* ctl;
  int* done;          // [nscn] tiles completed (run or skipped) per scenario
  int* ran;           // [nscn] tiles run per scenario
  int* status;        // [nscn] 0, or SWE_ETIMEOUT when a wait gave up
  const int* release; // [nscn] nonzero: the scenario may start
  int nscn;
  int period[kBatchMaxScn];   // finest substeps per macro step of each scenario
};

}  // namespace swe
