/*
 * swe.h -- C ABI of the GB300 nodal discontinuous Galerkin shallow-water engine.
 *
 * The library evaluates and advances the semi-discrete nodal DG discretisation
 * of the 2D nonlinear shallow water equations on triangles described in
 * "GPU Accelerated Discontinuous Galerkin Methods for Shallow Water Equations"
 * (Gandham, Medina, Warburton, arXiv:1403.1661):
 *   - Section 2, Eq. swe_conservative: Q = (h, hu, hv), fluxes F, G, source S;
 *   - Section 3, Eq. weak_form / Eq. ode: Lagrange basis on Warp & Blend nodes,
 *     cubature volume integrals, Gauss surface integrals, dQ/dt = R(Q);
 *   - Section 4, Eq. cfl and Algorithm 1: per-element time step, levels,
 *     multirate Adams-Bashforth (MRAB3);
 *   - Section 5.1, Eq. well_balance: well-balanced Lax-Friedrichs flux;
 *   - Section 5.2, Algorithms 2 and 3: limiting and the positivity limiter;
 *   - Section 5.3, Eq. modified_TVB: TVB limiter with positivity modification;
 *   - Section 7 (Eq. kernels): volume, surface and update kernels.
 *
 * Conventions (all entry points):
 *   - Every call returns SWE_OK (0) or a negative SWE_E* code; swe_last_error()
 *     gives a message for the calling thread's last failure.
 *   - Host arrays are read (or written) during the call only; the caller keeps
 *     ownership. Device memory is owned by the caller: swe_solver_create takes
 *     one device workspace of swe_workspace_bytes() bytes and the library never
 *     calls cudaMalloc/cudaFree. The library owns only the opaque handles.
 *   - All device work is enqueued on the caller's CUDA stream (cudaStream_t
 *     passed as void*). Calls that return host data (swe_get_state,
 *     swe_stats, swe_get_full_state) synchronise that stream.
 *   - Nodal arrays are element-major [K][Np] in the caller's element order and
 *     the library's node order (swe_ref_nodes); K = number of triangles,
 *     Np = (N+1)(N+2)/2.
 *   - Triangle vertices may come in either orientation; each element is made
 *     counter-clockwise (its vertices 1 and 2 swapped) and face f joins vertices
 *     f and f+1 mod 3 of the oriented element.
 */
#ifndef SWE_GB300_H
#define SWE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define SWE_OK 0
#define SWE_EINVAL (-1)       /* bad argument, bad mesh, call out of order      */
#define SWE_ENOMEM (-2)       /* workspace too small / over a memory budget      */
#define SWE_ECUDA (-3)        /* a CUDA runtime call failed                      */
#define SWE_ENAN (-4)         /* non-finite values detected in the state         */
#define SWE_ETIMEOUT (-5)     /* a bounded device wait gave up                   */
#define SWE_EUNSUPPORTED (-6) /* order / precision not built into this library   */

/* ---- precision tiers ---------------------------------------------------- */
#define SWE_FP64 0            /* everything in double precision                  */
#define SWE_FP32 1            /* single precision, FP64 in the positivity limiter */
#define SWE_FP32_TC 2         /* SWE_FP32 with the volume contractions on tensor cores
                                 (split-BF16 products, FP32 accumulation)         */

/* ---- spatial schemes (swe_params.scheme) -------------------------------- */
#define SWE_SCHEME_CUBATURE 0     /* Section 3: cubature + Gauss rules             */
#define SWE_SCHEME_COLLOCATION 1  /* nodal collocation (fewer operations, aliased) */
#define SWE_SCHEME_CUBATURE_2N 2  /* integration order 2N (Fig. 2's caption): conical
                                     product of (N+1)^2 points, N+1 Gauss points per
                                     face; pre-balanced form everywhere             */

/* ---- limiter mask bits (Algorithm 2) ----------------------------------- */
#define SWE_LIM_PP 1          /* positivity-preserving limiter M Pi (Algorithm 3) */
#define SWE_LIM_TVB 2         /* TVB limiter Lambda Pi (Section 5.3)              */

typedef struct swe_mesh swe_mesh;
typedef struct swe_solver swe_solver;

/* Physical and numerical parameters.
 *   g        gravity (Eq. swe_conservative)
 *   h0       dry threshold (Algorithm 3); eps of Algorithm 3 is taken equal to h0
 *            when eps <= 0
 *   eps      positivity trigger of Algorithm 3 (<= 0: use h0)
 *   tvb_M    TVB constant M; tvb_nu the minmod weight nu (<= 0: 1.5)
 *   cfl      CFL number; the per-element step is cfl/(N+1)^2 * H_k / a_k (Eq. cfl)
 *   N        polynomial order (1..5 in this build; 2..5 for the collocation and
 *            order-2N schemes)
 *   nlevels_max  number of MRAB levels allowed (>= 1; 1 = single-rate AB3)
 *   precision    SWE_FP64, SWE_FP32 or SWE_FP32_TC
 *   limiter_mask SWE_LIM_PP | SWE_LIM_TVB applied after every update
 *   dry_mode     0: a dry element is reset to h = h0, hu = hv = 0 (Algorithm 3,
 *                injected mass tallied); 1: reset to its mean depth (mass kept)
 *   scheme       SWE_SCHEME_CUBATURE (the paper's: volume cubature of degree
 *                3N-1, Gauss points on the faces), SWE_SCHEME_CUBATURE_2N (the
 *                same with rules of integration order 2N) or
 *                SWE_SCHEME_COLLOCATION (fluxes at the nodes and face nodes,
 *                their interpolants integrated exactly)
 *   compensated  single-precision tiers: 1 = the state (eta, hu, hv) is updated
 *                with a compensated sum (each commit's rounding error is kept in
 *                three workspace planes and taken back at the next), so the total
 *                mass keeps to about 3e-13 of itself per step instead of about 5e-9
 *                and long runs keep FP64's accuracy (the plain update accumulates
 *                its rounding); about 11 % more time per macro step. 0 (default)
 *                or 1; ignored in FP64. A compensated solver cannot join a batch. */
typedef struct {
  double g, h0, eps, tvb_M, tvb_nu, cfl;
  int32_t N, nlevels_max, precision, limiter_mask, dry_mode, scheme;
  int32_t compensated;
} swe_params;

/* ---- library ------------------------------------------------------------ */
int swe_version(void);                      /* 10000*major + 100*minor + patch */
const char* swe_strerror(int code);
const char* swe_last_error(void);

/* Reference element sizes for order N (Section 7, Table "Notation"):
 * Np nodes, Ncub cubature points (volume rule exact to degree 3N-1),
 * Ng Gauss points per face (exact to degree 3N). Any pointer may be NULL. */
int swe_ref_sizes(int32_t N, int32_t* Np, int32_t* Ncub, int32_t* Ng);

/* Warp & Blend interpolation nodes (Section 3) in the library's node order,
 * reference triangle (-1,-1),(1,-1),(-1,1). r, s: Np doubles each (host). */
int swe_ref_nodes(int32_t N, double* r, double* s);

/* Reference operators in FP64, row-major (host), for checking against an
 * independent construction. which: 0 Ic (Ncub x Np), 1 Icr, 2 Ics,
 * 3 Pr (Np x Ncub), 4 Ps, 5 P, 6 Lg (Np x 3Ng, Section 7.2), 7 face
 * interpolation from the Nfp face nodes to the Ng Gauss points (Ng x Nfp),
 * 8 element-mean weights (Np), 9 P1-projection vertex map (3 x Np),
 * 10 cubature weights (Ncub), 11 Gauss weights (Ng). count: capacity in doubles. */
int swe_ref_operator(int32_t N, int32_t which, double* out, size_t count);

/* ---- mesh (host only) --------------------------------------------------- */
/* vx, vy: nv vertex coordinates; EToV: K x 3 vertex indices. Faces are matched
 * by their vertex pair; a face on one element only is a boundary face, a
 * reflecting wall (Section 6.5) until a solver opens it. There is no per-face
 * boundary-tag argument: the kind of each boundary face is set on the solver,
 * swe_set_farfield (all boundary faces) and swe_set_open_faces (face by face),
 * which take the place of such tags. Fails with SWE_EINVAL on degenerate
 * triangles, bad indices or faces shared by more than two triangles. */
int swe_mesh_create(const double* vx, const double* vy, int32_t nv,
                    const int32_t* EToV, int32_t K, swe_mesh** out);
void swe_mesh_destroy(swe_mesh* mesh);
int swe_mesh_num_elements(const swe_mesh* mesh, int32_t* K);
/* EToE, EToF: K x 3 (host); neighbour element / face, -1 on a boundary face. */
int swe_mesh_connectivity(const swe_mesh* mesh, int32_t* EToE, int32_t* EToF);
/* Physical coordinates of the nodes of order N: x, y are K x Np (host). */
int swe_mesh_node_coords(const swe_mesh* mesh, int32_t N, double* x, double* y);

/* The level grouping swe_setup_levels would make for nodal state (h, hu, hv)
 * (K x Np each, host, caller order): level_out (K, 1-based), dt_min_out. Host only.
 * SWE_EINVAL for a non-finite value or a state without any positive depth (the CFL
 * rule then has no wave speed). */
int swe_mesh_levels(const swe_mesh* mesh, int32_t N, const double* h, const double* hu,
                    const double* hv, double g, double cfl, int32_t nlevels_max,
                    int32_t* level_out, double* dt_min_out);

/* The CFL regroup rule of swe_regroup (Section 4's regrouping remark, Eq. cfl's
 * level rule) for given per-element steps, on the host: dt (K), the current levels
 * (K, 1-based), the substep count k and dt_min give level_out (K) = the largest l
 * with 2^{l-1} dt_min <= dt_k in 1..nlevels_max, at most old + 1, at most 1 + the
 * power of two in k; margin_out (may be NULL) = min_k dt_k / (2^{l_k - 1} dt_min).
 * Host arrays, read or written during the call only. SWE_EINVAL for NULL arrays,
 * K < 0, k < 0, dt_min not finite and > 0, a step dt_k not finite and > 0, a
 * current level outside 1..nlevels_max or nlevels_max outside 1..8. */
int swe_regroup_rule(const double* dt, const int32_t* level, int32_t K, double dt_min, int64_t k,
                     int32_t nlevels_max, int32_t* level_out, double* margin_out);

/* ---- solver -------------------------------------------------------------- */
/* Bytes of caller-owned device memory a solver for (mesh, params) needs. */
int swe_workspace_bytes(const swe_mesh* mesh, const swe_params* params, size_t* bytes);

/* Create a solver in caller-owned device memory dev_workspace (bytes >= the
 * size above, 256-byte aligned) bound to stream (cudaStream_t, may be NULL for
 * the legacy default stream). Uploads geometry and operators; no allocation of
 * device memory. The mesh may be destroyed afterwards. */
int swe_solver_create(const swe_mesh* mesh, const swe_params* params,
                      void* dev_workspace, size_t bytes, void* stream, swe_solver** out);
void swe_solver_destroy(swe_solver* solver);

/* A new non-blocking CUDA stream (cudaStream_t) for one solver or batch, and its
 * release (waits for the stream's work first). Each solver needs a stream of its
 * own: its macro step is captured into a CUDA graph on that stream, and work that
 * another thread enqueues on a stream while it is capturing invalidates the
 * capture. Stream pools that hand the same stream to several users therefore do
 * not fit. SWE_EINVAL for a NULL argument, SWE_ECUDA when the runtime fails. */
int swe_stream_create(void** out);
int swe_stream_destroy(void* stream);

/* Nodal bathymetry B (K x Np, host, FP64). Must precede swe_set_state. */
int swe_set_bathymetry(swe_solver* solver, const double* B);

/* Initial state (K x Np each, host, FP64): interpolated nodal values (the caller
 * does Pi_H). Applies the limiters of the mask to it (Algorithm 2, first line),
 * clears the Adams-Bashforth history and sets t = 0. The arrays are copied to the
 * device as they are (page-locked host memory transfers fastest); the check for
 * non-finite values, the reordering and the precision conversion run there.
 * SWE_EINVAL for a non-finite value, with the previous state left in place.
 * Synchronises the stream. */
int swe_set_state(swe_solver* solver, const double* h, const double* hu, const double* hv);

/* Group elements into MRAB levels from the current state (Eq. cfl, Section 4):
 * dt_k = cfl/(N+1)^2 * H_k / a_k, H_k = the inradius, a_k = max over the
 * element's nodes of |u| + sqrt(g max(h, 1e-2 max h)); level l holds
 * 2^{l-1} dt_min <= dt_k < 2^l dt_min (capped at nlevels_max). level_out (K,
 * caller order, 1-based) and dt_min_out may be NULL. Restarts the history.
 * SWE_ENAN, with nothing changed, if the state holds a non-finite value;
 * SWE_EINVAL if it has no positive depth. */
int swe_setup_levels(swe_solver* solver, int32_t* level_out, double* dt_min_out);

/* Force a level assignment (K, caller order, values 1..nlevels_max) and the
 * finest step dt_min (finite, > 0). Restarts the history. SWE_EINVAL otherwise. */
int swe_set_levels(swe_solver* solver, const int32_t* level, double dt_min);

/* Regroup the elements into MRAB levels at the current level-synchronous time
 * without restarting (Section 4: elements may be regrouped every few steps to
 * follow the changing CFL bound). dt_min, the time, the state and the
 * Adams-Bashforth history are kept: an element that changes level from l to
 * l' gets R at its new step times t - s dt_l' (s = 1, 2) from the quadratic
 * in time through its R at t - s dt_l (s = 1, 2, 3).
 *   level   the new levels (K, caller order, 1..nlevels_max), or NULL for the
 *           CFL rule: the largest l with 2^{l-1} dt_min <= dt_k (dt_k of
 *           Eq. cfl as in swe_setup_levels), at most one level coarser than
 *           now (the history is extrapolated over at most one old step) and
 *           at most 1 + the power of two in the substep count k.
 * Requires k >= 3 * 2^{L-1} substeps since the last restart (three R values
 * of every level) and 2^{max level - 1} dividing k; SWE_EINVAL otherwise,
 * with the solver unchanged. level_out (K, caller order) and cfl_margin_out =
 * min over elements of dt_k / (its new step) may be NULL; a margin below 1
 * means an element's CFL step fell below dt_min: restart with
 * swe_setup_levels. Runs on the device through the state staging area;
 * SWE_ENOMEM for a mesh too small for it to hold one node plane (a single
 * element of low order). Synchronises the solver's stream. */
int swe_regroup(swe_solver* solver, const int32_t* level, int32_t* level_out, double* cfl_margin_out);

/* One evaluation of R(Q) = N(Q) + S(Q^{g,+}, Q^{g,-}) (Eq. ode) at the current,
 * level-synchronous state. dev_R: device array [3][K][Np] of the solver's
 * precision (double for SWE_FP64, float otherwise), caller order, written on
 * the solver's stream. */
int swe_rhs(swe_solver* solver, void* dev_R);

/* ---- kernel-structure ablations of swe_rhs (Section 7) ------------------
 * The same R(Q) as swe_rhs, computed by another kernel structure, for timing
 * the design choices of Section 7 against the fused stage kernel:
 *   SWE_RHS_FUSED       the solver's own kernel (identical to swe_rhs)
 *   SWE_RHS_FUSED_SIMT  the fused kernel without tensor cores, operators in
 *                       shared memory (the solver's kernel unless SWE_FP32_TC)
 *   SWE_RHS_GLOBAL_OPS  the same, operators read from global memory through
 *                       the L1 cache (the operator placement of Section 7.4)
 *   SWE_RHS_SPLIT       three kernels as in Sections 7.1-7.3: traces at the
 *                       face Gauss points (Q^g) stored in device memory, the
 *                       volume term, the surface term from the stored traces
 *                       of both sides
 * Results agree with swe_rhs up to rounding (the split adds the volume and
 * surface sums in another order); SWE_RHS_FUSED_SIMT and SWE_RHS_GLOBAL_OPS
 * equal it bit for bit unless the solver uses SWE_FP32_TC. */
#define SWE_RHS_FUSED 0
#define SWE_RHS_FUSED_SIMT 1
#define SWE_RHS_GLOBAL_OPS 2
#define SWE_RHS_SPLIT 3

/* Device scratch a variant needs: 0 except for SWE_RHS_SPLIT, whose traces
 * (3 Ng x 4 values + 6 face references per element) and volume term (3 Np per
 * element) live there. SWE_EINVAL for an unknown variant. */
int swe_rhs_scratch_bytes(const swe_solver* solver, int variant, size_t* bytes);

/* R(Q) by the given variant into dev_R (layout and precision as swe_rhs).
 * dev_scratch: caller-owned device memory of at least
 * swe_rhs_scratch_bytes() bytes, 256-byte aligned (NULL when that is 0);
 * SWE_ENOMEM if it is smaller. Enqueued on the solver's stream. */
int swe_rhs_variant(swe_solver* solver, int variant, void* dev_R, void* dev_scratch, size_t scratch_bytes);

/* Advance n finest substeps of the multirate schedule (Algorithm 2). At every
 * substep k, the levels l with k mod 2^{l-1} = 0 evaluate R, take one
 * Adams-Bashforth step of 2^{l-1} dt_min and are limited. */
int swe_substep(swe_solver* solver, int32_t n);

/* Advance n macro steps (2^{L-1} finest substeps each, L = levels in use) by
 * replaying a captured CUDA graph of one macro step. Requires a
 * level-synchronous state (a multiple of 2^{L-1} substeps taken). */
int swe_step(swe_solver* solver, int32_t n_macro);

/* Apply the limiters in mask to the current level-synchronous state. */
int swe_limit(swe_solver* solver, int32_t mask);

/* Copy the current state to the host (K x Np each, FP64, caller order) and the
 * simulated time t. The conversion to the caller's layout runs on the device,
 * then one copy per array; any of h, hu, hv, t may be NULL (not copied).
 * Requires a level-synchronous state. Synchronises the stream. */
int swe_get_state(const swe_solver* solver, double* h, double* hu, double* hv, double* t);

/* Diagnostics (synchronises): mass = sum_k |D^k| mean(h), injected mass of dry
 * resets since set_state, minimum nodal depth, DOF-updates done (elements x Np x 3
 * per element step). Any pointer may be NULL. Returns SWE_ENAN if the device
 * flagged non-finite values. */
int swe_stats(const swe_solver* solver, double* mass, double* injected_mass,
              double* hmin, int64_t* dof_updates);

/* Checkpoint: swe_full_state_bytes gives the size of an opaque host buffer
 * holding the state, the Adams-Bashforth history and the substep counter;
 * restoring it into a solver created for the same mesh and parameters resumes
 * bit-identically. swe_set_full_state needs the bathymetry set first and returns
 * SWE_EINVAL, with the solver's state untouched, for a buffer smaller than
 * swe_full_state_bytes, a buffer written for another mesh size, order, tier, scheme
 * or compensation, or one whose section sizes, levels (1..nlevels_max), dt_min,
 * time or step count are invalid. */
int swe_full_state_bytes(const swe_solver* solver, size_t* bytes);
int swe_get_full_state(const swe_solver* solver, void* host_buf, size_t bytes);
int swe_set_full_state(swe_solver* solver, const void* host_buf, size_t bytes);

/* Levels in use (L), elements per level (counts[0..L-1]) and dt_min. */
int swe_level_info(const swe_solver* solver, int32_t* L, int32_t* counts, double* dt_min);

/* ---- batched scenarios -------------------------------------------------- */
/* Many independent scenarios (solvers) advanced together on one GPU. The paper
 * solves one scenario at a time; this batching is a systems layer over its method
 * (Algorithms 1-3 per scenario, unchanged). The solvers are grouped by precision
 * tier and scheme / order (at most 48 per group); each group is advanced by ONE
 * persistent kernel that takes its work from a device queue of tickets, one ticket
 * being a tile of elements (64 of the stage kernel's phase, 128 of the TVB
 * limiter's, each phase one finest substep) of one scenario, taken by one warp. The
 * kernel's CTAs have the warps per CTA of the group's first solver
 * (swe_set_tc_warps on the tensor-core tier). Tickets are ordered phase by phase,
 * round-robin over the scenarios, and a ticket waits (bounded in time) until every
 * tile of its scenario's earlier phases is complete, so uneven scenarios fill each
 * other's gaps. One batch step is one replay of a captured CUDA graph (per group:
 * counters cleared, the persistent kernel, the macro-counter update; the groups as
 * parallel branches). Results equal those of each solver stepped alone, bit for
 * bit (the same per-element operations; nothing crosses scenarios). */
typedef struct swe_batch swe_batch;

/* Bytes of caller-owned device workspace (the ticket tables and counters) for a
 * batch of these solvers that advances each by at most max_macro macro steps per
 * swe_batch_step. SWE_EINVAL for NULL arrays, n < 1, max_macro < 1 or a solver
 * without state and levels. */
int swe_batch_workspace_bytes(swe_solver* const* solvers, int32_t n, int32_t max_macro, size_t* bytes);

/* Create a batch of n distinct solvers, each with a valid level-synchronous state
 * and its own (non-default) stream, in caller-owned device memory dev_workspace
 * (bytes >= swe_batch_workspace_bytes, 256-byte aligned; owned by the caller, not
 * freed by the library). stream: the batch's own non-default stream. The solvers
 * stay usable on their own; work issued on their streams is ordered before and
 * after a batch step. The batch keeps pointers to the solvers: destroy it before
 * any of them. SWE_ENOMEM if the workspace is too small; SWE_EUNSUPPORTED for a
 * compensated solver (swe_params.compensated). */
int swe_batch_create(swe_solver* const* solvers, int32_t n, int32_t max_macro, void* dev_workspace,
                     size_t bytes, void* stream, swe_batch** out);

/* Advance solver i by n_macro_each[i] macro steps (0..max_macro; host array of n),
 * all in one batch step, and report per solver in status_each (host array of n):
 * SWE_OK, or SWE_ETIMEOUT when one of its bounded waits gave up (its remaining
 * work is skipped; the others carry on). A solver that timed out before any of its
 * work ran (for instance while held, swe_batch_hold) keeps its state and time; one
 * that timed out later has no valid state until swe_set_state or
 * swe_set_full_state. Returns SWE_OK, or SWE_ETIMEOUT if any solver timed out.
 * Synchronises the batch stream (the statuses are read back). SWE_EINVAL, with
 * nothing launched, for a count outside 0..max_macro, a solver without a valid
 * level-synchronous state, or a solver whose levels, element order, launch shape
 * or boundary faces changed since swe_batch_create (swe_set_levels,
 * swe_setup_levels, swe_regroup, swe_set_launch_config, swe_set_tc_warps, swe_set_farfield,
 * swe_set_open_faces, swe_set_full_state): create the batch again. */
int swe_batch_step(swe_batch* batch, const int32_t* n_macro_each, int32_t* status_each);

/* Bound (seconds, in (0, 3600); default 10) of every device wait of a batch step:
 * a scenario's wait for its earlier phases and for its release. */
int swe_batch_set_wait_limit(swe_batch* batch, double seconds);

/* hold = 1: withhold solver i's release at the following batch steps, so its first
 * phase waits until the wait limit and the step reports SWE_ETIMEOUT for it with
 * its state unchanged (a scenario kept out of the batch without rebuilding it);
 * hold = 0 releases it again. */
int swe_batch_hold(swe_batch* batch, int32_t i, int32_t hold);

/* Kernels this batch has launched (two per group and step). */
int swe_batch_launches(const swe_batch* batch, int64_t* launches);

/* Waits for the batch stream, then frees the host handle (not the workspace). */
void swe_batch_destroy(swe_batch* batch);

/* Boundary faces (those without a neighbour) are reflecting walls (the default;
 * Section 6's tests) or open to a far field whose ghost state is the constant
 * (h, hu, hv) over the continued bed (B+ = B-); at an open face the TVB limiter
 * takes that state over the element's mean bed as the ghost mean.
 * swe_set_farfield sets the state and opens every boundary face (enable = 1) or
 * closes them all (enable = 0); h >= 0 and all finite, SWE_EINVAL otherwise.
 * swe_set_open_faces then chooses the open faces one by one: open (K x 3, caller
 * order and face numbering, host) = 1 for open, 0 for a wall; entries of interior
 * faces are ignored. Both take effect at the next launch (a captured macro step
 * is captured again; batches must be created again). */
int swe_set_farfield(swe_solver* solver, int32_t enable, double h, double hu, double hv);
int swe_set_open_faces(swe_solver* solver, const uint8_t* open);

/* Launch shape of the stage and limiter kernels: at most ctas_per_sm CTAs per
 * SM in their grid-stride loops (0 = as many as fit). Used by the autotuner;
 * results do not depend on it. */
int swe_set_launch_config(swe_solver* solver, int32_t ctas_per_sm);

/* Warps per CTA of the tensor-core stage kernel and of the persistent batch kernel
 * (FP32 tensor-core tier; default 4, 2 at N = 5). Each warp owns its shared-memory tiles and the
 * CTA one copy of the operators, so more warps per CTA share that copy: at N = 5
 * (29 KB of tiles per warp) seven warps fit on an SM as one CTA where two CTAs of
 * four do not. warps in 1..8; SWE_EINVAL when that many warps' tiles do not fit on
 * an SM, SWE_EUNSUPPORTED on the other tiers. Used by the autotuner; results do not
 * depend on it. A batch takes the warps of the first solver of each group at
 * swe_batch_create. */
int swe_set_tc_warps(swe_solver* solver, int32_t warps);

/* Advance n finest substeps like swe_substep, timing every kernel launch with CUDA
 * events on the solver's stream (synchronises at the end). out[0..5]: total ms of
 * the stage kernels (R + commit + positivity), of the TVB kernels, of the other
 * kernels; number of stage launches; elements processed by the stage kernels; by
 * the TVB kernels. For measurement only: the events add a little launch overhead. */
int swe_profile_substeps(swe_solver* solver, int32_t n, double* out);

/* Number of CUDA kernel launches this solver has issued (direct or inside
 * replayed graphs), for launch accounting. */
int swe_kernel_launches(const swe_solver* solver, int64_t* launches);

/* Mass and minimum depth of nodal data the caller already holds on the device,
 * with no device allocation at all: the same reduction as swe_stats, but its
 * per-block partial sums go to a fixed 16 KiB scratch array compiled into this
 * library (it stays resident on every GPU that loads the library until the
 * process exits) instead of a solver workspace. It is meant for callers that
 * may not call cudaMalloc themselves: code whose device memory belongs to a
 * host application with its own fixed arena, and latency-sensitive monitoring
 * loops for which a cudaMalloc could synchronise the device. The paper has no
 * counterpart of this call; it is a deployment convenience.
 *   N         polynomial order, 1..5
 *   K         number of elements, with K*Np <= 2^31-1 (SWE_EINVAL beyond)
 *   dev_h     device, K x Np doubles: nodal depth h, element-major (row k holds
 *             element k's Np nodal values, contiguous, in the library's node order),
 *             elements in the same order as dev_area -- the layout swe_get_state
 *             returns, not the solver's internal device layout
 *   dev_area  device, K doubles: element areas
 *   dev_out   device, 2 doubles written: [0] sum_k area_k mean(h_k), [1] min nodal h;
 *             a NaN depth makes both NaN (the minimum keeps NaN; an infinite depth
 *             shows in the mass)
 *   stream    cudaStream_t (as void*), may be NULL
 * The first call on each device looks up the scratch array's device address
 * (cudaGetSymbolAddress, with that device current) and keeps it for the rest of
 * the process: the call assumes the context current then (a runtime-API caller's
 * primary context) and no cudaDeviceReset afterwards. Make that first call before
 * any stream capture. Every call shares the one scratch array per device, so
 * calls whose kernels overlap on the GPU (concurrent streams) race and give
 * wrong results; serialise them. Nothing in the scratch needs clearing: each
 * call overwrites what it reads. Returns SWE_EINVAL / SWE_ECUDA with a message
 * in swe_last_error(). */
int swe_mass_hmin_static(int32_t N, int32_t K, const double* dev_h, const double* dev_area,
                         double* dev_out, void* stream);

/* ---- measurement probe: the volume projection on the two tensor-core paths ----
 * Section 7.1 writes the volume term per field as N(Q) = Pr cF1 + Ps cF2 + P cS, a
 * product Flux[elements x cubature points] * Op^T. This probe times that product
 * for N = 4 shapes (16 padded nodes, 40 padded cubature points) on 128-element
 * tiles, with a flux generated in registers as a[e][q] = x[e] c[q] + y[e]:
 *   impl 0: warp-level mma.sync m16n8k8 TF32, flux in the A-fragment layout,
 *           accumulators in registers;
 *   impl 1: tcgen05.mma kind::tf32 (M = 128, N = 16, K = 8), flux stored to shared
 *           memory in the canonical K-major layout (double-buffered, two CTA
 *           barriers per tile), accumulator in TMEM, committed to an mbarrier, read
 *           back with tcgen05.ld;
 *   impl 2: the same product through four A buffers synchronised by mbarriers only
 *           (threads arrive on a buffer's "full" barrier, the issuing thread commits
 *           to its "empty" barrier), 83 KB of shared memory per CTA;
 *   impl 3, 4: impl 1 with N = 64 or 128 (the operator's 16 columns repeated), to
 *           time wider instructions on the same flux tiles; only the first 16
 *           columns are read back;
 *   impl 5: the flux stored from registers into TMEM (tcgen05.st, lane = element)
 *           and read by the MMA as its A operand: no shared-memory tile.
 * CTA i handles tiles [i * tiles_per_cta, (i + 1) * tiles_per_cta); row r of tile t
 * is element (t * 128 + r). Device arrays: dev_x, dev_y [nctas * tiles_per_cta * 128];
 * dev_c [40]; dev_b [40 * 16] row-major (b[q * 16 + n]); dev_d [nctas * 128 * 16]
 * receives, per CTA, D[r][n] = sum over its tiles t and q of tf32(a_t[r][q]) *
 * tf32(b[q][n]) (operands rounded to nearest, ties away). dev_status [nctas]
 * (impl >= 1): SWE_OK, or SWE_ETIMEOUT where a wait on the tensor core gave up after
 * one second (that CTA's row of dev_d is then not written). All arrays are the
 * caller's; launches on `stream`, returns without synchronising. Returns SWE_EINVAL
 * for a bad argument, SWE_ECUDA for a failed launch, with swe_last_error(). */
int swe_tc_projection_probe(int32_t impl, int32_t nctas, int32_t tiles_per_cta, const float* dev_x,
                            const float* dev_y, const float* dev_c, const float* dev_b, float* dev_d,
                            int32_t* dev_status, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SWE_GB300_H */
