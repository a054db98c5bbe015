"""Python front end of the C ABI: mesh and solver handles with torch-owned device memory.

PyTorch provides the device workspace (one uint8 tensor) and the CUDA stream; all
numerical work runs in the native library's kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _native as nat


def _prec_code(precision):
    if isinstance(precision, int):
        return precision
    p = str(precision).lower()
    if p in ("fp64", "f64", "double"):
        return nat.SWE_FP64
    if p in ("fp32", "f32", "float"):
        return nat.SWE_FP32
    if p in ("fp32tc", "fp32_tc", "tc", "bf16x3"):
        return nat.SWE_FP32_TC
    raise ValueError(f"unknown precision {precision!r}")


class Mesh:
    """Triangle mesh (host): connectivity and geometry built by the library."""

    def __init__(self, vx, vy, EToV):
        L = nat.lib()
        self.vx = np.ascontiguousarray(vx, np.float64)
        self.vy = np.ascontiguousarray(vy, np.float64)
        self.EToV = np.ascontiguousarray(EToV, np.int32)
        if self.vx.ndim != 1 or self.vx.shape != self.vy.shape:
            raise ValueError("vx and vy must be 1-D arrays of the same length")
        if self.EToV.ndim != 2 or self.EToV.shape[1] != 3:
            raise ValueError("EToV must have shape (K, 3)")
        h = C.c_void_p()
        nat.check(L.swe_mesh_create(nat.dptr(self.vx), nat.dptr(self.vy), self.vx.size,
                                    nat.iptr(self.EToV), self.EToV.shape[0], C.byref(h)),
                  "swe_mesh_create")
        self.handle = h
        self.K = int(self.EToV.shape[0])

    def connectivity(self):
        L = nat.lib()
        E = np.zeros((self.K, 3), np.int32)
        F = np.zeros((self.K, 3), np.int32)
        nat.check(L.swe_mesh_connectivity(self.handle, nat.iptr(E), nat.iptr(F)), "swe_mesh_connectivity")
        return E, F

    def node_coords(self, N):
        L = nat.lib()
        np_ = (N + 1) * (N + 2) // 2
        x = np.zeros((self.K, np_))
        y = np.zeros((self.K, np_))
        nat.check(L.swe_mesh_node_coords(self.handle, N, nat.dptr(x), nat.dptr(y)), "swe_mesh_node_coords")
        return x, y

    def levels(self, N, h, hu, hv, g, cfl, nlevels_max):
        """Level grouping (Section 4) the solver would make for this nodal state."""
        np_ = (N + 1) * (N + 2) // 2
        h, hu, hv = (np.ascontiguousarray(a, np.float64).reshape(self.K, np_) for a in (h, hu, hv))
        lev = np.zeros(self.K, np.int32)
        dtm = C.c_double()
        nat.check(nat.lib().swe_mesh_levels(self.handle, N, nat.dptr(h), nat.dptr(hu), nat.dptr(hv), g, cfl,
                                            nlevels_max, nat.iptr(lev), C.byref(dtm)), "swe_mesh_levels")
        return lev, dtm.value

    def centroids(self):
        return self.vx[self.EToV].mean(axis=1), self.vy[self.EToV].mean(axis=1)

    def close(self):
        if getattr(self, "handle", None):
            nat.lib().swe_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ref_sizes(N):
    L = nat.lib()
    a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
    nat.check(L.swe_ref_sizes(N, C.byref(a), C.byref(b), C.byref(c)), "swe_ref_sizes")
    return a.value, b.value, c.value


def ref_nodes(N):
    np_ = ref_sizes(N)[0]
    r = np.zeros(np_)
    s = np.zeros(np_)
    nat.check(nat.lib().swe_ref_nodes(N, nat.dptr(r), nat.dptr(s)), "swe_ref_nodes")
    return r, s


_OP_SHAPES = {0: ("Ncub", "Np"), 1: ("Ncub", "Np"), 2: ("Ncub", "Np"), 3: ("Np", "Ncub"),
              4: ("Np", "Ncub"), 5: ("Np", "Ncub"), 6: ("Np", "3Ng"), 7: ("Ng", "Nfp"),
              8: ("Np",), 9: ("3", "Np"), 10: ("Ncub",), 11: ("Ng",)}


def ref_operator(N, which):
    Np, Ncub, Ng = ref_sizes(N)
    dims = {"Np": Np, "Ncub": Ncub, "Ng": Ng, "3Ng": 3 * Ng, "Nfp": N + 1, "3": 3}
    shape = tuple(dims[d] for d in _OP_SHAPES[which])
    out = np.zeros(int(np.prod(shape)))
    nat.check(nat.lib().swe_ref_operator(N, which, nat.dptr(out), out.size), "swe_ref_operator")
    return out.reshape(shape)


class Solver:
    """One shallow-water problem resident on the GPU (state, history, geometry)."""

    def __init__(self, mesh: Mesh, N: int, g: float = 9.81, h0: float = 1e-5, cfl: float = 0.5,
                 nlevels_max: int = 1, precision="fp32", limiter_mask: int = 0, tvb_M: float = 0.0,
                 tvb_nu: float = 1.5, dry_mode: int = 0, eps: float = 0.0, device=None, stream=None,
                 scheme: str = "cubature", compensated: bool = False):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        L = nat.lib()
        self.mesh = mesh
        self.N = N
        self.K = mesh.K
        self.Np = (N + 1) * (N + 2) // 2
        self.prm = nat.swe_params(g, h0, eps, tvb_M, tvb_nu, cfl, N, nlevels_max,
                                  _prec_code(precision), limiter_mask, dry_mode,
                                  {"cubature": nat.SWE_SCHEME_CUBATURE,
                                   "collocation": nat.SWE_SCHEME_COLLOCATION,
                                   "cubature_2n": nat.SWE_SCHEME_CUBATURE_2N}[scheme],
                                  1 if compensated else 0)
        self.precision = self.prm.precision
        nbytes = C.c_size_t()
        nat.check(L.swe_workspace_bytes(mesh.handle, C.byref(self.prm), C.byref(nbytes)),
                  "swe_workspace_bytes")
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self._own_stream = None
        with torch.cuda.device(self.device):
            # a stream of its own (not one from torch's pool, which hands the same
            # stream to several users): the macro step is captured into a CUDA graph
            # on it, and work another thread enqueues there meanwhile would void that
            self.stream = own_stream(self) if stream is None else stream
            self.workspace = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8, device=self.device)
            self.stream.wait_stream(torch.cuda.current_stream(self.device))
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            nat.check(L.swe_solver_create(mesh.handle, C.byref(self.prm), C.c_void_p(self._ws_ptr),
                                          nbytes.value, C.c_void_p(self.stream.cuda_stream), C.byref(h)),
                      "swe_solver_create")
        self.handle = h
        self.workspace_bytes = int(nbytes.value)

    # -- inputs -----------------------------------------------------------
    def set_bathymetry(self, B):
        B = np.ascontiguousarray(B, np.float64).reshape(self.K, self.Np)
        nat.check(nat.lib().swe_set_bathymetry(self.handle, nat.dptr(B)), "swe_set_bathymetry")

    def set_state(self, h, hu, hv):
        h, hu, hv = (np.ascontiguousarray(a, np.float64).reshape(self.K, self.Np) for a in (h, hu, hv))
        nat.check(nat.lib().swe_set_state(self.handle, nat.dptr(h), nat.dptr(hu), nat.dptr(hv)),
                  "swe_set_state")

    def setup_levels(self):
        lev = np.zeros(self.K, np.int32)
        dtm = C.c_double()
        nat.check(nat.lib().swe_setup_levels(self.handle, nat.iptr(lev), C.byref(dtm)), "swe_setup_levels")
        self.level = lev
        return lev, dtm.value

    def set_levels(self, level, dt_min):
        lev = np.ascontiguousarray(level, np.int32).reshape(self.K)
        nat.check(nat.lib().swe_set_levels(self.handle, nat.iptr(lev), float(dt_min)), "swe_set_levels")
        self.level = lev.copy()

    def set_farfield(self, state=None, open_faces=None):
        """Boundary faces: reflecting walls (state=None) or open to the far field
        (h, hu, hv); open_faces (K x 3 bool, caller order) opens only those faces."""
        if state is None:
            nat.check(nat.lib().swe_set_farfield(self.handle, 0, 0.0, 0.0, 0.0), "swe_set_farfield")
            return
        h, hu, hv = (float(v) for v in state)
        nat.check(nat.lib().swe_set_farfield(self.handle, 1, h, hu, hv), "swe_set_farfield")
        if open_faces is not None:
            o = np.ascontiguousarray(open_faces, np.uint8).reshape(self.K, 3)
            nat.check(nat.lib().swe_set_open_faces(self.handle, C.c_void_p(o.ctypes.data)), "swe_set_open_faces")

    def regroup(self, level=None):
        """Regroup into new levels without restarting (history kept); level=None
        applies the CFL rule. Returns (levels in caller order, CFL margin)."""
        out = np.zeros(self.K, np.int32)
        margin = C.c_double()
        lp = None
        if level is not None:
            lv = np.ascontiguousarray(level, np.int32).reshape(self.K)
            lp = nat.iptr(lv)
        nat.check(nat.lib().swe_regroup(self.handle, lp, nat.iptr(out), C.byref(margin)), "swe_regroup")
        self.level = out
        return out, margin.value

    # -- the hot path -----------------------------------------------------
    def rhs(self):
        """R(Q) as a device tensor of shape (3, K, Np) in the solver's precision."""
        import torch
        dt = torch.float64 if self.precision == nat.SWE_FP64 else torch.float32
        out = torch.empty((3, self.K, self.Np), dtype=dt, device=self.device)
        cur = torch.cuda.current_stream(self.device)
        self.stream.wait_stream(cur)
        nat.check(nat.lib().swe_rhs(self.handle, C.c_void_p(out.data_ptr())), "swe_rhs")
        # the caller's stream waits for the solver's: out stays the caller stream's
        # tensor (no record_stream, which would tie it to a stream that close() ends)
        cur.wait_stream(self.stream)
        return out

    def rhs_variant(self, variant, scratch=None):
        """R(Q) by a kernel-structure ablation (nat.SWE_RHS_*), same layout as rhs().
        scratch: a device uint8 tensor of at least rhs_scratch_bytes(variant) bytes
        (allocated here when None)."""
        import torch
        need = C.c_size_t()
        nat.check(nat.lib().swe_rhs_scratch_bytes(self.handle, int(variant), C.byref(need)),
                  "swe_rhs_scratch_bytes")
        if need.value and scratch is None:
            scratch = torch.empty(need.value, dtype=torch.uint8, device=self.device)
        elif need.value and (not scratch.is_cuda or scratch.device != torch.device(self.device)
                             or not scratch.is_contiguous()):
            raise ValueError("scratch must be a contiguous tensor on the solver's device")
        dt = torch.float64 if self.precision == nat.SWE_FP64 else torch.float32
        out = torch.empty((3, self.K, self.Np), dtype=dt, device=self.device)
        cur = torch.cuda.current_stream(self.device)
        self.stream.wait_stream(cur)
        sp = C.c_void_p(scratch.data_ptr()) if need.value else None
        sb = scratch.numel() * scratch.element_size() if need.value else 0
        nat.check(nat.lib().swe_rhs_variant(self.handle, int(variant), C.c_void_p(out.data_ptr()), sp, sb),
                  "swe_rhs_variant")
        cur.wait_stream(self.stream)
        return out

    def rhs_scratch_bytes(self, variant):
        need = C.c_size_t()
        nat.check(nat.lib().swe_rhs_scratch_bytes(self.handle, int(variant), C.byref(need)),
                  "swe_rhs_scratch_bytes")
        return need.value

    def substep(self, n=1):
        nat.check(nat.lib().swe_substep(self.handle, int(n)), "swe_substep")

    def step(self, n_macro=1):
        nat.check(nat.lib().swe_step(self.handle, int(n_macro)), "swe_step")

    def limit(self, mask):
        nat.check(nat.lib().swe_limit(self.handle, int(mask)), "swe_limit")

    # -- outputs ------------------------------------------------------------
    def get_state(self, out=None):
        """(h, hu, hv, t); out = three preallocated (K, Np) float64 C-contiguous arrays
        (for example views of page-locked memory) to fill instead of new ones."""
        if out is None:
            h = np.zeros((self.K, self.Np))
            hu = np.zeros_like(h)
            hv = np.zeros_like(h)
        else:
            h, hu, hv = out
            for a in out:
                if a.dtype != np.float64 or a.shape != (self.K, self.Np) or not a.flags.c_contiguous:
                    raise ValueError("out arrays must be C-contiguous float64 of shape (K, Np)")
        t = C.c_double()
        nat.check(nat.lib().swe_get_state(self.handle, nat.dptr(h), nat.dptr(hu), nat.dptr(hv), C.byref(t)),
                  "swe_get_state")
        return h, hu, hv, t.value

    def stats(self):
        m, inj, hmin = C.c_double(), C.c_double(), C.c_double()
        dofs = C.c_int64()
        rc = nat.lib().swe_stats(self.handle, C.byref(m), C.byref(inj), C.byref(hmin), C.byref(dofs))
        out = {"mass": m.value, "injected_mass": inj.value, "hmin": hmin.value, "dof_updates": dofs.value,
               "nonfinite": rc == nat.SWE_ENAN}
        if rc not in (nat.SWE_OK, nat.SWE_ENAN):
            nat.check(rc, "swe_stats")
        return out

    def level_info(self):
        Lc = C.c_int32()
        counts = np.zeros(8, np.int32)
        dtm = C.c_double()
        nat.check(nat.lib().swe_level_info(self.handle, C.byref(Lc), nat.iptr(counts), C.byref(dtm)),
                  "swe_level_info")
        return Lc.value, counts[:Lc.value].copy(), dtm.value

    def kernel_launches(self):
        n = C.c_int64()
        nat.check(nat.lib().swe_kernel_launches(self.handle, C.byref(n)), "swe_kernel_launches")
        return n.value

    def set_launch_config(self, shape):
        """A launch shape: CTAs per SM of the grid-stride kernels (an int, 0 = as
        many as fit), or a dict {"ctas_per_sm": c, "tc_warps": w} as the autotuner
        returns it (tc_warps: warps per CTA of the tensor-core kernels)."""
        if isinstance(shape, dict):
            nat.check(nat.lib().swe_set_launch_config(self.handle, int(shape.get("ctas_per_sm", 0))),
                      "swe_set_launch_config")
            if shape.get("tc_warps") is not None:
                self.set_tc_warps(shape["tc_warps"])
        else:
            nat.check(nat.lib().swe_set_launch_config(self.handle, int(shape)), "swe_set_launch_config")

    def set_tc_warps(self, warps):
        nat.check(nat.lib().swe_set_tc_warps(self.handle, int(warps)), "swe_set_tc_warps")

    def profile_substeps(self, n):
        """Run n substeps with CUDA events around every kernel; per-kernel totals."""
        out = np.zeros(6)
        nat.check(nat.lib().swe_profile_substeps(self.handle, int(n), nat.dptr(out)), "swe_profile_substeps")
        return {"stage_ms": out[0], "tvb_ms": out[1], "other_ms": out[2], "stage_launches": int(out[3]),
                "stage_elements": int(out[4]), "tvb_elements": int(out[5])}

    def full_state(self):
        nb = C.c_size_t()
        nat.check(nat.lib().swe_full_state_bytes(self.handle, C.byref(nb)), "swe_full_state_bytes")
        buf = np.zeros(nb.value, np.uint8)
        nat.check(nat.lib().swe_get_full_state(self.handle, buf.ctypes.data_as(C.c_void_p), nb.value),
                  "swe_get_full_state")
        return buf

    def load_full_state(self, buf):
        buf = np.ascontiguousarray(buf, np.uint8)
        nat.check(nat.lib().swe_set_full_state(self.handle, buf.ctypes.data_as(C.c_void_p), buf.size),
                  "swe_set_full_state")

    def close(self):
        if getattr(self, "handle", None):
            nat.lib().swe_solver_destroy(self.handle)
            self.handle = None
            self.workspace = None
        release_stream(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def own_stream(owner):
    """A dedicated non-blocking stream created by the library, wrapped for torch;
    owner._own_stream keeps the handle for release_stream."""
    import torch
    h = C.c_void_p()
    nat.check(nat.lib().swe_stream_create(C.byref(h)), "swe_stream_create")
    owner._own_stream = h.value
    return torch.cuda.ExternalStream(h.value, device=torch.cuda.current_device())


def release_stream(owner):
    h = getattr(owner, "_own_stream", None)
    if h:
        owner._own_stream = None
        nat.lib().swe_stream_destroy(C.c_void_p(h))


def scenario_inputs(scn, mesh: Mesh):
    """Evaluate a workloads.scenarios.Scenario at this library's nodes."""
    x, y = mesh.node_coords(scn.N)
    cx, cy = mesh.centroids()
    cx = np.repeat(cx[:, None], x.shape[1], axis=1)
    cy = np.repeat(cy[:, None], x.shape[1], axis=1)
    B = np.asarray(scn.bathymetry(x, y, cx, cy), np.float64)
    h, hu, hv = scn.init(x, y, cx, cy, B)
    return B, np.asarray(h, np.float64), np.asarray(hu, np.float64), np.asarray(hv, np.float64)


def solver_from_scenario(scn, precision="fp32", levels=None, dt_min=None, mesh_arrays=None, **kw):
    """Mesh + solver + inputs for a scenario; levels from the CFL rule unless given."""
    vx, vy, E = scn.build_mesh() if mesh_arrays is None else mesh_arrays
    mesh = Mesh(vx, vy, E)
    s = Solver(mesh, scn.N, g=scn.g, h0=scn.h0, cfl=scn.cfl, nlevels_max=max(scn.nlevels, 1),
               precision=precision, limiter_mask=scn.limiter_mask, tvb_M=scn.tvb_M, tvb_nu=scn.tvb_nu,
               dry_mode=scn.dry_mode, **kw)
    B, h, hu, hv = scenario_inputs(scn, mesh)
    s.set_bathymetry(B)
    s.set_state(h, hu, hv)
    if levels is None:
        s.setup_levels()
    else:
        s.set_levels(levels, dt_min)
    return s
