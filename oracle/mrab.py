"""Multirate Adams-Bashforth time stepping with limiting (Algorithms 1 and 2), oracle.

Levels (Section 4): level l holds the elements with 2^{l-1} dt_min <= dt_k < 2^l dt_min
and is stepped with dt_l = 2^{l-1} dt_min by the third-order Adams-Bashforth rule
Q <- Q + dt_l (alpha_1 R^(0) + alpha_2 R^(-1) + alpha_3 R^(-2)),
alpha = (23, -16, 5)/12 (Algorithm 1), followed by the limiters
Q <- Lambda Pi M Pi { ... } (Algorithm 2).

Reading of the level coupling (the algorithms do not say how a level sees a
neighbour of another level between that neighbour's steps):
* the schedule runs on the finest substeps t_k = k dt_min; level l is active at
  t_k when k is a multiple of 2^{l-1}. Active elements evaluate R at t_k, commit to
  t_k + dt_l, then are limited (positivity, then TVB).
* a neighbour whose level is not active at t_k (always a coarser one) is seen at
  t_k through its Adams-Bashforth polynomial: Q_start + dt_nb sum_s beta_s(theta)
  R_nb^(s), theta = (t_k - t_start)/dt_nb, where beta_s integrates the Lagrange
  interpolant of the R history over [0, theta] (theta = 1 gives alpha).
* start-up per level: first step Euler (AB1), second AB2, then AB3; the same
  depth is used for the reconstruction.
* the TVB limiter reads each element's latest committed means and dry flags.
* reconstructed neighbour values are not limited.
* one "macro step" is 2^{L-1} finest substeps; all levels then sit at the same time.
"""
from __future__ import annotations

import math

import numpy as np

from .limiters import pp_limit, tvb_limit, tvb_geometry
from .swe import SWEModel


def cfl_regroup_levels(dt, dt_min: float, level, k: int, nlevels: int):
    """The regroup rule of MRAB.cfl_levels for per-element CFL steps dt."""
    dt = np.asarray(dt, np.float64)
    lev = np.ones(dt.shape, np.int64)
    for i, d in enumerate(dt):
        _, e = math.frexp(d / dt_min)          # d / dt_min = m 2^e, m in [0.5, 1)
        lev[i] = min(max(e, 1), nlevels)
    lev = np.minimum(lev, np.asarray(level, np.int64) + 1)
    v2 = (k & -k).bit_length() - 1 if k > 0 else 62
    lev = np.minimum(lev, 1 + v2)
    margin = float((dt / (dt_min * 2.0 ** (lev - 1))).min())
    return lev, margin


def ab_coefficients(depth: int):
    """Adams-Bashforth weights for R^(0), R^(-1), R^(-2) (equal steps)."""
    if depth == 1:
        return (1.0,)
    if depth == 2:
        return (1.5, -0.5)
    return (23.0 / 12.0, -16.0 / 12.0, 5.0 / 12.0)


def ab_partial_coefficients(depth: int, theta: float):
    """Integral over [0, theta] of the Lagrange interpolant through R at tau = 0, -1, -2."""
    t = float(theta)
    if depth == 1:
        return (t,)
    if depth == 2:
        return (t + t * t / 2.0, -t * t / 2.0)
    return (t ** 3 / 6.0 + 3.0 * t * t / 4.0 + t, -(t ** 3 / 3.0 + t * t), t ** 3 / 6.0 + t * t / 4.0)


class MRAB:
    """State + history of the multirate integrator (all elements)."""

    def __init__(self, model: SWEModel, h, hu, hv, levels, dt_min: float,
                 limiter_mask: int = 0, tvb_M: float = 0.0, tvb_nu: float = 1.5,
                 dry_mode: int = 0):
        self.model = model
        self.level = np.asarray(levels, np.int64)
        self.L = int(self.level.max())
        self.dt_min = float(dt_min)
        self.dtl = self.dt_min * 2.0 ** (self.level - 1)
        self.limiter_mask = limiter_mask
        self.tvb_M = tvb_M
        self.tvb_nu = tvb_nu
        self.dry_mode = dry_mode
        K = h.shape[0]
        self.dry = np.zeros(K, bool)
        self.injected = 0.0
        self.geom = tvb_geometry(model.mesh) if (limiter_mask & 2) else None
        q = [np.array(h, np.float64), np.array(hu, np.float64), np.array(hv, np.float64)]
        q = self._limit(q, np.ones(K, bool))            # Algorithm 2, first line
        self.q_end = np.stack(q)                         # latest committed state
        self.q_start = self.q_end.copy()                 # state at the start of the current step
        self.hist = np.zeros((3,) + self.q_end.shape)    # ring of R, slot = activation % 3
        self.count = np.zeros(K, np.int64)               # completed activations per element
        self.k = 0                                       # global finest-substep index
        self.dof_updates = 0

    def _limit(self, q, active):
        m = self.model
        if self.limiter_mask & 1:
            h, hu, hv, dry, inj = pp_limit(m, q[0], q[1], q[2], active=active,
                                           dry_mode=self.dry_mode)
            self.injected += inj
            self.dry = np.where(active, dry, self.dry)
            q = [h, hu, hv]
        if self.limiter_mask & 2:
            h, hu, hv, _ = tvb_limit(m, q[0], q[1], q[2], self.dry, active=active,
                                     M=self.tvb_M, nu=self.tvb_nu, geom=self.geom)
            q = [h, hu, hv]
        return q

    @property
    def time(self):
        return self.k * self.dt_min

    def state_at_tk(self):
        """Every element's state at t_k (reconstructed where its level is between steps)."""
        k = self.k
        qtk = self.q_start.copy()
        for lev in range(1, self.L + 1):
            period = 2 ** (lev - 1)
            ph = k % period
            if ph == 0:
                continue
            sel = (self.level == lev)
            if not np.any(sel):
                continue
            a_last = self.count[sel] - 1                 # index of the latest activation
            theta = ph / period
            acc = np.zeros_like(qtk[:, sel])
            for depth in (1, 2, 3):
                dsel = np.minimum(a_last + 1, 3) == depth
                if not np.any(dsel):
                    continue
                beta = ab_partial_coefficients(depth, theta)
                for s, b in enumerate(beta):
                    slot = (a_last[dsel] - s) % 3
                    idx = np.nonzero(sel)[0][dsel]
                    acc[:, dsel] += b * self.hist[slot, :, idx].transpose(1, 0, 2)
            qtk[:, sel] = self.q_start[:, sel] + self.dtl[sel][None, :, None] * acc
        return qtk

    def substep(self):
        k = self.k
        active = (k % (2 ** (self.level - 1))) == 0
        self.q_start[:, active] = self.q_end[:, active]
        qtk = self.state_at_tk()
        R = self.model.rhs(qtk[0], qtk[1], qtk[2], t=self.time)
        a = self.count[active]
        idx = np.nonzero(active)[0]
        slot = a % 3
        self.hist[slot, :, idx] = R[:, idx].transpose(1, 0, 2)
        acc = np.zeros_like(self.q_start[:, active])
        depth = np.minimum(a + 1, 3)
        for d in (1, 2, 3):
            dsel = depth == d
            if not np.any(dsel):
                continue
            for s, c in enumerate(ab_coefficients(d)):
                sl = (a[dsel] - s) % 3
                acc[:, dsel] += c * self.hist[sl, :, idx[dsel]].transpose(1, 0, 2)
        qn = self.q_start[:, active] + self.dtl[active][None, :, None] * acc
        self.q_end[:, active] = qn
        self.count[active] += 1
        q = self._limit([self.q_end[0], self.q_end[1], self.q_end[2]], active)
        self.q_end = np.stack(q)
        self.dof_updates += int(active.sum()) * self.q_end.shape[2] * 3
        self.k += 1

    def regroup(self, levels):
        """Regroup the elements into new levels at a level-synchronous time t_k
        (Section 4: "elements can be regrouped after every few time steps"), keeping
        dt_min, the state and the Adams-Bashforth history.

        Reading: an element moved from level l to l' needs its R history at
        t_k - dt_l' and t_k - 2 dt_l'. It holds R at t_k - s dt_l, s = 1, 2, 3 (its
        last three activations); the quadratic through those three values is
        evaluated at the new times (tau' = -r, -2r, -3r in units of dt_l,
        r = dt_l' / dt_l). The activation count becomes k / 2^{l'-1}, so the ring
        slot of activation a stays a mod 3. Requires k to be a multiple of
        2^{max(l')-1} and of 2^{L-1}, and k >= 3 * 2^{L-1} (three activations
        of every level)."""
        lev = np.asarray(levels, np.int64)
        k = self.k
        if k % (2 ** (self.L - 1)) != 0:
            raise ValueError("regroup needs a level-synchronous state")
        if k < 3 * 2 ** (self.L - 1):
            raise ValueError("regroup needs three activations of every level")
        if lev.min() < 1 or k % (2 ** (int(lev.max()) - 1)) != 0:
            raise ValueError("new levels must divide the substep count")
        moved = np.nonzero(lev != self.level)[0]
        for e in moved:
            l0, l1 = int(self.level[e]), int(lev[e])
            a0, a1 = k >> (l0 - 1), k >> (l1 - 1)
            H = [self.hist[(a0 - s) % 3, :, e].copy() for s in (1, 2, 3)]   # tau = -1, -2, -3
            r = 2.0 ** (l1 - l0)
            for s in (1, 2, 3):
                x = -s * r
                w = ((x + 2) * (x + 3) / 2.0, -(x + 1) * (x + 3), (x + 1) * (x + 2) / 2.0)
                self.hist[(a1 - s) % 3, :, e] = w[0] * H[0] + w[1] * H[1] + w[2] * H[2]
        self.level = lev
        self.L = int(lev.max())
        self.dtl = self.dt_min * 2.0 ** (lev - 1)
        self.count = k >> (lev - 1)
        self.q_start = self.q_end.copy()

    def cfl_levels(self, cfl: float, nlevels: int):
        """Levels for a regroup by the CFL rule (Eq. cfl) with dt_min kept: the
        largest l with 2^{l-1} dt_min <= dt_k, in 1..nlevels; at most one level
        coarser than now (the history is extrapolated over at most one old step)
        and at most 1 + (the power of 2 in k). Returns (levels, margin) with
        margin = min_k dt_k / dt_l'(k) (< 1: some element's CFL step fell below
        dt_min and a restart with a smaller dt_min is needed)."""
        from .mesh import element_dt
        m = self.model
        q = self.q_end
        dt = element_dt(m.mesh, m.ref.N, q[0], q[1], q[2], m.g, cfl)
        return cfl_regroup_levels(dt, self.dt_min, self.level, self.k, nlevels)

    def macro_step(self, n: int = 1):
        for _ in range(n * 2 ** (self.L - 1)):
            self.substep()
