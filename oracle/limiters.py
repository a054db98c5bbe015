"""Positivity-preserving limiter (Algorithm 3) and characteristic TVB limiter with the
positivity modification (Section 5.3, Eq. modified_TVB), oracle version (FP64).

Readings where the paper is silent or garbled:
* eps = h0 in Algorithm 3; the P1 mean equals the P^N mean, so the garbled
  h-bar^{n,1} vs h-bar^n are the same number; theta = min(1, (hbar - h0)/(hbar - h1min))
  with h1min over the three vertices of the P1 projection and theta = 1 when the
  denominator is not positive; the same theta scales h, hu and hv.
* the wet/dry test of Algorithm 3 uses h_dry = (1 + 1e-2) h0 (an element reset to
  h0 that receives no water stays classified dry under rounding); that
  classification is the element's "dry" flag for the TVB skip.
* dry_mode 0: h = h0, hu = hv = 0 (literal; injected mass is tallied);
  dry_mode 1: h = hbar (mean preserving).
* TVB (Cockburn & Shu 1998, RKDG V, triangles) acts on the P1 part of (eta, hu, hv)
  with eta = h + B: edge-midpoint deltas against the combination of neighbour means
  alpha_i (u_Ki - u_0) + beta_i (u_Kj - u_0) (alpha, beta >= 0), characteristic
  variables of the flux Jacobian at the element mean in the direction m_i - b_0,
  TVB minmod with threshold M |m_i - b_0|^2 and nu = 1.5 (plus a round-off floor
  of 1e-6 (hbar + |m-bar|/c) in depth units, times c for the shear component, so
  that deltas at round-off level never count as limited), positive/negative
  redistribution so the deltas sum to zero. The P^N solution is kept when no
  characteristic component was changed. A far-field face uses the far-field state
  (over the own mean bed) as its ghost mean. A wall face uses a ghost neighbour whose
  barycentre is b_0 reflected across the face and whose mean has the normal
  momentum reversed.
* the limited depth is P1: h = (limited eta) - Pi1 B, then the positivity
  modification of Eq. modified_TVB rescales the h deltas so every vertex value is
  >= h0 (applied only when some vertex is below h0, theta clipped to [0, 1]).
* elements classified dry, and their immediate neighbours, are skipped
  (Section 5.3, last paragraph).
"""
from __future__ import annotations

import numpy as np

from .swe import SWEModel

DRY_MARGIN = 1e-2
TVB_FLOOR = 1e-6


def pp_limit(model: SWEModel, h, hu, hv, active=None, dry_mode: int = 0, eps=None):
    """Algorithm 3 on every active element. Returns (h, hu, hv, dry_flag, injected_mass)."""
    ref = model.ref
    h0 = model.h0
    eps = h0 if eps is None else eps
    h, hu, hv = h.copy(), hu.copy(), hv.copy()
    K = h.shape[0]
    act = np.ones(K, bool) if active is None else np.asarray(active, bool)
    dry = np.zeros(K, bool)
    hmin = h.min(axis=1)
    trig = act & (hmin <= eps)
    idx = np.nonzero(trig)[0]
    injected = 0.0
    if idx.size == 0:
        return h, hu, hv, dry, injected
    q = [h[idx], hu[idx], hv[idx]]
    q1 = [x @ ref.Pi1.T for x in q]
    qbar = [x @ ref.mean_w for x in q]
    hbar = qbar[0]
    isdry = hbar < (1.0 + DRY_MARGIN) * h0
    # dry elements
    d = idx[isdry]
    if d.size:
        if dry_mode == 0:
            h[d] = h0
        else:
            h[d] = hbar[isdry][:, None]
        hu[d] = 0.0
        hv[d] = 0.0
        newmean = np.full(d.size, h0) if dry_mode == 0 else hbar[isdry]
        injected = float(np.sum(model.mesh.area[d] * (newmean - hbar[isdry])))
        dry[d] = True
    # wet (or partially wet) elements: theta-rescale of the P1 projection
    w = ~isdry
    if np.any(w):
        wi = idx[w]
        h1 = q1[0][w]
        h1min = h1[:, ref.vertex_nodes].min(axis=1)
        hb = hbar[w]
        den = hb - h1min
        theta = np.where(den > 0.0, np.minimum(1.0, (hb - h0) / np.where(den > 0.0, den, 1.0)), 1.0)
        for arr, x1, xb in ((h, q1[0], qbar[0]), (hu, q1[1], qbar[1]), (hv, q1[2], qbar[2])):
            arr[wi] = theta[:, None] * (x1[w] - xb[w][:, None]) + xb[w][:, None]
    return h, hu, hv, dry, injected


# ----------------------------------------------------------------------------
# TVB


def _tvb_minmod(a, b, thr):
    """TVB-modified minmod m~(a, b): a if |a| <= thr, else minmod(a, b)."""
    same = (np.sign(a) == np.sign(b)) & (a != 0.0) & (b != 0.0)
    mm = np.where(same, np.sign(a) * np.minimum(np.abs(a), np.abs(b)), 0.0)
    return np.where(np.abs(a) <= thr, a, mm)


def tvb_geometry(mesh):
    """Per element and edge: midpoint-centroid vector, and (alpha, beta, j) such that
    m_i - b0 = alpha (b_i - b0) + beta (b_j - b0) with alpha, beta >= 0 (when possible;
    otherwise the j with the larger min(alpha, beta))."""
    K = mesh.K
    b0 = np.stack([mesh.cx, mesh.cy], axis=1)
    mid = np.zeros((K, 3, 2))
    bn = np.zeros((K, 3, 2))
    for f, (a, b) in enumerate(((0, 1), (1, 2), (2, 0))):
        mid[:, f, 0] = 0.5 * (mesh.xv[:, a] + mesh.xv[:, b])
        mid[:, f, 1] = 0.5 * (mesh.yv[:, a] + mesh.yv[:, b])
        nb = mesh.EToE[:, f]
        inner = nb >= 0
        bn[inner, f, 0] = mesh.cx[nb[inner]]
        bn[inner, f, 1] = mesh.cy[nb[inner]]
        # ghost barycentre: reflect b0 across the face line
        nx, ny = mesh.nx[:, f], mesh.ny[:, f]
        dist = (mid[:, f, 0] - b0[:, 0]) * nx + (mid[:, f, 1] - b0[:, 1]) * ny
        gx = b0[:, 0] + 2.0 * dist * nx
        gy = b0[:, 1] + 2.0 * dist * ny
        bn[~inner, f, 0] = gx[~inner]
        bn[~inner, f, 1] = gy[~inner]
    dm = mid - b0[:, None, :]
    db = bn - b0[:, None, :]
    alpha = np.zeros((K, 3))
    beta = np.zeros((K, 3))
    jsel = np.zeros((K, 3), np.int64)
    for i in range(3):
        best = None
        for jj in ((i + 1) % 3, (i + 2) % 3):
            a11, a21 = db[:, i, 0], db[:, i, 1]
            a12, a22 = db[:, jj, 0], db[:, jj, 1]
            det = a11 * a22 - a12 * a21
            al = (dm[:, i, 0] * a22 - a12 * dm[:, i, 1]) / det
            be = (a11 * dm[:, i, 1] - a21 * dm[:, i, 0]) / det
            score = np.minimum(al, be)
            if best is None:
                best = (score, al, be, np.full(K, jj))
            else:
                take = score > best[0]
                best = (np.where(take, score, best[0]), np.where(take, al, best[1]),
                        np.where(take, be, best[2]), np.where(take, jj, best[3]))
        alpha[:, i], beta[:, i], jsel[:, i] = best[1], best[2], best[3]
    return dm, alpha, beta, jsel


def swe_eigenvectors(h, u, v, nx, ny, g):
    """Right eigenvectors (columns) of the x-y SWE flux Jacobian in direction n."""
    c = np.sqrt(g * h)
    R = np.zeros(h.shape + (3, 3))
    R[..., 0, 0] = 1.0
    R[..., 1, 0] = u - c * nx
    R[..., 2, 0] = v - c * ny
    R[..., 0, 1] = 0.0
    R[..., 1, 1] = -ny
    R[..., 2, 1] = nx
    R[..., 0, 2] = 1.0
    R[..., 1, 2] = u + c * nx
    R[..., 2, 2] = v + c * ny
    return R


def positivity_modify(hb, dh, h0):
    """Positivity modification of the limited depth deltas (Section 5.3,
    Eq. modified_TVB). hb: (n,) mean depths; dh: (n, 3) depth deltas at the three
    edge midpoints. The vertex values of the P1 depth are hb + S_a with
    S_a = d_a + d_{a-1} - d_{a+1} (the vertex opposite midpoint a+1). Where the lowest
    of them lies below h0, the deltas are pulled toward their average dbar by
    theta = clip((hb + dbar - h0) / (dbar - min_a S_a), 0, 1), which puts that vertex
    exactly at h0 and keeps the average delta (so the element mean). Returns the
    modified deltas."""
    S = np.stack([dh[:, 0] + dh[:, 2] - dh[:, 1], dh[:, 1] + dh[:, 0] - dh[:, 2],
                  dh[:, 2] + dh[:, 1] - dh[:, 0]], axis=1)
    dbar = dh.mean(axis=1)
    need = (hb + S.min(axis=1)) < h0
    den = dbar - S.min(axis=1)
    th = np.where(need & (den > 0), np.clip((hb + dbar - h0) / np.where(den > 0, den, 1.0), 0.0, 1.0), 1.0)
    return dbar[:, None] + th[:, None] * (dh - dbar[:, None])


def tvb_limit(model: SWEModel, h, hu, hv, dry, active=None, M: float = 0.0, nu: float = 1.5,
              geom=None):
    """Characteristic TVB limiter + positivity modification on every active, wet
    element whose neighbours are all wet. Returns (h, hu, hv, limited_mask)."""
    ref, mesh, g, h0 = model.ref, model.mesh, model.g, model.h0
    K = h.shape[0]
    act = np.ones(K, bool) if active is None else np.asarray(active, bool)
    dm, alpha, beta, jsel = tvb_geometry(mesh) if geom is None else geom
    nbdry = np.zeros(K, bool)
    for f in range(3):
        nb = mesh.EToE[:, f]
        inner = nb >= 0
        nbdry[inner] |= dry[nb[inner]]
    sel = act & ~dry & ~nbdry
    h, hu, hv = h.copy(), hu.copy(), hv.copy()
    limited = np.zeros(K, bool)
    idx = np.nonzero(sel)[0]
    if idx.size == 0:
        return h, hu, hv, limited
    B = model.B
    eta = h + B
    # element means of (eta, hu, hv) for every element (neighbour lookups)
    mw = ref.mean_w
    ubar = np.stack([eta @ mw, hu @ mw, hv @ mw], axis=1)         # (K, 3)
    Bbar = B @ mw
    e = idx
    n = e.size
    u0 = ubar[e]                                                   # (n, 3)
    # neighbour means (ghost at walls)
    unb = np.zeros((n, 3, 3))
    for f in range(3):
        nb = mesh.EToE[e, f]
        inner = nb >= 0
        unb[inner, f, :] = ubar[nb[inner]]
        gi = ~inner
        go = np.zeros_like(gi)                  # open (far-field) boundary faces
        if getattr(model, "farfield", None) is not None:
            ffm = getattr(model, "farfield_faces", None)
            go = gi if ffm is None else gi & ffm[e, f]
        gw = gi & ~go                           # walls
        if np.any(go):
            hf, huf, hvf = model.farfield       # far-field ghost mean over the own mean bed
            unb[go, f, 0] = hf + Bbar[e[go]]
            unb[go, f, 1] = huf
            unb[go, f, 2] = hvf
        if np.any(gw):
            nx, ny = mesh.nx[e[gw], f], mesh.ny[e[gw], f]
            mn = u0[gw, 1] * nx + u0[gw, 2] * ny
            unb[gw, f, 0] = u0[gw, 0]
            unb[gw, f, 1] = u0[gw, 1] - 2.0 * mn * nx
            unb[gw, f, 2] = u0[gw, 2] - 2.0 * mn * ny
    # P1 part and the edge-midpoint deltas
    vn = ref.vertex_nodes
    qv = np.stack([(eta[e] @ ref.Pi1.T)[:, vn], (hu[e] @ ref.Pi1.T)[:, vn],
                   (hv[e] @ ref.Pi1.T)[:, vn]], axis=2)            # (n, 3 vertices, 3 fields)
    mids = np.stack([0.5 * (qv[:, 0] + qv[:, 1]), 0.5 * (qv[:, 1] + qv[:, 2]),
                     0.5 * (qv[:, 2] + qv[:, 0])], axis=1)          # (n, 3 edges, 3 fields)
    dtil = mids - u0[:, None, :]
    dnb = np.zeros((n, 3, 3))
    for i in range(3):
        j = jsel[e, i]
        uj = unb[np.arange(n), j, :]
        dnb[:, i, :] = alpha[e, i, None] * (unb[:, i, :] - u0) + beta[e, i, None] * (uj - u0)
    # characteristic limiting per edge
    hb = u0[:, 0] - Bbar[e]
    ub = u0[:, 1] / hb
    vb = u0[:, 2] / hb
    dist = np.hypot(dm[e, :, 0], dm[e, :, 1])                      # (n, 3)
    cb = np.sqrt(g * hb)
    floor = TVB_FLOOR * (hb + np.hypot(u0[:, 1], u0[:, 2]) / cb)
    fscale = np.stack([np.ones_like(cb), cb, np.ones_like(cb)], axis=1)   # (n, 3 components)
    changed = np.zeros(n, bool)
    dlim = np.zeros((n, 3, 3))
    for i in range(3):
        nx = dm[e, i, 0] / dist[:, i]
        ny = dm[e, i, 1] / dist[:, i]
        R = swe_eigenvectors(hb, ub, vb, nx, ny, g)
        L = np.linalg.inv(R)
        wt = np.einsum("nab,nb->na", L, dtil[:, i, :])
        wn = np.einsum("nab,nb->na", L, dnb[:, i, :])
        thr = (M * dist[:, i] ** 2 + floor)[:, None] * fscale
        wl = _tvb_minmod(wt, nu * wn, thr)
        changed |= np.any(wl != wt, axis=1)
        dlim[:, i, :] = np.einsum("nab,nb->na", R, wl)
    # redistribution so that the three deltas of each field sum to zero
    pos = np.maximum(dlim, 0.0).sum(axis=1)                          # (n, 3)
    neg = np.maximum(-dlim, 0.0).sum(axis=1)
    tp = np.where(pos > 0, np.minimum(1.0, neg / np.where(pos > 0, pos, 1.0)), 1.0)
    tn = np.where(neg > 0, np.minimum(1.0, pos / np.where(neg > 0, neg, 1.0)), 1.0)
    dhat = tp[:, None, :] * np.maximum(dlim, 0.0) - tn[:, None, :] * np.maximum(-dlim, 0.0)
    # depth deltas: eta deltas minus those of Pi1 B
    Bv = (B[e] @ ref.Pi1.T)[:, vn]
    Bmid = np.stack([0.5 * (Bv[:, 0] + Bv[:, 1]), 0.5 * (Bv[:, 1] + Bv[:, 2]),
                     0.5 * (Bv[:, 2] + Bv[:, 0])], axis=1)
    dh = dhat[:, :, 0] - (Bmid - Bbar[e][:, None])
    dh = positivity_modify(hb, dh, h0)
    # rebuild P1 nodal values where anything changed
    lam = np.stack([-(ref.r + ref.s) / 2.0, (1.0 + ref.r) / 2.0, (1.0 + ref.s) / 2.0], axis=0)  # (3, Np)

    def vertex_vals(mean, d):
        return np.stack([mean + d[:, 0] + d[:, 2] - d[:, 1], mean + d[:, 1] + d[:, 0] - d[:, 2],
                         mean + d[:, 2] + d[:, 1] - d[:, 0]], axis=1)

    c = np.nonzero(changed)[0]
    if c.size:
        ec = e[c]
        hvv = vertex_vals(hb[c], dh[c])
        h[ec] = hvv @ lam
        hu[ec] = vertex_vals(u0[c, 1], dhat[c, :, 1]) @ lam
        hv[ec] = vertex_vals(u0[c, 2], dhat[c, :, 2]) @ lam
        limited[ec] = True
    return h, hu, hv, limited
