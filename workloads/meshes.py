"""Seeded triangle-mesh generators shared by the oracle tests and the CUDA tests.

These functions only lay out vertices and triangles; they contain none of the
discretisation's arithmetic (no nodes, no operators, no geometric factors).

Conventions
-----------
* ``vx, vy``: float64 vertex coordinates, shape (Nv,).
* ``EToV``: int32 (K, 3) vertex indices, counter-clockwise.
* Each square cell (i, j) with corners v00, v10, v11, v01 is split into the two
  triangles (v00, v10, v11) and (v00, v11, v01), both counter-clockwise.
"""
from __future__ import annotations

import numpy as np


def _split_cells(nx: int, ny: int) -> np.ndarray:
    """Triangles of an (nx x ny) vertex-lattice of cells, row-major cell order."""
    vid = np.arange((nx + 1) * (ny + 1), dtype=np.int64).reshape(ny + 1, nx + 1)
    v00 = vid[:-1, :-1].ravel()
    v10 = vid[:-1, 1:].ravel()
    v11 = vid[1:, 1:].ravel()
    v01 = vid[1:, :-1].ravel()
    t1 = np.stack([v00, v10, v11], axis=1)
    t2 = np.stack([v00, v11, v01], axis=1)
    # interleave so the two triangles of a cell are adjacent in memory
    tri = np.empty((2 * t1.shape[0], 3), dtype=np.int64)
    tri[0::2] = t1
    tri[1::2] = t2
    return tri.astype(np.int32)


def structured_rect(x0: float, x1: float, y0: float, y1: float, nx: int, ny: int):
    """Uniform nx x ny cells on [x0,x1] x [y0,y1], each cut into two triangles."""
    xs = np.linspace(x0, x1, nx + 1)
    ys = np.linspace(y0, y1, ny + 1)
    X, Y = np.meshgrid(xs, ys)
    return X.ravel().astype(np.float64), Y.ravel().astype(np.float64), _split_cells(nx, ny)


def graded_x_coords(x0: float, x1: float, nx: int, ratio: float) -> np.ndarray:
    """nx+1 x-coordinates whose spacing shrinks geometrically from x0 to x1.

    The first spacing is ``ratio`` times the last one (coarse at x0, fine at x1).
    """
    if nx < 1:
        raise ValueError("nx must be >= 1")
    if ratio == 1.0:
        return np.linspace(x0, x1, nx + 1)
    q = (1.0 / ratio) ** (1.0 / max(nx - 1, 1))
    d = q ** np.arange(nx)
    d = d / d.sum() * (x1 - x0)
    xs = np.concatenate([[x0], x0 + np.cumsum(d)])
    xs[-1] = x1
    return xs


def graded_jittered_rect(x0: float, x1: float, y0: float, y1: float, nx: int, ny: int,
                         ratio: float = 8.0, jitter: float = 0.15, seed: int = 3):
    """Graded (in x) structured grid with seeded interior-vertex jitter.

    Interior vertices move by U(-jitter, jitter) times the local spacing in each
    direction (numpy PCG64 generator seeded with ``seed``); boundary vertices
    stay on the boundary (they move only along it, not at corners).
    """
    xs = graded_x_coords(x0, x1, nx, ratio)
    ys = np.linspace(y0, y1, ny + 1)
    X, Y = np.meshgrid(xs, ys)
    dxl = np.diff(xs)
    # local spacing at each vertex column: the smaller adjacent interval
    hx = np.empty(nx + 1)
    hx[0] = dxl[0]
    hx[-1] = dxl[-1]
    hx[1:-1] = np.minimum(dxl[:-1], dxl[1:])
    hy = (y1 - y0) / ny
    rng = np.random.Generator(np.random.PCG64(seed))
    jx = rng.uniform(-jitter, jitter, size=X.shape) * hx[None, :]
    jy = rng.uniform(-jitter, jitter, size=Y.shape) * hy
    jx[:, 0] = 0.0
    jx[:, -1] = 0.0
    jy[0, :] = 0.0
    jy[-1, :] = 0.0
    X = X + jx
    Y = Y + jy
    return X.ravel().astype(np.float64), Y.ravel().astype(np.float64), _split_cells(nx, ny)


def centroids(vx, vy, EToV):
    """Element centroids (mean of the three vertices)."""
    cx = vx[EToV].mean(axis=1)
    cy = vy[EToV].mean(axis=1)
    return cx, cy
