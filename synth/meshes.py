"""Meshes for the synthetic workloads.

* ``interval_mesh``: uniform 1D intervals.
* ``rect_tri_mesh``: structured triangulation of a rectangle; every grid square
  (i, j) is cut along its (i, j) -> (i+1, j+1) diagonal into two
  counter-clockwise triangles.  Interior vertices may be jittered by a seeded
  uniform perturbation of +-``jitter`` grid spacings per coordinate
  (numpy ``default_rng(seed)``, PCG64).
"""
import numpy as np


def interval_mesh(n_el, x0=0.0, x1=1.0):
    """Uniform mesh of [x0, x1]: coords (n_el+1, 1) float64, EToV (n_el, 2) int32."""
    x = np.linspace(x0, x1, n_el + 1)
    etov = np.stack([np.arange(n_el), np.arange(1, n_el + 1)], axis=1).astype(np.int32)
    return x.reshape(-1, 1).astype(np.float64), etov


def rect_tri_mesh(nx, ny, x0=-1.0, x1=1.0, y0=-1.0, y1=1.0, jitter=0.0, seed=None):
    """Structured triangulation with 2*nx*ny CCW triangles.

    Returns coords (n_v, 2) float64 and EToV (2*nx*ny, 3) int32.  Vertex (i, j)
    has index j*(nx+1)+i.  Square (i, j) gives triangles
    (v(i,j), v(i+1,j), v(i+1,j+1)) and (v(i,j), v(i+1,j+1), v(i,j+1)), stored
    square by square, row by row.
    """
    xs = np.linspace(x0, x1, nx + 1)
    ys = np.linspace(y0, y1, ny + 1)
    X, Y = np.meshgrid(xs, ys, indexing="xy")  # (ny+1, nx+1)
    coords = np.stack([X.ravel(), Y.ravel()], axis=1).astype(np.float64)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        hx = (x1 - x0) / nx
        hy = (y1 - y0) / ny
        d = rng.uniform(-jitter, jitter, size=coords.shape)
        ii = np.tile(np.arange(nx + 1), ny + 1)
        jj = np.repeat(np.arange(ny + 1), nx + 1)
        interior = (ii > 0) & (ii < nx) & (jj > 0) & (jj < ny)
        coords[interior, 0] += d[interior, 0] * hx
        coords[interior, 1] += d[interior, 1] * hy

    def v(i, j):
        return j * (nx + 1) + i

    i = np.tile(np.arange(nx), ny)
    j = np.repeat(np.arange(ny), nx)
    a, b, c, dd = v(i, j), v(i + 1, j), v(i + 1, j + 1), v(i, j + 1)
    t1 = np.stack([a, b, c], axis=1)
    t2 = np.stack([a, c, dd], axis=1)
    etov = np.empty((2 * nx * ny, 3), dtype=np.int32)
    etov[0::2] = t1
    etov[1::2] = t2
    return coords, etov
