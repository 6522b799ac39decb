"""Reference-element quadrature, modal bases and node sets for the oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* Basis: orthonormal Legendre polynomials on [-1, 1] (Sec. 5 uses normalized
  Legendre polynomials) and, on the reference triangle
  T = {r, s >= -1, r + s <= 0}, the orthonormal collapsed-coordinate (Dubiner)
  basis psi_ij = sqrt(2) P_i(a) P_j^{(2i+1,0)}(b) (1-b)^i with
  a = 2(1+r)/(1-s) - 1, b = s, ordered (i, j) with i outer, i + j <= p.
  Derivatives follow from the chain rule on (a, b), derived here.
* Quadrature (the paper does not name a rule): Gauss-Legendre on lines; on
  the triangle the collapsed product of Gauss-Legendre in a and Gauss-Jacobi
  (1, 0) in b.  Volume rules take n = ceil(3p/2) points per direction (exact
  to degree 3p - 1), edge rules n = ceil((3p+1)/2) (exact to degree 3p): the
  degrees of the h^2 flux and the h dH/dx source terms, so that a lake at rest
  is preserved exactly.
* Nodes (where initial data and the bed are sampled): equispaced;
  line node i at -1 + 2i/p; triangle node (i, j) at (-1 + 2i/p, -1 + 2j/p) for
  j = 0..p outer, i = 0..p-j inner.
"""
import math
import numpy as np
from numpy.polynomial import legendre as npleg
from scipy.special import roots_jacobi, eval_jacobi

TRI_VERTS = np.array([[-1.0, -1.0], [1.0, -1.0], [-1.0, 1.0]])


def n_vol(p):
    return int(math.ceil(3 * p / 2))


def n_face(p):
    return int(math.ceil((3 * p + 1) / 2))


def rule_line(n):
    x, w = npleg.leggauss(n)
    return x, w


def rule_tri(n):
    a, wa = npleg.leggauss(n)
    b, wb = roots_jacobi(n, 1.0, 0.0)
    A, B = np.meshgrid(a, b, indexing="ij")
    r = 0.5 * (1.0 + A) * (1.0 - B) - 1.0
    s = B
    w = 0.5 * wa[:, None] * wb[None, :]
    return r.ravel(), s.ravel(), w.ravel()


def legendre_orthonormal(x, n):
    """Orthonormal Legendre P_n on [-1,1] and its derivative at x."""
    c = np.zeros(n + 1)
    c[n] = 1.0
    scale = math.sqrt((2 * n + 1) / 2.0)
    return scale * npleg.legval(x, c), scale * npleg.legval(x, npleg.legder(c))


def jacobi_orthonormal(x, a, b, n):
    """Orthonormal Jacobi P_n^{(a,b)} (weight (1-x)^a (1+x)^b) and derivative."""
    hn = (2.0 ** (a + b + 1) / (2 * n + a + b + 1)
          * math.gamma(n + a + 1) * math.gamma(n + b + 1)
          / (math.gamma(n + a + b + 1) * math.gamma(n + 1)))
    val = eval_jacobi(n, a, b, x) / math.sqrt(hn)
    if n == 0:
        der = np.zeros_like(np.asarray(x, dtype=float))
    else:
        der = 0.5 * (n + a + b + 1) * eval_jacobi(n - 1, a + 1, b + 1, x) / math.sqrt(hn)
    return val, der


def modes_tri(p):
    return [(i, j) for i in range(p + 1) for j in range(p + 1 - i)]


def n_modes(dim, p):
    return p + 1 if dim == 1 else (p + 1) * (p + 2) // 2


def basis_line(p, r):
    r = np.asarray(r, dtype=float)
    Phi = np.empty((r.size, p + 1))
    dPhi = np.empty((r.size, p + 1))
    for n in range(p + 1):
        Phi[:, n], dPhi[:, n] = legendre_orthonormal(r, n)
    return Phi, dPhi


def basis_tri(p, r, s):
    """Values and (d/dr, d/ds) of the orthonormal triangle basis at (r, s)."""
    r = np.asarray(r, dtype=float)
    s = np.asarray(s, dtype=float)
    one_m_b = 1.0 - s
    safe = one_m_b > 1e-14
    a = np.where(safe, 2.0 * (1.0 + r) / np.where(safe, one_m_b, 1.0) - 1.0, -1.0)
    b = s
    modes = modes_tri(p)
    Phi = np.empty((r.size, len(modes)))
    Pr = np.empty_like(Phi)
    Ps = np.empty_like(Phi)
    for m, (i, j) in enumerate(modes):
        f, df = legendre_orthonormal(a, i)
        g, dg = jacobi_orthonormal(b, 2 * i + 1, 0, j)
        c = math.sqrt(2.0)
        Phi[:, m] = c * f * g * one_m_b ** i
        # d/dr: da/dr = 2/(1-b)
        # d/ds: da/ds = (1+a)/(1-b), db/ds = 1
        if i == 0:
            Pr[:, m] = 0.0
            Ps[:, m] = c * f * dg
        else:
            q = one_m_b ** (i - 1)
            Pr[:, m] = c * 2.0 * df * g * q
            Ps[:, m] = c * (df * (1.0 + a) * g * q + f * (dg * one_m_b ** i - i * g * q))
    return Phi, Pr, Ps


def nodes_line(p):
    return -1.0 + 2.0 * np.arange(p + 1) / p


def nodes_tri(p):
    pts = [(-1.0 + 2.0 * i / p, -1.0 + 2.0 * j / p) for j in range(p + 1) for i in range(p + 1 - j)]
    return np.array(pts)


def basis(dim, p, pts):
    """(Phi, [dPhi/dr, dPhi/ds]) at reference points pts (npts, dim)."""
    pts = np.atleast_2d(np.asarray(pts, dtype=float))
    if dim == 1:
        Phi, dr = basis_line(p, pts[:, 0])
        return Phi, [dr]
    Phi, dr, ds = basis_tri(p, pts[:, 0], pts[:, 1])
    return Phi, [dr, ds]


def vol_rule(dim, p):
    """Volume points (nq, dim) and weights."""
    n = n_vol(p)
    if dim == 1:
        x, w = rule_line(n)
        return x.reshape(-1, 1), w
    r, s, w = rule_tri(n)
    return np.stack([r, s], axis=1), w


def ref_nodes(dim, p):
    if dim == 1:
        return nodes_line(p).reshape(-1, 1)
    return nodes_tri(p)


def face_points_ref(dim, p):
    """Reference coordinates of the face quadrature points, (nf, nfq, dim), the
    1D edge parameters t (nfq,) and edge weights (nfq,).  Triangle face f runs
    from vertex f to vertex (f+1) % 3; a point at parameter t sits at
    (1-t)/2 v_f + (1+t)/2 v_{f+1}.  Line faces are the end points r = -1, +1."""
    if dim == 1:
        return np.array([[[-1.0]], [[1.0]]]), np.array([0.0]), np.array([1.0])
    t, w = rule_line(n_face(p))
    out = np.empty((3, t.size, 2))
    for f in range(3):
        va, vb = TRI_VERTS[f], TRI_VERTS[(f + 1) % 3]
        out[f] = 0.5 * (1 - t)[:, None] * va + 0.5 * (1 + t)[:, None] * vb
    return out, t, w
