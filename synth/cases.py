"""Synthetic workloads: dam breaks, lakes at rest, random smooth states.

A ``Case`` bundles a mesh, boundary tags, physical parameters and the initial
fields as functions of physical coordinates.  ``Case.initial_state`` samples
them at node coordinates supplied by the caller (each consumer computes its
own nodes), so the same seeded input reaches the oracle and the library.

Sampling rule: every field function takes ``(x, xc)``: the sample points and
the centroid of the element each point belongs to.  Smooth fields use ``x``
only; step functions (dam lines) decide the side by ``xc``, so each element
lies wholly on one side and the initial discontinuity sits on element faces.

Regularization ids follow the paper's numbering (smooth max = 1, local
quadratic = 2, tanh = 3); 4 (exponential, Papanastasiou) and 5 (bi-viscosity)
are extensions the paper does not define.
"""
from dataclasses import dataclass, field
import math
import numpy as np

from .meshes import interval_mesh, rect_tri_mesh

REG_NONE, REG_SMOOTH_MAX, REG_LOCAL_QUAD, REG_TANH, REG_EXP, REG_BIVISC = 0, 1, 2, 3, 4, 5
BC_COPY, BC_DIRICHLET, BC_WALL = 0, 1, 2

def default_params(**kw):
    p = dict(g=9.81, rho=1.0, alpha=0.0, eta=0.01, sigma0=0.0, gamma=1e3, beta=1e3,
             pap_m=1e3, h_floor=1e-6, cfl=0.3, reg=REG_NONE)
    p.update(kw)
    return p


@dataclass
class Case:
    name: str
    dim: int
    coords: np.ndarray          # (n_v, dim) float64
    etov: np.ndarray            # (K, dim+1) int32
    face_bc: np.ndarray         # (K, n_faces) int8: boundary descriptor index per element face
    bcs: list                   # list of (modes[7], values[7]); slots = V fields then E fields
    order: int
    params: dict
    h_fn: object = None         # depth h(x) ; x has shape (npts, dim)
    u_fn: object = None         # velocity (npts, dim)
    bed_fn: object = None       # bed H(x) or None (flat)
    n_steps: int = 0
    dt: float = 0.0             # fixed step for the implicit integrator (0: CFL)
    t_final: float = 0.0
    m3: int = -1                # order of E (-1: same as order)
    extra: dict = field(default_factory=dict)

    @property
    def n_elements(self):
        return int(self.etov.shape[0])

    @property
    def n_faces(self):
        return self.dim + 1

    @property
    def nV(self):
        return self.dim + 1

    @property
    def nE(self):
        return self.dim * self.dim

    def centroids(self):
        return self.coords[self.etov].mean(axis=1)

    def initial_state(self, node_xyz):
        """Nodal initial state V (nV, K, Np) and bed (K, Np) (zeros if flat)."""
        K, Np, d = node_xyz.shape
        x = node_xyz.reshape(-1, d)
        xc = np.repeat(self.centroids(), Np, axis=0)
        h = np.asarray(self.h_fn(x, xc), dtype=np.float64).reshape(K, Np)
        u = np.asarray(self.u_fn(x, xc), dtype=np.float64).reshape(K, Np, d)
        V = np.empty((d + 1, K, Np))
        V[0] = h
        for j in range(d):
            V[1 + j] = u[:, :, j]
        if self.bed_fn is None:
            bed = np.zeros((K, Np))
        else:
            bed = np.asarray(self.bed_fn(x, xc), dtype=np.float64).reshape(K, Np)
        return V, bed


def _bc(modes=None, values=None):
    m = [BC_COPY] * 7
    v = [0.0] * 7
    if modes:
        for k, val in modes.items():
            m[k] = val
    if values:
        for k, val in values.items():
            v[k] = float(val)
    return (m, v)


def _face_bc_1d(K):
    fb = np.zeros((K, 2), dtype=np.int8)
    fb[:, 1] = 1  # right ends use descriptor 1, left ends descriptor 0
    return fb


def _face_bc_2d(K, value=0):
    return np.full((K, 3), value, dtype=np.int8)


def _zero_u(dim):
    return lambda x, xc=None: np.zeros((x.shape[0], dim))


# ---------------------------------------------------------------- workloads

def dam_break_1d(n_el=200, order=1, reg=REG_EXP, sigma0=0.05, eta=0.01, pap_m=1e3,
                 hl=1.0, hr=0.5, x_dam=0.5, n_steps=2000, cfl=0.3, **kw):
    """1D Bingham dam break on [0, 1]: depth hl left of x_dam, hr right, zero
    velocity, copy (homogeneous Neumann) boundaries."""
    coords, etov = interval_mesh(n_el, 0.0, 1.0)
    params = default_params(reg=reg, sigma0=sigma0, eta=eta, pap_m=pap_m, cfl=cfl, **kw)
    return Case("dam_break_1d", 1, coords, etov, _face_bc_1d(n_el), [_bc(), _bc()], order,
                params, h_fn=lambda x, xc: np.where(xc[:, 0] < x_dam, hl, hr), u_fn=_zero_u(1),
                n_steps=n_steps)


def radial_dam_2d(n=64, order=2, reg=REG_SMOOTH_MAX, sigma0=0.02, eta=0.01, gamma=1e3,
                  beta=1e3, h_in=2.0, h_out=0.5, r0=0.3, n_steps=5000, cfl=0.3, **kw):
    """2D radial dam break on [-1, 1]^2 (n x n squares, 2 n^2 triangles)."""
    coords, etov = rect_tri_mesh(n, n)
    params = default_params(reg=reg, sigma0=sigma0, eta=eta, gamma=gamma, beta=beta, cfl=cfl,
                            **kw)
    K = etov.shape[0]

    def h_fn(x, xc):
        r = np.sqrt(xc[:, 0] ** 2 + xc[:, 1] ** 2)
        return np.where(r < r0, h_in, h_out)

    return Case("radial_dam_2d", 2, coords, etov, _face_bc_2d(K), [_bc()], order, params,
                h_fn=h_fn, u_fn=_zero_u(2), n_steps=n_steps)


def bump_dam_2d(n=512, order=3, seed=3, sigma0=0.05, eta=0.01, gamma=1e3, amp=0.2, width=0.1,
                x_dam=-0.5, s_up=1.0, s_down=0.5, n_steps=1000, cfl=0.3, **kw):
    """2D dam break over a Gaussian bed bump on a jittered n x n triangulation."""
    coords, etov = rect_tri_mesh(n, n, jitter=0.1, seed=seed)
    params = default_params(reg=REG_TANH, sigma0=sigma0, eta=eta, gamma=gamma, cfl=cfl, **kw)
    K = etov.shape[0]

    def bed(x, xc=None):
        return amp * np.exp(-(x[:, 0] ** 2 + x[:, 1] ** 2) / (2 * width ** 2))

    def h_fn(x, xc):
        surf = np.where(xc[:, 0] < x_dam, s_up, s_down)
        return surf - bed(x)

    return Case("bump_dam_2d", 2, coords, etov, _face_bc_2d(K), [_bc()], order, params,
                h_fn=h_fn, u_fn=_zero_u(2), bed_fn=bed, n_steps=n_steps)


def dry_dam_2d(n=1024, order=1, hl=1.0, x_dam=0.0, cfl=0.3, **kw):
    """Dam break onto a dry bed on [-1, 1]^2 (n x n squares, 2 n^2
    triangles): depth hl for x_1 < x_dam, exactly 0 beyond, at rest, flat
    bed, Newtonian limit (no yield stress, no viscosity), reflecting walls,
    wet/dry mode on.  Its x_1 profile follows Ritter's solution until the
    waves reach the walls."""
    coords, etov = rect_tri_mesh(n, n)
    params = default_params(reg=REG_NONE, sigma0=0.0, eta=0.0, cfl=cfl, positivity=1, **kw)
    K = etov.shape[0]
    wall = _bc(modes={1: BC_WALL, 2: BC_WALL})
    return Case("dry_dam_2d", 2, coords, etov, _face_bc_2d(K), [wall], order, params,
                h_fn=lambda x, xc: np.where(xc[:, 0] < x_dam, hl, 0.0), u_fn=_zero_u(2))


def _fourier_bed(seed, n_modes=16, kmax=4 * math.pi, amp=0.05):
    rng = np.random.default_rng(seed)
    ks = []
    while len(ks) < n_modes:
        k = rng.uniform(-kmax, kmax, size=2)
        if np.hypot(*k) <= kmax:
            ks.append(k)
    ks = np.array(ks)
    ph = rng.uniform(0, 2 * math.pi, size=n_modes)
    a = rng.normal(size=n_modes)
    grid = np.linspace(-1, 1, 201)
    X, Y = np.meshgrid(grid, grid)
    probe = sum(a[m] * np.cos(ks[m, 0] * X + ks[m, 1] * Y + ph[m]) for m in range(n_modes))
    scale = amp / np.abs(probe).max()

    def bed(x, xc=None):
        out = np.zeros(x.shape[0])
        for m in range(n_modes):
            out += a[m] * np.cos(ks[m, 0] * x[:, 0] + ks[m, 1] * x[:, 1] + ph[m])
        return scale * out
    return bed


def slump_2d(n=2048, order=2, seed=5, sigma0=0.05, eta=0.01, gamma=1e3, width=0.15,
             h_min=1e-3, n_steps=10000, cfl=0.3, **kw):
    """Bingham slump: Gaussian mound on an inclined plane (slope 0.05) over a
    seeded smooth bed; bi-viscosity regularization.  Depth is bounded below by
    ``h_min`` (a thin wet film)."""
    coords, etov = rect_tri_mesh(n, n)
    params = default_params(reg=REG_BIVISC, sigma0=sigma0, eta=eta, gamma=gamma,
                            alpha=math.atan(0.05), cfl=cfl, **kw)
    K = etov.shape[0]
    bed = _fourier_bed(seed)

    def h_fn(x, xc=None):
        return np.maximum(np.exp(-(x[:, 0] ** 2 + x[:, 1] ** 2) / (2 * width ** 2)), h_min)

    return Case("slump_2d", 2, coords, etov, _face_bc_2d(K), [_bc()], order, params,
                h_fn=h_fn, u_fn=_zero_u(2), bed_fn=bed, n_steps=n_steps)


def lake_at_rest_1d(n_el=100, order=1, eta=1.0, sigma0=1.0, reg=REG_SMOOTH_MAX, h0=3.0, L=10.0,
                    dt=1e-2, t_final=1.0, m3=-1, **kw):
    """Constant free surface on an inclined plane with bed cos(pi x): the fluid
    is at rest; Dirichlet data on both ends."""
    alpha = math.pi / 18
    coords, etov = interval_mesh(n_el, 0.0, L)
    params = default_params(reg=reg, eta=eta, sigma0=sigma0, alpha=alpha, gamma=1e3, beta=1e3,
                            **kw)
    ca, ta = math.cos(alpha), math.tan(alpha)

    def bed(x, xc=None):
        return np.cos(math.pi * x[:, 0])

    def h_fn(x, xc=None):
        return h0 / ca - x[:, 0] * ta - bed(x)

    hL = h0 / ca - 1.0
    hR = h0 / ca - L * ta - math.cos(math.pi * L)
    bcs = [_bc({0: BC_DIRICHLET, 1: BC_DIRICHLET, 2: BC_DIRICHLET}, {0: hL}),
           _bc({0: BC_DIRICHLET, 1: BC_DIRICHLET, 2: BC_DIRICHLET}, {0: hR})]
    return Case("lake_at_rest_1d", 1, coords, etov, _face_bc_1d(n_el), bcs, order, params,
                h_fn=h_fn, u_fn=_zero_u(1), bed_fn=bed, dt=dt, t_final=t_final, m3=m3)


def parallel_surface_1d(n_el=100, order=1, eta=1.0, sigma0=9.035, reg=REG_TANH, gamma=1e3,
                        beta=1e3, h0=3.0, L=10.0, dt=1e-3, t_final=1.0, m3=-1, **kw):
    """Free surface parallel to the inclined plane, bed cos(pi x); the material
    stays at rest when the yield stress exceeds the driving stress.  Copy
    boundaries except u = 0 at x = L."""
    alpha = math.pi / 18
    coords, etov = interval_mesh(n_el, 0.0, L)
    params = default_params(reg=reg, eta=eta, sigma0=sigma0, alpha=alpha, gamma=gamma, beta=beta,
                            **kw)

    def bed(x, xc=None):
        return np.cos(math.pi * x[:, 0])

    bcs = [_bc(), _bc({1: BC_DIRICHLET})]
    return Case("parallel_surface_1d", 1, coords, etov, _face_bc_1d(n_el), bcs, order, params,
                h_fn=lambda x, xc=None: h0 - bed(x), u_fn=_zero_u(1), bed_fn=bed, dt=dt, t_final=t_final,
                m3=m3)


def paper_dam_break_1d(n_el=100, order=1, m3=0, reg=REG_SMOOTH_MAX, sigma0=0.2, eta=0.02,
                       gamma=1e2, beta=1e2, h1=1.5, h2=0.5, L=3.0, dt=1e-6, t_final=0.15, **kw):
    """Dam break on a wet bed, Dirichlet depth at both ends, copy velocity,
    E = 0 at both ends."""
    coords, etov = interval_mesh(n_el, 0.0, L)
    params = default_params(reg=reg, eta=eta, sigma0=sigma0, gamma=gamma, beta=beta, **kw)
    bcs = [_bc({0: BC_DIRICHLET, 2: BC_DIRICHLET}, {0: h1}),
           _bc({0: BC_DIRICHLET, 2: BC_DIRICHLET}, {0: h2})]
    return Case("paper_dam_break_1d", 1, coords, etov, _face_bc_1d(n_el), bcs, order, params,
                h_fn=lambda x, xc: np.where(xc[:, 0] < L / 2, h1, h2), u_fn=_zero_u(1), dt=dt,
                t_final=t_final, m3=m3)


def random_smooth_fields(dim, seed, h_mean=1.0, h_amp=0.3, u_amp=0.5, n_modes=3, bed_amp=0.0):
    """Seeded smooth random (h, u, bed) functions: sums of low-wavenumber
    sinusoids; h stays above h_mean - h_amp * n_modes / n_modes."""
    rng = np.random.default_rng(seed)

    def make(amp):
        k = rng.uniform(0.5, 3.0, size=(n_modes, dim)) * rng.choice([-1, 1], size=(n_modes, dim))
        ph = rng.uniform(0, 2 * math.pi, size=n_modes)
        a = rng.uniform(-1, 1, size=n_modes) * amp / n_modes

        def f(x, xc=None):
            out = np.zeros(x.shape[0])
            for m in range(n_modes):
                out += a[m] * np.sin(x @ k[m] + ph[m])
            return out
        return f

    hf = make(h_amp)
    ufs = [make(u_amp) for _ in range(dim)]
    bf = make(bed_amp) if bed_amp > 0 else None

    def h_fn(x, xc=None):
        return h_mean + hf(x)

    def u_fn(x, xc=None):
        return np.stack([uf(x) for uf in ufs], axis=1)

    return h_fn, u_fn, bf


def ensemble_cases(n_inst=256, seed=4, n_min=1000, n_max=50000, n_steps=1000, eta=0.01,
                   gamma=1e3, beta=1e3, hr=0.5, cfl=0.3, size_scale=1.0):
    """Heterogeneous ensemble: per instance a log-uniform size in [n_min,
    n_max] elements (scaled by ``size_scale``), dimension 1 or 2 with equal
    probability, order uniform in {1, 2, 3}, yield stress log-uniform in
    [1e-3, 0.2], depth ratio uniform in [1.5, 4]; regularization cycles 1, 2, 3."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_inst):
        n_el = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max))) * size_scale))
        dim = int(rng.integers(1, 3))
        order = int(rng.integers(1, 4))
        sigma0 = float(math.exp(rng.uniform(math.log(1e-3), math.log(0.2))))
        ratio = float(rng.uniform(1.5, 4.0))
        reg = (REG_SMOOTH_MAX, REG_LOCAL_QUAD, REG_TANH)[i % 3]
        if dim == 1:
            c = dam_break_1d(n_el=max(n_el, 2), order=order, reg=reg, sigma0=sigma0, eta=eta,
                             hl=hr * ratio, hr=hr, n_steps=n_steps, cfl=cfl, gamma=gamma,
                             beta=beta)
        else:
            n = max(2, int(round(math.sqrt(n_el / 2.0))))
            coords, etov = rect_tri_mesh(n, n)
            params = default_params(reg=reg, sigma0=sigma0, eta=eta, gamma=gamma, beta=beta,
                                    cfl=cfl)
            hl = hr * ratio
            c = Case("ensemble_2d", 2, coords, etov, _face_bc_2d(etov.shape[0]), [_bc()], order,
                     params, h_fn=lambda x, xc, hl=hl: np.where(xc[:, 0] < 0.0, hl, hr),
                     u_fn=_zero_u(2), n_steps=n_steps)
        c.name = f"ensemble_{i}"
        out.append(c)
    return out
