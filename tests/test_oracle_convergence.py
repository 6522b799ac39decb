"""Solution-level pins of the oracle: design order of convergence on forced
manufactured solutions, and the regularized solutions approaching the ideal
Bingham law as the regularization parameter grows.

Manufactured solutions (tests/oracle_forced.py): a smooth pulse of depth and
velocity on a still layer over a slope (alpha = 0.1), with the forcing that
makes it an exact solution of Eq. shallowR2/3 added to the source.  The
oracle's SSP-RK3 run to time T, started from the nodal interpolant, must
converge to it in L2 (measured with a quadrature rule three orders finer
than the scheme's) at the design rate: p + 1 without stress (HLL fluxes,
slope source, primitive mass matrix), and at least p with the viscous
stress and the tanh regularization of Sec. 4 (Eq. sigmaTwoC) handled by the
central fluxes of the E-step and Q.  A dropped or mis-signed term leaves an
error of the size of that term times T, which does not converge at all.

The stress is kept mild here (eta = 0.01, sigma0 = 0.02, gamma = 2): with a
sharper regularization (gamma = 5 and above; the tanh transition has width
1/gamma in E) or a stronger viscosity (eta = 0.05) the meshes below are
pre-asymptotic for p = 3 in 1D (rate 2.9 only at 160 elements for
gamma = 5, 1.6 at 160 elements for gamma = 20).  A mistake in a stress term
still leaves a non-converging error of its size times T (about 1e-3 here,
against converged errors of 1e-5 to 1e-9).
"""
import math

import numpy as np
import pytest

import oracle_forced
import synth
from oracle import refelem as R
from oracle.dg import Discretization
from oracle.run import node_coords

INVISCID = dict(reg=0, eta=0.0, sigma0=0.0, alpha=0.1)
VISCOUS = dict(reg=3, eta=0.01, sigma0=0.02, gamma=2.0, alpha=0.1)


def _forced_run(dim, p, n, prm, T, L=1.5):
    if dim == 1:
        coords, etov = synth.interval_mesh(n, -L, L)
    else:
        coords, etov = synth.rect_tri_mesh(n, n, -L, L, -L, L)
    exact, forcing = oracle_forced.forced_problem(dim, prm)
    d = Discretization(dim, coords, etov, p, prm, face_bc=np.zeros((etov.shape[0], dim + 1), dtype=np.int64))
    Vh = d.to_modal(exact(0.0, node_coords(dim, coords, etov, p)))
    xq = d.map_to_phys(d.rq)

    def rhs(V, t):
        r = d.spatial_residual(V, d.e_step(V))
        r = r - np.einsum("kq,qa,vkq->vka", d.wJ, d.Phi, forcing(t, xq))
        return d.mass_solve(V, r)

    steps = int(math.ceil(T / d.stable_dt(Vh)))
    dt = T / steps
    t = 0.0
    for _ in range(steps):  # Shu-Osher SSP-RK3 with the forcing at the stage times
        V1 = Vh + dt * rhs(Vh, t)
        V2 = 0.75 * Vh + 0.25 * (V1 + dt * rhs(V1, t + dt))
        Vh = Vh / 3.0 + 2.0 / 3.0 * (V2 + dt * rhs(V2, t + 0.5 * dt))
        t += dt
    rh, wh = R.vol_rule(dim, p + 3)
    Vq = np.einsum("qa,vka->vkq", R.basis(dim, p, rh)[0], Vh)
    ex = exact(T, d.map_to_phys(rh))
    w = wh[None, :] * d.J[:, None]
    return np.array([math.sqrt(np.sum(w * (Vq[v] - ex[v]) ** 2)) for v in range(dim + 1)])


def _rates(dim, p, ns, prm, T):
    e = np.array([_forced_run(dim, p, n, synth.cases.default_params(**prm), T) for n in ns])
    return np.log2(e[:-1] / e[1:]), e


@pytest.mark.parametrize("p", [1, 2, 3])
def test_design_order_inviscid_1d(p):
    """Measured rates on 20 -> 40 elements: 1.96-2.00 (p = 1), 2.98-3.01
    (p = 2), 3.94-3.95 (p = 3)."""
    rates, e = _rates(1, p, (10, 20, 40), INVISCID, 0.1)
    assert rates[-1].min() > p + 1 - 0.2, (rates, e)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_design_order_viscous_bingham_1d(p):
    """Measured on 40 -> 80 elements: 1.97-2.00, 2.82-3.16, 3.09-3.56."""
    rates, e = _rates(1, p, (20, 40, 80), VISCOUS, 0.03)
    assert rates[-1].min() > p, (rates, e)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_design_order_inviscid_2d(p):
    """Structured triangulations of 4x4, 8x8 and 16x16 squares; rates on the
    finest pair approach p + 1 from below (measured 1.65-1.77, 3.02-3.22,
    3.52-3.70)."""
    rates, e = _rates(2, p, (4, 8, 16), INVISCID, 0.1)
    assert rates[-1].min() > p + 0.4, (rates, e)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_design_order_viscous_bingham_2d(p):
    """Measured 1.66-1.77 (p = 1), 3.11-3.20 (p = 2), 3.71-3.80 (p = 3)."""
    rates, e = _rates(2, p, (4, 8, 16), VISCOUS, 0.02)
    assert rates[-1].min() > p, (rates, e)


# ------------------------------------------------------------------ regularization limit

@pytest.mark.parametrize("reg", [1, 2, 3])
def test_regularized_solutions_form_cauchy_sequence(reg):
    """Sec. 4 / Sec. 6.2: as the regularization parameter grows the
    regularized solutions approach the ideal Bingham solution.  On the
    inclined layer with a parallel free surface (the paper's yield test
    geometry) and yield stress 8, the backward-Euler Newton oracle (Sec. 5.1)
    to t = 1 at gamma = beta = 1e2, 1e3, 1e4 gives velocities whose
    successive L2 differences shrink: by about 4 (regularizations 1 and 2)
    and 9 (regularization 3) per decade of gamma, with the material creeping
    towards rest (active region 0 %).  In a flowing state (yield stress 6)
    this Newton does not converge at gamma >= 1e3 with dt = 0.05-0.1, even
    with continuation in gamma, so the flowing regime is not part of the pin."""
    import warnings
    from oracle.implicit import Implicit1D
    from oracle.run import build
    sols, w = [], None
    for gamma in (1e2, 1e3, 1e4):
        c = synth.parallel_surface_1d(n_el=60, order=1, reg=reg, gamma=gamma, beta=gamma, m3=1, sigma0=8.0)
        d, V0, _ = build(c)
        im = Implicit1D(d, 0.1)
        with warnings.catch_warnings():
            warnings.simplefilter("error")
            X, its, fails = im.run(d.to_modal(V0), 10)
        assert fails == 0
        assert im.active_percent(X) == 0.0
        sols.append(d.eval_at_quad(im.unpack(X)[0])[1])
        w = d.wJ
    l2 = lambda a: math.sqrt(np.sum(w * a ** 2))  # noqa: E731
    d12, d23 = l2(sols[1] - sols[0]), l2(sols[2] - sols[1])
    assert d12 > 3.0 * d23, (d12, d23)
    # and the velocities themselves decrease towards the ideal law's rest state
    assert l2(sols[0]) > l2(sols[1]) > l2(sols[2])
