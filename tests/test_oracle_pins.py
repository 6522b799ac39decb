"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed-form
integrals, polynomial exactness, the paper's well-balanced (lake at rest)
property (Sec. 6.1, Tables errorsEx1a/b: preserved to round-off for m0 <= m1),
HLL identities, the paper's regularization formulas against their limits and
finite differences (Sec. 4, Appendix A), a symbolic manufactured consistency
check of the whole spatial operator, mass conservation, the exact
Newtonian dam-break solution (Sec. 6.3) and the time integrator's order.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import refelem as R
from oracle import constitutive as C
from oracle import riemann
from oracle.dg import Discretization
from oracle.run import build, node_coords, residual_nodal

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ quadrature / basis

def _tri_monomial_exact(a, b):
    """Integral of r^a s^b over the reference triangle, from the unit-triangle
    formula  int x^i y^j = i! j! / (i+j+2)!  with r = 2x - 1, s = 2y - 1."""
    tot = Fraction(0)
    for i in range(a + 1):
        for j in range(b + 1):
            coef = (math.comb(a, i) * 2 ** i * (-1) ** (a - i)
                    * math.comb(b, j) * 2 ** j * (-1) ** (b - j))
            tot += coef * Fraction(math.factorial(i) * math.factorial(j),
                                   math.factorial(i + j + 2))
    return float(4 * tot)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_quadrature_exact(p):
    deg = 3 * p - 1
    x, w = R.vol_rule(1, p)
    for a in range(deg + 1):
        exact = (1 - (-1) ** (a + 1)) / (a + 1)
        assert abs(np.sum(w * x[:, 0] ** a) - exact) < 1e-14
    rs, w = R.vol_rule(2, p)
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            assert abs(np.sum(w * rs[:, 0] ** a * rs[:, 1] ** b) - _tri_monomial_exact(a, b)) < 1e-13
    t, wf = R.rule_line(R.n_face(p))
    for a in range(3 * p + 1):
        exact = (1 - (-1) ** (a + 1)) / (a + 1)
        assert abs(np.sum(wf * t ** a) - exact) < 1e-14


@pytest.mark.parametrize("dim,p", [(1, 1), (1, 3), (2, 1), (2, 2), (2, 3)])
def test_basis_orthonormal_and_gradient(dim, p):
    pts, w = R.vol_rule(dim, p + 1)  # exact to degree 3p+2 >= 2p
    Phi, d = R.basis(dim, p, pts)
    M = (Phi * w[:, None]).T @ Phi
    assert np.abs(M - np.eye(M.shape[0])).max() < 1e-13
    rng = np.random.default_rng(0)
    if dim == 1:
        P = rng.uniform(-0.9, 0.9, size=(5, 1))
    else:
        P = rng.uniform(-0.9, -0.1, size=(5, 2))
    eps = 1e-6
    _, dP = R.basis(dim, p, P)
    for a in range(dim):
        dp = np.zeros(dim)
        dp[a] = eps
        fd = (R.basis(dim, p, P + dp)[0] - R.basis(dim, p, P - dp)[0]) / (2 * eps)
        assert np.abs(fd - dP[a]).max() < 1e-7


# ------------------------------------------------------------------ well balance (P1, P2)

@pytest.mark.parametrize("dim", [1, 2])
def test_still_water_flat(dim):
    case = synth.dam_break_1d(n_el=12, order=2) if dim == 1 else synth.radial_dam_2d(n=4, order=2)
    case.h_fn = lambda x, xc=None: np.full(x.shape[0], 0.7)
    d, V0, _ = build(case)
    dv, E = residual_nodal(d, V0)
    assert np.abs(dv).max() < 1e-12 and np.abs(E).max() == 0.0


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("eta,sigma0", [(0.0, 0.0), (1.0, 0.0), (1.0, 1.0)])
@pytest.mark.parametrize("reg", [1, 2, 3])
def test_lake_at_rest_1d(p, eta, sigma0, reg):
    """Sec. 6.1 (constant free surface on a slope with bed cos(pi x)): with
    m0 = m1 the state is an equilibrium of the discrete scheme, whatever the
    viscosity, yield stress or regularization (Tables errorsEx1a/b)."""
    c = synth.lake_at_rest_1d(n_el=40, order=p, eta=eta, sigma0=sigma0, reg=reg)
    d, V0, _ = build(c)
    dv, E = residual_nodal(d, V0)
    assert np.abs(dv).max() < 1e-11
    assert np.abs(E).max() < 1e-12


@pytest.mark.parametrize("p", [1, 2, 3])
def test_lake_at_rest_2d_bump(p):
    c = synth.bump_dam_2d(n=6, order=p)
    c.h_fn = lambda x, xc=None, b=c.bed_fn: 1.0 - b(x)
    d, V0, _ = build(c)
    dv, _ = residual_nodal(d, V0)
    assert np.abs(dv).max() < 1e-11


def test_lake_at_rest_unbalanced_bed_moves():
    """The equilibrium needs m0 <= m1 (Sec. 6.1): a bed the depth space cannot
    balance (bed sampled at degree 2, depth at degree 1 -> the modal bed of
    degree 1 differs) must produce motion, so the pin above is not vacuous."""
    c = synth.lake_at_rest_1d(n_el=40, order=1)
    d, V0, bed = build(c)
    d2 = Discretization(1, c.coords, c.etov, 1, c.params, face_bc=c.face_bc, bcs=c.bcs,
                        bed_nodal=bed + 0.05 * np.sin(np.arange(bed.size)).reshape(bed.shape))
    dv, _ = residual_nodal(d2, V0)
    assert np.abs(dv[1]).max() > 1e-3


# ------------------------------------------------------------------ E-step (P3)

@pytest.mark.parametrize("p", [1, 2, 3])
def test_estep_exact_for_polynomials(p):
    coords, etov = synth.rect_tri_mesh(5, 5, jitter=0.1, seed=1)
    prm = synth.cases.default_params()
    d = Discretization(2, coords, etov, p, prm)
    x, y = d.node_xyz[..., 0], d.node_xyz[..., 1]
    u1 = x ** p + 0.5 * y
    u2 = x * y ** (p - 1)
    V = np.stack([np.ones_like(x), u1, u2])
    En = d.E_to_nodal(d.e_step(d.to_modal(V)))
    exact = [p * x ** (p - 1), y ** (p - 1), 0.5 + 0 * x, (p - 1) * x * y ** max(p - 2, 0)]
    for k in range(4):  # component 2i+j = d u_j / d x_i
        assert np.abs(En[k] - exact[k]).max() < 1e-12


# ------------------------------------------------------------------ HLL (P4)

@pytest.mark.parametrize("dim", [1, 2])
def test_hll_identities(dim):
    prm = synth.cases.default_params()
    if dim == 1:
        coords, etov = synth.interval_mesh(2)
    else:
        coords, etov = synth.rect_tri_mesh(1, 1)
    d = Discretization(dim, coords, etov, 1, prm)
    rng = np.random.default_rng(3)
    n = rng.normal(size=(dim, 50))
    n /= np.sqrt((n ** 2).sum(axis=0))
    Vm = np.vstack([rng.uniform(0.2, 2.0, 50), rng.normal(size=(dim, 50))])
    Vp = np.vstack([rng.uniform(0.2, 2.0, 50), rng.normal(size=(dim, 50))])
    # consistency: F_bar(U, U; n) = F(U) . n
    Fn = d.hll(Vm, Vm, n)
    F = d.flux_F(Vm)
    assert np.abs(Fn - sum(F[i] * n[i] for i in range(dim))).max() < 1e-13
    # conservation: F_bar(U-, U+; n) = -F_bar(U+, U-; -n)
    assert np.abs(d.hll(Vm, Vp, n) + d.hll(Vp, Vm, -n)).max() < 1e-13
    # supersonic flow to the right: upwind on the interior state
    Vs = Vm.copy()
    Vs[0] = 0.1
    Vs[1:] = 5.0 * n
    assert np.abs(d.hll(Vs, Vs * 1.01, n) - sum(d.flux_F(Vs)[i] * n[i] for i in range(dim))).max() < 1e-12


# ------------------------------------------------------------------ constitutive (P5, P12)

def _prm(reg, s0=1.0, gamma=10.0, beta=1.0, m=10.0, eta=0.0):
    return dict(reg=reg, sigma0=s0, gamma=gamma, beta=beta, pap_m=m, eta=eta)


@pytest.mark.parametrize("reg", [1, 2, 3, 4, 5])
def test_regularized_stress_2d_reduces_to_1d(reg):
    prm = _prm(reg, eta=0.3, gamma=50.0, beta=40.0)
    e = np.linspace(-0.2, 0.2, 41)
    E2 = np.zeros((4, e.size))
    E2[0] = e  # only du1/dx1
    s2 = C.stress(E2, 2, prm)
    s1 = C.stress(e[None], 1, prm)[0, 0]
    expected = 4 * 0.3 * e + np.sign(e) * C.phi(np.abs(e), prm)
    assert np.abs(s1 - expected).max() < 1e-13
    assert np.abs(s2[0, 0] - expected).max() < 1e-13
    assert np.abs(s2[0, 1]).max() == 0.0


def test_regs_1_and_2_coincide_outside_transition():
    """Regularizations 1 and 2 agree wherever |gamma|E| - sigma0| >= 1/(2 beta)
    (consistent with the identical columns of Table errorsEx1c)."""
    for s0, g, b in [(1.0, 10.0, 1.0), (0.2, 1e2, 1e2), (0.05, 1e3, 1e3)]:
        s = np.linspace(0, 3 * s0 / g, 301)
        x = g * s
        mask = np.abs(x - s0) >= 1 / (2 * b)
        p1 = C.phi(s, _prm(1, s0, g, b))
        p2 = C.phi(s, _prm(2, s0, g, b))
        assert np.abs(p1 - p2)[mask].max() < 1e-12 * s0


@pytest.mark.parametrize("reg", [1, 2, 3, 4, 5])
def test_regularizations_converge_to_bingham(reg):
    """Each regularization tends to 2 sigma0 sign(E) (Eq. bingham1D) at fixed
    E != 0 as its parameter grows."""
    e = np.array([-0.3, -0.01, 0.02, 0.5])
    errs = []
    for g in (1e2, 1e3, 1e4, 1e5):
        prm = _prm(reg, s0=0.7, gamma=g, beta=g, m=g)
        errs.append(np.abs(np.sign(e) * C.phi(np.abs(e), prm) - 2 * 0.7 * np.sign(e)).max())
    assert errs[-1] < 1e-9
    assert all(errs[i + 1] <= errs[i] for i in range(len(errs) - 1))


@pytest.mark.parametrize("reg", [1, 2, 3, 4, 5])
def test_regularization_derivatives_match_fd(reg):
    prm = _prm(reg, s0=1.0, gamma=10.0, beta=1.0, m=10.0)
    s = np.linspace(1e-3, 0.4, 397)
    eps = 1e-7
    fd = (C.phi(s + eps, prm) - C.phi(s - eps, prm)) / (2 * eps)
    ds = C.dphi(s, prm)
    # skip the kinks of the C^0 bi-viscosity law
    mask = np.abs(10.0 * s - 1.0) > 1e-4 if reg == 5 else np.ones_like(s, bool)
    assert np.abs(fd - ds)[mask].max() < 1e-6
    # slope at zero: 2 gamma (regs 1, 2, 5), 2 sigma0 gamma (3), 2 sigma0 m (4)
    assert abs(C.dphi(np.array([0.0]), prm)[0] - 20.0) < 1e-12


def test_paper_figure_parameters_continuity():
    """Fig. regFunctions parameters (sigma0 = 1, gamma = 10, beta = 1): the
    three paper regularizations are continuous and odd and stay within
    [-2 sigma0, 2 sigma0]."""
    e = np.linspace(-0.5, 0.5, 2001)
    for reg in (1, 2, 3):
        prm = _prm(reg)
        sig = np.sign(e) * C.phi(np.abs(e), prm)
        assert np.abs(np.diff(sig)).max() < 0.02
        assert np.abs(sig + sig[::-1]).max() < 1e-12
        assert np.abs(sig).max() <= 2.0 + 1e-12


def test_yield_threshold_golden():
    """Eq. conditonTest2 closed form vs the paper's printed 9.0341."""
    with open(os.path.join(GOLDEN, "paper_values.json")) as f:
        gold = json.load(f)
    t = gold["yield_threshold_test2"]
    rho, g, a, h0, L = 1.0, 9.81, math.pi / 18, 3.0, 10.0
    val = rho * g * math.sin(a) * h0 * L / (2 * math.sqrt(2) * (h0 - 1))
    assert abs(val - t["value"]) < 0.5 * 10 ** (-t["digits"])


# ------------------------------------------------------------------ consistency (symbolic)

def _consistency(dim, p, ns, prm):
    import oracle_mms
    ex = oracle_mms.exact_rhs(dim, prm)
    out = []
    for n in ns:
        if dim == 1:
            coords, etov = synth.interval_mesh(n, 0, 1)
        else:
            coords, etov = synth.rect_tri_mesh(n, n, jitter=0.1, seed=2)
        xyz = node_coords(dim, coords, etov, p)
        X = [xyz[..., i] for i in range(dim)]
        bed = np.broadcast_to(ex["H"](*X), X[0].shape).astype(float)
        V = np.stack([ex["h"](*X)] + [np.broadcast_to(c(*X), X[0].shape) for c in ex["u"]])
        d = Discretization(dim, coords, etov, p, prm, bed_nodal=bed)
        dV, _ = d.rhs(d.to_modal(V))
        dq = d.eval_at_quad(dV)
        xq = d.map_to_phys(d.rq)
        Xq = [xq[..., i] for i in range(dim)]
        exq = [ex["ht"](*Xq)] + [c(*Xq) for c in ex["ut"]]
        out.append([math.sqrt(np.sum(d.wJ * (dq[f] - exq[f]) ** 2) / np.sum(d.wJ * exq[f] ** 2))
                    for f in range(dim + 1)])
    e = np.array(out)
    return np.log2(e[:-1] / e[1:]), e


@pytest.mark.parametrize("dim,p", [(1, 1), (1, 2), (1, 3), (2, 1), (2, 2)])
def test_consistency_inviscid(dim, p):
    """Inviscid flux, slope and bed source, HLL faces and the mass matrix:
    the discrete dV/dt of a smooth state converges to the exact one at rate p."""
    prm = synth.cases.default_params(reg=0, eta=0.0, sigma0=0.0, alpha=0.1)
    ns = (8, 16, 32) if dim == 1 else (4, 8, 16)
    rates, _ = _consistency(dim, p, ns, prm)
    assert rates[-1].min() > p - 0.2


@pytest.mark.parametrize("dim,p", [(1, 2), (1, 3), (2, 2), (2, 3)])
def test_consistency_viscous_bingham(dim, p):
    """With viscosity and the tanh Bingham law the stress divergence (E-step,
    Q and its central flux) converges at rate p - 1, the depth still at p."""
    prm = synth.cases.default_params(reg=3, eta=0.05, sigma0=0.1, gamma=5.0, alpha=0.1)
    ns = (8, 16, 32) if dim == 1 else ((4, 8, 16) if p == 2 else (4, 8))
    rates, _ = _consistency(dim, p, ns, prm)
    assert rates[-1][0] > p - 0.2
    assert rates[-1][1:].min() > p - 1 - 0.25


# ------------------------------------------------------------------ conservation, exact solution, order

def test_mass_conservation_walls():
    c = synth.radial_dam_2d(n=6, order=2, reg=1, sigma0=0.02, eta=0.01, gamma=10.0, beta=10.0)
    c.bcs = [([0, 2, 2, 0, 0, 0, 0], [0.0] * 7)]
    d, V0, _ = build(c)
    Vh = d.to_modal(V0)
    m0 = d.total_mass(Vh)
    for _ in range(10):
        Vh, _ = d.ssp_rk3_step(Vh)
    assert abs(d.total_mass(Vh) - m0) / m0 < 1e-13


@pytest.mark.slow
def test_newtonian_dam_break_vs_exact():
    """eta = sigma0 = 0: the DG solution converges in L1 to the exact wet-bed
    dam-break solution (the analytic reference of Sec. 6.3)."""
    errs = []
    for n in (50, 100, 200):
        c = synth.dam_break_1d(n_el=n, order=1, reg=0, eta=0.0, sigma0=0.0)
        d, V0, _ = build(c)
        Vh = d.to_modal(V0)
        t = 0.0
        while t < 0.1 - 1e-14:
            dt = min(d.stable_dt(Vh), 0.1 - t)
            Vh, _ = d.ssp_rk3_step(Vh, dt)
            t += dt
        Vq = d.eval_at_quad(Vh)
        xq = d.map_to_phys(d.rq)[..., 0]
        he, _ = riemann.sample(xq.ravel(), 0.1, 0.5, 1.0, 0.0, 0.5, 0.0, 9.81)
        errs.append(np.sum(d.wJ.ravel() * np.abs(Vq[0].ravel() - he)))
    rate = math.log2(errs[0] / errs[-1]) / 2
    assert errs[-1] < 2e-3 and rate > 0.8


def test_riemann_solver_jump_conditions():
    """The exact solver's star state satisfies the Rankine-Hugoniot relations
    of the right shock (mass and momentum) for the dam-break data."""
    g = 9.81
    hs, us = riemann.star_state(1.0, 0.0, 0.5, 0.0, g)
    s = us * hs / (hs - 0.5)  # mass jump
    mom_l = hs * us * us + 0.5 * g * hs * hs
    mom_r = 0.5 * g * 0.25
    assert abs(s * (hs * us - 0.0) - (mom_l - mom_r)) < 1e-10
    # Riemann invariant across the left rarefaction
    assert abs((us + 2 * math.sqrt(g * hs)) - 2 * math.sqrt(g * 1.0)) < 1e-10


def test_ssp_rk3_third_order_in_time():
    c = synth.dam_break_1d(n_el=10, order=2, reg=3, eta=0.02, sigma0=0.02, pap_m=1.0)
    c.params["gamma"] = 5.0
    h_fn, u_fn, _ = synth.random_smooth_fields(1, seed=7, h_amp=0.2, u_amp=0.3)
    c.h_fn, c.u_fn = h_fn, u_fn
    d, V0, _ = build(c)
    T = 4 * d.stable_dt(d.to_modal(V0))
    sols = []
    for n in (4, 8, 16):
        Vh = d.to_modal(V0)
        for _ in range(n):
            Vh, _ = d.ssp_rk3_step(Vh, T / n)
        sols.append(Vh)
    e1 = np.abs(sols[0] - sols[1]).max()
    e2 = np.abs(sols[1] - sols[2]).max()
    assert 2.7 < math.log2(e1 / e2) < 3.3
