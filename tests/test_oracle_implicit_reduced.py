"""Pins of the reduced backward-Euler Newton oracle (E eliminated, any
dimension; oracle/implicit_reduced.py): it reproduces the paper's own 1D
monolithic Newton with the Appendix A tangent (Sec. 5.1), keeps the lake at
rest, conserves mass, and tends to the explicit Euler step as dt -> 0."""
import numpy as np
import pytest

import synth
from helpers import rel_l2, smooth_case
from oracle.implicit import Implicit1D
from oracle.implicit_reduced import ImplicitReduced
from oracle.run import build


@pytest.mark.parametrize("p,reg", [(1, 1), (2, 3), (1, 0)])
def test_matches_paper_monolithic_newton_1d(p, reg):
    """Same backward-Euler step two ways: the (V, E) Newton with the
    Appendix A Jacobian (analytic, pinned elsewhere against the paper's
    tables) and the reduced Newton with a finite-difference Jacobian."""
    c = synth.dam_break_1d(n_el=24, order=p, reg=reg, sigma0=0.05 if reg else 0.0, eta=0.01,
                           gamma=100.0, beta=100.0)
    d, V0, _ = build(c, m3=p)
    Vh = d.to_modal(V0)
    dt = 20 * d.stable_dt(Vh)
    ref = Implicit1D(d, dt)
    X, _, ok = ref.step(ref.pack(Vh, ref.initial_E(Vh)), max_it=20, rtol=1e-14, atol=1e-13)
    assert ok
    V_ref = ref.unpack(X)[0]
    V_red, its, res = ImplicitReduced(d, dt).step(Vh, max_it=20, rtol=1e-14, atol=1e-12)
    assert its >= 1
    assert rel_l2(V_red, V_ref) < 1e-10


def test_lake_at_rest_needs_no_iteration():
    c = smooth_case(2, 2, 3, n=5, seed=3)
    c.h_fn = lambda x, xc: 1.0 - c.bed_fn(x, xc) if c.bed_fn else np.ones(len(x))
    c.u_fn = lambda x, xc: np.zeros((len(x), 2))
    c.params["alpha"] = 0.0
    d, V0, _ = build(c)
    Vh = d.to_modal(V0)
    im = ImplicitReduced(d, 1e-3)
    V1, its, res = im.step(Vh, atol=1e-11)
    assert its == 0 and res < 1e-11
    assert np.array_equal(V1, Vh)


def test_mass_conserved_with_walls_2d():
    c = smooth_case(2, 1, 3, n=5, seed=4, bc="wall", sigma0=0.02, gamma=50.0)
    d, V0, _ = build(c)
    Vh = d.to_modal(V0)
    im = ImplicitReduced(d, 10 * d.stable_dt(Vh))
    m0 = d.total_mass(Vh)
    V2, its = im.run(Vh, 2, rtol=1e-13, atol=1e-11)
    assert max(its) <= 10
    assert abs(d.total_mass(V2) - m0) < 1e-11 * m0


def test_small_step_limit_is_explicit_euler():
    """V_BE(dt) - V_FE(dt) = O(dt^2): halving dt quarters the gap."""
    c = smooth_case(2, 1, 3, n=4, seed=6, sigma0=0.02, gamma=50.0)
    d, V0, _ = build(c)
    Vh = d.to_modal(V0)
    dV, _ = d.rhs(Vh)
    gaps = []
    for dt in (2e-5, 1e-5):
        V_be, _, _ = ImplicitReduced(d, dt).step(Vh, rtol=1e-14, atol=1e-12)
        gaps.append(np.linalg.norm(V_be - (Vh + dt * dV)))
    assert 3.3 < gaps[0] / gaps[1] < 4.7, gaps
