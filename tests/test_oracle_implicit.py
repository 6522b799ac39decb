"""Pins of the oracle's backward-Euler Newton integrator (Sec. 5.1, App. A).

* The Appendix A Jacobian (HLL wave speeds held fixed) equals the finite
  difference of the residual taken with the same fixed speeds.
* Lake at rest (Sec. 6.1) is an exact equilibrium of the implicit scheme.
* Yield stress above the driving stress (Sec. 6.2, sigma0 = 9.035): the
  material creeps with a velocity of order 1/gamma; the L-infinity velocity
  reproduces Table errorsEx2 (regularization 3: 1.6e-3 at gamma = 1e3,
  1.6e-4 at gamma = 1e4; regularization 1: 1.3e-2), and nothing is active.
* Newton converges quadratically on a dam break (Sec. 6.3 setup).
* Backward Euler agrees with SSP-RK3 to first order in dt (same spatial
  operator).
* With reflecting walls the implicit scheme conserves mass to the Newton
  tolerance.
"""
import json
import math
import os
import warnings

import numpy as np
import pytest

import synth
from oracle.implicit import Implicit1D
from oracle.run import build

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.mark.parametrize("p,m3,reg", [(1, 1, 1), (2, 0, 3), (3, 2, 2), (1, 0, 4), (2, 2, 5)])
def test_jacobian_matches_finite_differences(p, m3, reg):
    c = synth.paper_dam_break_1d(n_el=6, order=p, m3=m3, reg=reg, gamma=3.0, beta=5.0, sigma0=0.5, alpha=0.1)
    c.params["pap_m"] = 3.0
    h_fn, u_fn, b_fn = synth.random_smooth_fields(1, 3, h_amp=0.3, u_amp=1.0, bed_amp=0.1)
    c.h_fn, c.u_fn, c.bed_fn = h_fn, u_fn, b_fn
    d, V0, _ = build(c)
    im = Implicit1D(d, 1e-2)
    Vh = d.to_modal(V0)
    X = im.pack(Vh, im.initial_E(Vh)) + 0.05 * np.random.default_rng(1).standard_normal((d.K, im.nb))
    Uold = im.old_term(Vh)
    Vm, Vp, _, _ = im.face_states(*im.unpack(X))
    spd = im.speeds(Vm, Vp, d.n[:, :, 0])
    J = im.jacobian(X)
    eps = 1e-6
    Jfd = np.zeros_like(J)
    for j in range(X.size):
        xp = X.ravel().copy()
        xm = X.ravel().copy()
        xp[j] += eps
        xm[j] -= eps
        Jfd[:, j] = (im.residual(xp.reshape(X.shape), Uold, spd)
                     - im.residual(xm.reshape(X.shape), Uold, spd)).ravel() / (2 * eps)
    assert np.abs(J - Jfd).max() < 1e-8 * np.abs(J).max()


@pytest.mark.parametrize("eta,sigma0", [(0.0, 0.0), (1.0, 1.0)])
def test_lake_at_rest_implicit(eta, sigma0):
    c = synth.lake_at_rest_1d(n_el=40, order=2, eta=eta, sigma0=sigma0)
    d, V0, _ = build(c)
    im = Implicit1D(d, 1e-2)
    X, its, fails = im.run(d.to_modal(V0), 5)
    Vh, _ = im.unpack(X)
    Vn = d.to_nodal(Vh)
    assert fails == 0
    assert np.abs(Vn[1]).max() < 1e-12
    assert np.abs(Vn[0] - V0[0]).max() < 1e-12


def _yield(reg, gamma, beta=1e3):
    c = synth.parallel_surface_1d(n_el=100, order=1, reg=reg, gamma=gamma, beta=beta, m3=1)
    d, V0, _ = build(c)
    im = Implicit1D(d, 0.1)
    X, its, fails = im.run(d.to_modal(V0), 10)
    Vh, _ = im.unpack(X)
    return np.abs(d.eval_at_quad(Vh)[1]).max(), im.active_percent(X), fails


def test_yield_stress_keeps_material_nearly_at_rest_table_errorsEx2():
    g3 = GOLD["yield_test_velocity_linf_reg3"]
    g1 = GOLD["yield_test_velocity_linf_reg1"]
    u3a, act3a, f1 = _yield(3, g3["gamma"][0])
    u3b, act3b, f2 = _yield(3, g3["gamma"][1])
    u1, act1, f3 = _yield(1, g1["gamma"][0], g1["beta"][0])
    assert f1 == f2 == f3 == 0
    # within 15 % of the printed two-digit values
    assert abs(u3a / g3["linf_u"][0] - 1) < 0.15
    assert abs(u3b / g3["linf_u"][1] - 1) < 0.15
    assert abs(u1 / g1["linf_u"][0] - 1) < 0.15
    # velocity scales like 1/gamma
    assert 9.0 < u3a / u3b < 11.0
    assert act3a == act3b == act1 == GOLD["yield_test_active_percent"]["value"]


def test_newton_quadratic_convergence_dam_break():
    c = synth.paper_dam_break_1d(n_el=40, order=1, m3=0, gamma=1e2, beta=1e2)
    d, V0, _ = build(c)
    im = Implicit1D(d, 1e-6)  # the paper's step for this problem (Sec. 6.3)
    Vh = d.to_modal(V0)
    X = im.pack(Vh, im.initial_E(Vh))
    Uold = im.old_term(Vh)
    norms = [np.linalg.norm(im.residual(X, Uold))]
    for _ in range(4):
        dx = np.linalg.solve(im.jacobian(X), -im.residual(X, Uold).ravel()).reshape(X.shape)
        X = X + dx
        norms.append(np.linalg.norm(im.residual(X, Uold)))
    # quadratic phase: each residual at most a constant times the square of the previous
    ratios = [norms[i + 1] / norms[i] ** 2 for i in range(1, 3) if norms[i] > 1e-10]
    assert norms[3] < 1e-9 * norms[0]
    assert all(r < 1e3 for r in ratios)


def test_implicit_matches_explicit_first_order():
    c = synth.dam_break_1d(n_el=20, order=2, reg=3, sigma0=0.05, eta=0.05)
    c.params["gamma"] = 5.0
    h_fn, u_fn, _ = synth.random_smooth_fields(1, 11, h_amp=0.2, u_amp=0.3)
    c.h_fn, c.u_fn = h_fn, u_fn
    d, V0, _ = build(c)
    Vh0 = d.to_modal(V0)
    T = 4e-3
    ref = Vh0.copy()
    n_ref = 200
    for _ in range(n_ref):
        ref, _ = d.ssp_rk3_step(ref, T / n_ref)
    errs = []
    for n in (4, 8, 16):
        im = Implicit1D(d, T / n)
        X, _, _ = im.run(Vh0, n, rtol=1e-13, atol=1e-14)
        Vh, _ = im.unpack(X)
        errs.append(np.abs(Vh - ref).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(0.8 < r < 1.3 for r in rates)


def test_implicit_mass_conservation_walls():
    c = synth.paper_dam_break_1d(n_el=30, order=2, m3=2)
    c.bcs = [([0, 2, 0, 0, 0, 0, 0], [0.0] * 7)] * 2
    d, V0, _ = build(c)
    im = Implicit1D(d, 1e-6)
    Vh0 = d.to_modal(V0)
    m0 = d.total_mass(Vh0)
    X, _, fails = im.run(Vh0, 10)
    Vh, _ = im.unpack(X)
    assert fails == 0
    assert abs(d.total_mass(Vh) - m0) < 1e-12 * m0


def test_gamma_continuation_converges_to_final_gamma():
    """Continuation (Sec. 6.3) ends each step at the target gamma: one step
    with gamma0 -> gamma equals a plain step at gamma to the Newton
    tolerance, and takes at least as many iterations in total."""
    c = synth.paper_dam_break_1d(n_el=40, order=1, m3=0, reg=1, gamma=1e3, beta=1e3)
    d, V0, _ = build(c)
    im = Implicit1D(d, 1e-6)
    Vh0 = d.to_modal(V0)
    X0 = im.pack(Vh0, im.initial_E(Vh0))
    Xa, ita, oka = im.step(X0)
    Xb, itb, okb = im.step_continuation(X0, 3, 1e2)
    assert oka and okb and itb >= ita
    assert np.abs(Xa - Xb).max() < 1e-9 * np.abs(Xa).max()
    assert im.prm["gamma"] == 1e3  # restored after the stages
