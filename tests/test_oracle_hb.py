"""Herschel-Bulkley extension of the oracle's constitutive law (the paper's
introduction cites the law; its scheme is Bingham): the power-law viscous
part eta max(s, rate_floor)^(n - 1)."""
import numpy as np
import pytest

import synth
from synth.cases import default_params
from oracle import constitutive as C
from oracle.run import build


def _prm(**kw):
    p = default_params(reg=0, sigma0=0.0, eta=0.05)
    p.update(kw)
    return p


def test_flow_index_one_is_the_papers_law_bit_for_bit():
    rng = np.random.default_rng(0)
    E2 = rng.standard_normal((4, 50))
    E1 = rng.standard_normal((1, 50))
    for reg in (1, 2, 3):
        base = _prm(reg=reg, sigma0=0.3, gamma=20.0, beta=20.0)
        hb1 = dict(base, flow_index=1.0, rate_floor=1e-3)
        assert np.array_equal(C.stress(E2, 2, base), C.stress(E2, 2, hb1))
        assert np.array_equal(C.stress(E1, 1, base), C.stress(E1, 1, hb1))


@pytest.mark.parametrize("n", [0.3, 0.5, 0.8])
def test_power_law_is_homogeneous_of_degree_n(n):
    """sigma0 = 0: sigma(lambda E) = lambda^n sigma(E) above the rate floor
    (1D and 2D), the defining scaling of a power-law fluid."""
    prm = _prm(flow_index=n, rate_floor=1e-4)
    rng = np.random.default_rng(1)
    E = rng.uniform(0.1, 2.0, (4, 40)) * np.sign(rng.standard_normal((4, 40)))
    for lam in (0.5, 3.0, 17.0):
        assert np.allclose(C.stress(lam * E, 2, prm), lam ** n * C.stress(E, 2, prm), rtol=1e-13)
        assert np.allclose(C.stress(lam * E[:1], 1, prm), lam ** n * C.stress(E[:1], 1, prm), rtol=1e-13)


def test_continuous_at_the_floor_and_linear_below():
    prm = _prm(flow_index=0.4, rate_floor=2e-2)
    f = prm["rate_floor"]
    e = np.array([[f * (1 - 1e-12), f, f * (1 + 1e-12)]])
    s = C.stress(e, 1, prm)[0, 0]
    assert np.ptp(s) < 1e-12
    below = np.array([[0.25 * f, 0.5 * f]])
    sb = C.stress(below, 1, prm)[0, 0]
    assert abs(sb[1] / sb[0] - 2.0) < 1e-13


def test_2d_law_reduces_to_1d():
    prm = _prm(reg=3, sigma0=0.2, gamma=30.0, flow_index=0.6, rate_floor=1e-3)
    e = np.linspace(-2.0, 2.0, 41)
    E2 = np.zeros((4, e.size))
    E2[0] = e
    s1 = C.stress(e[None], 1, prm)[0, 0]
    s2 = C.stress(E2, 2, prm)
    # 1D: sigma = mu 2 E ; 2D with D = diag(E, 0): sigma_11 = mu (2 E), sigma_22 = mu E
    assert np.allclose(s2[0, 0], s1, rtol=1e-13, atol=1e-15)
    assert np.allclose(s2[1, 1], 0.5 * s1, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("n", [0.3, 0.7])
def test_step_bound_slope_is_the_largest_slope(n):
    """max_viscosity: the largest d sigma_N / dE over E (divided by 4), found
    by differencing the 1D law on a fine grid."""
    prm = _prm(flow_index=n, rate_floor=1e-2)
    e = np.linspace(0.0, 1.0, 200001)
    sig = C.stress(e[None], 1, prm)[0, 0]
    slope = np.diff(sig) / np.diff(e)
    assert abs(slope.max() / 4.0 - C.max_viscosity(prm)) < 1e-6 * C.max_viscosity(prm)


def test_lake_at_rest_and_mass_with_power_law():
    c = synth.bump_dam_2d(n=6, order=2, flow_index=0.5, rate_floor=1e-3)
    c.h_fn = lambda x, xc=None, b=c.bed_fn: 1.0 - b(x)
    d, V0, _ = build(c)
    dV, _ = d.rhs(d.to_modal(V0))
    assert np.abs(dV).max() < 1e-11
    c2 = synth.dam_break_1d(n_el=30, order=2, reg=3, sigma0=0.05, gamma=50.0, flow_index=0.5, rate_floor=1e-3)
    d2, V2, _ = build(c2)
    Vh = d2.to_modal(V2)
    m0 = d2.total_mass(Vh)
    for _ in range(20):
        Vh, _ = d2.ssp_rk3_step(Vh)
    assert abs(d2.total_mass(Vh) - m0) < 1e-13 * m0
