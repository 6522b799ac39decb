"""Herschel-Bulkley viscous part (dg_swe_params.flow_index, an extension the
paper's introduction cites) on the GPU against the oracle: residuals,
explicit runs, batches and the Newton-Krylov integrator, plus the argument
checks."""
import numpy as np
import pytest

import synth
from helpers import both, rel_l2, sensitivity, smooth_case
from oracle.implicit_reduced import ImplicitReduced
from oracle.run import residual_nodal, run_explicit

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _hb(c, n=0.5, floor=1e-3):
    c.params.update(flow_index=n, rate_floor=floor)
    return c


@pytest.mark.parametrize("dim,p,reg", [(1, 1, 0), (1, 3, 3), (2, 1, 1), (2, 2, 3), (2, 3, 5)])
def test_residual_matches_oracle(dim, p, reg):
    c = _hb(smooth_case(dim, p, reg, n=60 if dim == 1 else 8, seed=20 + p + 3 * reg), n=0.4, floor=1e-2)
    d, V0, _, s = both(c)
    dv_o, E_o = residual_nodal(d, V0)
    dv, E = s.residual(V0)
    sv, se = sensitivity(d, V0)
    assert rel_l2(dv.cpu().numpy(), dv_o) < max(1e-12, 10 * sv)
    assert rel_l2(E.cpu().numpy(), E_o) < max(1e-12, 10 * se)
    s.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_run_matches_oracle(prec, tol):
    c = _hb(synth.radial_dam_2d(n=10, order=2, reg=3, sigma0=0.05, gamma=50.0, eta=0.01))
    d, V0, _, s = both(c, precision=prec)
    Vo, dts, t = run_explicit(d, V0, 25)
    s.set_state(V0)
    st = s.run(25)
    V, _ = s.get_state()
    assert abs(st["t"] - t) <= 1e-6 * t if prec else abs(st["t"] - t) <= 1e-12 * t
    assert rel_l2(V, Vo) < tol
    s.close()


def test_batch_bitwise_equals_solo():
    import paper_2301_11238_gb300 as G
    cases = [_hb(synth.dam_break_1d(n_el=50, order=2, reg=1, sigma0=0.05)),
             _hb(synth.radial_dam_2d(n=6, order=3, reg=2, sigma0=0.1), n=0.7),
             synth.radial_dam_2d(n=6, order=2, reg=1, sigma0=0.02)]
    B, _ = G.batch_from_cases(cases)
    B.run(10)
    for i, c in enumerate(cases):
        s, _, _ = G.solver_from_case(c)
        s.run(10)
        assert np.array_equal(B.get_state(i), s.get_state(with_E=False)), i
        s.close()
    B.close()


def test_newton_krylov_matches_reduced_oracle():
    import paper_2301_11238_gb300 as G
    c = _hb(synth.radial_dam_2d(n=7, order=1, reg=3, sigma0=0.02, gamma=50.0, eta=0.01), n=0.6, floor=1e-2)
    d, V0, _, s = both(c)
    Vh = d.to_modal(V0)
    dt = 10 * d.stable_dt(Vh)
    Vo, _ = ImplicitReduced(d, dt).run(Vh, 2, rtol=1e-14, atol=1e-11)
    s.set_state(V0)
    nk = G.Newton(s, dt, rtol=1e-13, atol=1e-11, krylov_dim=64, krylov_rtol=1e-11)
    st = nk.run(2)
    assert st["failed_steps"] == 0
    assert rel_l2(s.get_state(with_E=False), d.to_nodal(Vo)) < 1e-9
    nk.close()
    s.close()


def test_argument_checks():
    import paper_2301_11238_gb300 as G
    for n, floor in ((1.5, 1e-3), (-0.5, 1e-3), (0.5, 0.0)):
        c = _hb(synth.radial_dam_2d(n=3, order=1), n=n, floor=floor)
        with pytest.raises(G.DGError) as ei:
            G.solver_from_case(c)
        assert ei.value.status == G.DG_ERR_ARG
    c = _hb(synth.paper_dam_break_1d(n_el=20, order=1, m3=0))
    with pytest.raises(G.DGError) as ei:
        G.implicit_from_case(c, dt=1e-6)
    assert ei.value.status == G.DG_ERR_UNSUPPORTED
