"""Backward Euler with the Jacobian-free Newton-Krylov solve on the GPU
(include/dg_newton.h) against the oracles: the reduced Newton with E
eliminated (oracle/implicit_reduced.py) in 1D and 2D and the paper's own
monolithic 1D Newton with the Appendix A tangent.  Converged backward-Euler
states are unique, so both sides agree to the Newton tolerances."""
import numpy as np
import pytest

import synth
from helpers import both, rel_l2, smooth_case
from oracle.implicit import Implicit1D
from oracle.implicit_reduced import ImplicitReduced

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _gpu_run(s, V0, dt, steps, **kw):
    import paper_2301_11238_gb300 as G
    s.set_state(V0)
    nk = G.Newton(s, dt, rtol=1e-13, atol=1e-11, krylov_dim=64, krylov_rtol=1e-11, **kw)
    st = nk.run(steps)
    V = s.get_state(with_E=False)
    nk.close()
    return V, st


@pytest.mark.parametrize("p,reg,fac", [(1, 3, 10.0), (2, 0, 30.0)])
def test_2d_matches_reduced_oracle(p, reg, fac):
    """162 triangles (one 128-element tile and a ragged tail), two steps of
    10-30 times the explicit step."""
    c = synth.radial_dam_2d(n=9, order=p, reg=reg, sigma0=0.02 if reg else 0.0, gamma=50.0, eta=0.01)
    d, V0, _, s = both(c)
    Vh = d.to_modal(V0)
    dt = fac * d.stable_dt(Vh)
    Vo, its = ImplicitReduced(d, dt).run(Vh, 2, rtol=1e-14, atol=1e-11)
    V, st = _gpu_run(s, V0, dt, 2)
    assert st["steps"] == 2 and st["failed_steps"] == 0 and st["krylov_its"] > 0
    assert abs(st["t"] - 2 * dt) < 1e-15
    assert rel_l2(V, d.to_nodal(Vo)) < 1e-9, rel_l2(V, d.to_nodal(Vo))
    s.close()


def test_1d_matches_paper_monolithic_newton():
    c = synth.dam_break_1d(n_el=150, order=1, reg=1, sigma0=0.05, eta=0.01, gamma=100.0, beta=100.0)
    d, V0, _, s = both(c)
    Vh = d.to_modal(V0)
    dt = 20 * d.stable_dt(Vh)
    ref = Implicit1D(d, dt)
    X = ref.pack(Vh, ref.initial_E(Vh))
    for _ in range(2):
        X, _, ok = ref.step(X, max_it=20, rtol=1e-14, atol=1e-12)
        assert ok
    V, st = _gpu_run(s, V0, dt, 2)
    assert rel_l2(V, d.to_nodal(ref.unpack(X)[0])) < 1e-9
    s.close()


def test_lake_at_rest_and_mass():
    import paper_2301_11238_gb300 as G
    c = smooth_case(2, 2, 3, n=6, seed=3)
    c.h_fn = lambda x, xc: 1.0 - c.bed_fn(x, xc)
    c.u_fn = lambda x, xc: np.zeros((len(x), 2))
    c.params["alpha"] = 0.0
    d, V0, _, s = both(c)
    V, st = _gpu_run(s, V0, 1e-3, 3)
    assert st["newton_its"] == 0
    assert np.array_equal(V, V0)
    s.close()
    w = smooth_case(2, 1, 3, n=9, seed=4, bc="wall", sigma0=0.02, gamma=50.0)
    d, V0, _, s = both(w)
    s.set_state(V0)
    m0 = s.sync()["mass"]
    V, st = _gpu_run(s, V0, 10 * d.stable_dt(d.to_modal(V0)), 3)
    assert abs(s.sync()["mass"] - m0) < 1e-11 * m0
    s.close()


def test_rejects_fp32_and_bad_parameters():
    import paper_2301_11238_gb300 as G
    c = synth.radial_dam_2d(n=4, order=1)
    s32, _, _ = G.solver_from_case(c, precision=G.PREC_FP32)
    with pytest.raises(G.DGError) as ei:
        G.Newton(s32, 1e-4)
    assert ei.value.status == G.DG_ERR_UNSUPPORTED
    s64, _, _ = G.solver_from_case(c)
    for kw in (dict(dt=-1.0), dict(dt=1e-4, krylov_dim=0), dict(dt=1e-4, krylov_dim=65),
               dict(dt=1e-4, krylov_rtol=1.5), dict(dt=1e-4, max_newton=0)):
        with pytest.raises(G.DGError) as ei:
            G.Newton(s64, **kw)
        assert ei.value.status == G.DG_ERR_ARG
    s32.close()
    s64.close()


def test_unconverged_step_is_reported():
    import paper_2301_11238_gb300 as G
    c = synth.radial_dam_2d(n=6, order=1, reg=3, sigma0=0.02, gamma=50.0)
    s, V0, _ = G.solver_from_case(c)
    nk = G.Newton(s, 1e-5, max_newton=1, rtol=1e-14, atol=0.0, krylov_dim=8, on_fail_continue=0)
    with pytest.raises(G.DGError) as ei:
        nk.run(1)
    assert ei.value.status == G.DG_ERR_NEWTON
    nk.close()
    s.close()
