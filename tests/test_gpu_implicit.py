"""GPU backward-Euler Newton (1D) vs the oracle's implicit integrator.

Newton is affine invariant, so the modal oracle and the nodal GPU path take
the same iterates; after each converged step both sit at round-off of the
same state.  States are compared at the nodes (relative L2, 1e-12 or 10x the
problem's rounding sensitivity), Newton iteration counts must match, and
the paper's yield-stress table is reproduced on the GPU too.
"""
import json
import os

import numpy as np
import pytest

import synth
from helpers import rel_l2
from oracle.implicit import Implicit1D
from oracle.run import build

pytestmark = pytest.mark.gpu
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _oracle_run(case, dt, n):
    d, V0, _ = build(case)
    im = Implicit1D(d, dt)
    Vh0 = d.to_modal(V0)
    X = im.pack(Vh0, im.initial_E(Vh0))
    its = []
    for _ in range(n):
        X, it, ok = im.step(X)
        its.append(it)
    Vh, Eh = im.unpack(X)
    return d, im, X, d.to_nodal(Vh), its


def _gpu(case, dt, n):
    import paper_2301_11238_gb300 as G
    s, V0 = G.implicit_from_case(case, dt=dt)
    its = []
    for _ in range(n):
        st = s.run(1)
        its.append(st["last_its"])
    V, E = s.get_state()
    return s, V, its


@pytest.mark.parametrize("p", [1, 2])
def test_lake_at_rest_gpu_implicit(p):
    c = synth.lake_at_rest_1d(n_el=60, order=p)
    import paper_2301_11238_gb300 as G
    s, V0 = G.implicit_from_case(c, dt=1e-2)
    st = s.run(5)
    V, _ = s.get_state()
    assert st["failed_steps"] == 0
    assert np.abs(V[1]).max() < 1e-12 and np.abs(V[0] - V0[0]).max() < 1e-12


def test_paper_dam_break_matches_oracle():
    c = synth.paper_dam_break_1d(n_el=100, order=1, m3=0, gamma=1e2, beta=1e2)
    d, im, X, Vo, its_o = _oracle_run(c, 1e-6, 20)
    s, V, its_g = _gpu(c, 1e-6, 20)
    assert its_g == its_o
    assert rel_l2(V, Vo) < 1e-12
    assert abs(s.active_percent() - im.active_percent(X)) < 1e-9


def test_yield_stress_gpu_matches_oracle_and_table():
    g3 = GOLD["yield_test_velocity_linf_reg3"]
    c = synth.parallel_surface_1d(n_el=100, order=1, reg=3, gamma=g3["gamma"][0], m3=1)
    d, im, X, Vo, its_o = _oracle_run(c, 0.1, 10)
    s, V, its_g = _gpu(c, 0.1, 10)
    # the relative stopping test can flip by one iteration at the round-off floor
    assert all(abs(a - b) <= 1 for a, b in zip(its_g, its_o))
    assert rel_l2(V, Vo) < 1e-10
    # L-infinity of u at the quadrature points, as in Table errorsEx2
    uq = np.einsum("qa,ka->kq", d.Phi, d.to_modal(V)[1])
    assert abs(np.abs(uq).max() / g3["linf_u"][0] - 1) < 0.15
    assert s.active_percent() == 0.0


@pytest.mark.parametrize("p,m3,reg,bc", [(2, 1, 3, "dirichlet"), (3, 2, 1, "copy"), (2, 2, 4, "wall"),
                                         (3, 0, 5, "copy")])
def test_random_smooth_states_match_oracle(p, m3, reg, bc):
    c = synth.paper_dam_break_1d(n_el=50, order=p, m3=m3, reg=reg, gamma=5.0, beta=5.0, sigma0=0.5,
                                 alpha=0.05)
    c.params["pap_m"] = 5.0
    h_fn, u_fn, b_fn = synth.random_smooth_fields(1, 17, h_amp=0.3, u_amp=0.5, bed_amp=0.1)
    c.h_fn, c.u_fn, c.bed_fn = h_fn, u_fn, b_fn
    if bc == "copy":
        c.bcs = [([0] * 7, [0.0] * 7)] * 2
    elif bc == "wall":
        c.bcs = [([0, 2, 0, 0, 0, 0, 0], [0.0] * 7)] * 2
    d, im, X, Vo, its_o = _oracle_run(c, 2e-4, 5)
    s, V, its_g = _gpu(c, 2e-4, 5)
    assert all(abs(a - b) <= 1 for a, b in zip(its_g, its_o))
    assert rel_l2(V, Vo) < 1e-11


def test_newton_failure_is_reported():
    import paper_2301_11238_gb300 as G
    c = synth.paper_dam_break_1d(n_el=40, order=1, m3=0)
    s, _ = G.implicit_from_case(c, dt=1e-3, max_it=1, on_fail_continue=False)
    with pytest.raises(G.DGError) as ei:
        s.run(3)
    assert ei.value.status == G.DG_ERR_NEWTON


def _gpu_mixed(case, dt, n):
    import paper_2301_11238_gb300 as G
    s, V0 = G.implicit_from_case(case, dt=dt, mixed=True)
    its = []
    for _ in range(n):
        its.append(s.run(1)["last_its"])
    V, _ = s.get_state()
    return s, V, its


def test_mixed_precision_solve_matches_oracle_dam_break():
    """FP32 block-Thomas factorization + two FP64 refinement rounds: the
    Newton iterates match the FP64 oracle's (iteration counts within one,
    states within 1e-12)."""
    c = synth.paper_dam_break_1d(n_el=100, order=1, m3=0, gamma=1e2, beta=1e2)
    d, im, X, Vo, its_o = _oracle_run(c, 1e-6, 20)
    s, V, its_g = _gpu_mixed(c, 1e-6, 20)
    assert all(abs(a - b) <= 1 for a, b in zip(its_g, its_o))
    assert rel_l2(V, Vo) < 1e-12


def test_mixed_precision_solve_yield_and_p2():
    c = synth.parallel_surface_1d(n_el=100, order=1, reg=3, gamma=1e3, m3=1)
    d, im, X, Vo, its_o = _oracle_run(c, 0.1, 10)
    s, V, its_g = _gpu_mixed(c, 0.1, 10)
    assert all(abs(a - b) <= 1 for a, b in zip(its_g, its_o))
    assert rel_l2(V, Vo) < 1e-10
    c2 = synth.paper_dam_break_1d(n_el=50, order=2, m3=1, reg=3, gamma=5.0, sigma0=0.5)
    h_fn, u_fn, _ = synth.random_smooth_fields(1, 19, h_amp=0.3, u_amp=0.5)
    c2.h_fn, c2.u_fn = h_fn, u_fn
    d, im, X, Vo, its_o = _oracle_run(c2, 2e-4, 5)
    s, V, its_g = _gpu_mixed(c2, 2e-4, 5)
    assert rel_l2(V, Vo) < 1e-11


@pytest.mark.parametrize("mixed", [False, True])
def test_gamma_continuation_matches_oracle(mixed):
    """Continuation gamma0 = 1e2 -> gamma = 1e3 in two stages per step
    (Sec. 6.3, Table damBreakContinuation setup): iteration counts (summed over
    stages) and states match the oracle."""
    import paper_2301_11238_gb300 as G
    c = synth.paper_dam_break_1d(n_el=100, order=1, m3=0, reg=1, gamma=1e3, beta=1e3)
    d, V0, _ = build(c)
    im = Implicit1D(d, 1e-6)
    Vh0 = d.to_modal(V0)
    X = im.pack(Vh0, im.initial_E(Vh0))
    its_o = []
    for _ in range(15):
        X, it, ok = im.step_continuation(X, 2, 1e2)
        its_o.append(it)
        assert ok
    Vo = d.to_nodal(im.unpack(X)[0])
    s, _ = G.implicit_from_case(c, dt=1e-6, n_gamma=2, gamma0=1e2, mixed=mixed)
    its_g = [s.run(1)["last_its"] for _ in range(15)]
    V, _ = s.get_state()
    assert all(abs(a - b) <= 1 for a, b in zip(its_g, its_o))
    assert rel_l2(V, Vo) < 1e-12


def test_paper_dam_break_active_region_table_damBreakFuns():
    """The paper's dam break run to t = 0.15 s (150,000 backward-Euler steps
    of 1e-6 s on 100 elements, regularization 1 with gamma = beta = 1e2):
    the active region and Newton iterations per step of Table damBreakFuns
    (about three minutes on the GPU)."""
    import paper_2301_11238_gb300 as G
    gold = GOLD["dam_break_active_percent_n100"]
    c = synth.paper_dam_break_1d(n_el=100, order=1, m3=0, reg=1, gamma=1e2, beta=1e2)
    s, _ = G.implicit_from_case(c, dt=1e-6, mixed=True)
    st = s.run(150000)
    assert st["failed_steps"] == 0 and abs(st["t"] - 0.15) < 1e-9
    assert abs(s.active_percent() - gold["reg1_gamma1e2_beta1e2"]) <= 1.0
    assert abs(st["newton_its"] / st["steps"] - gold["nr_its_per_step"]) < 0.5
