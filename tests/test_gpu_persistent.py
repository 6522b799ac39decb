"""Persistent batch step (dg_batch_set_persistent: one launch per group and
step, work items claimed from a counter, per-instance phase counters) against
the graph form's 11 launches per group and step.

The per-element and per-face-point arithmetic is shared, but it is compiled
into a different kernel, where the compiler may fuse some multiply-adds
differently (measured: 1.8e-16 relative after 12 steps in FP64), so FP64
states agree to 1e-13 relative and times to 1e-14, step counts exactly;
FP32 states to 1e-6 (FP32 rounding: measured 9e-8).  Cases: 1D
and 2D groups of every order with beds, walls and Dirichlet boundaries; a
group whose instance has more tiles than the grid has blocks (blocks claim
many items); the nine-instance radial sweep; and one instance against the
oracle."""
import numpy as np
import pytest

import synth
from helpers import rel_l2, smooth_case
from oracle.run import build as oracle_build, run_explicit

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _mixed_cases():
    return [synth.dam_break_1d(n_el=70, order=1),
            synth.radial_dam_2d(n=10, order=2, reg=1, sigma0=0.02),
            synth.radial_dam_2d(n=7, order=2, reg=3, sigma0=0.1, gamma=50.0),
            smooth_case(1, 3, 2, n=40, seed=5, bc="dirichlet"),
            smooth_case(2, 1, 5, n=6, seed=6, bc="wall"),
            synth.bump_dam_2d(n=6, order=3)]


def _run(cases, precision, persistent, steps):
    import paper_2301_11238_gb300 as G
    B, _ = G.batch_from_cases(cases, precision=precision)
    if persistent:
        B.set_persistent(True)
    st = B.run(steps)
    out = [B.get_state(i) for i in range(len(cases))]
    B.close()
    return out, st


@pytest.mark.parametrize("prec", [0, 1])
def test_persistent_equals_graph_mixed_groups(prec):
    cases = _mixed_cases()
    ref, st_ref = _run(cases, prec, False, 12)
    got, st = _run(cases, prec, True, 12)
    for i in range(len(cases)):
        if prec == 0:
            assert rel_l2(got[i], ref[i]) < 1e-13, (i, rel_l2(got[i], ref[i]))
            assert abs(st[i]["t"] - st_ref[i]["t"]) <= 1e-14 * st_ref[i]["t"] and st[i]["steps"] == 12
        else:
            assert rel_l2(got[i], ref[i]) < 1e-6, (i, rel_l2(got[i], ref[i]))
        assert st[i]["status"] == 0


def test_persistent_many_items_per_block():
    """A 32,768-triangle instance (256 element tiles and 1,536 face-point
    tiles per phase) next to two small ones."""
    cases = [synth.radial_dam_2d(n=128, order=2, reg=1, sigma0=0.02), synth.dam_break_1d(n_el=30, order=2),
             synth.radial_dam_2d(n=5, order=1)]
    ref, _ = _run(cases, 0, False, 5)
    got, _ = _run(cases, 0, True, 5)
    for i in range(len(cases)):
        assert rel_l2(got[i], ref[i]) < 1e-13, (i, rel_l2(got[i], ref[i]))


def test_persistent_radial_sweep_and_oracle():
    import paper_2301_11238_gb300 as G
    cases = [synth.radial_dam_2d(n=16, order=2, reg=reg, sigma0=s0, eta=0.01, gamma=1e3, beta=1e3)
             for s0 in (0.0, 0.02, 0.1) for reg in (1, 2, 3)]
    ref, _ = _run(cases, 0, False, 8)
    got, st = _run(cases, 0, True, 8)
    for i in range(len(cases)):
        assert rel_l2(got[i], ref[i]) < 1e-13, i
    d, V0, _ = oracle_build(cases[4])
    Vo, _, t = run_explicit(d, V0, 8)
    assert abs(st[4]["t"] - t) < 1e-12 * t
    assert rel_l2(got[4], Vo) < 1e-12


def test_persistent_rejected_for_tensor_core_batches():
    import paper_2301_11238_gb300 as G
    B, _ = G.batch_from_cases([synth.radial_dam_2d(n=4, order=2)], precision=G.PREC_FP32_TC)
    with pytest.raises(G.DGError) as ei:
        B.set_persistent(True)
    assert ei.value.status == G.DG_ERR_UNSUPPORTED
    B.close()
