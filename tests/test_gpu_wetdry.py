"""Wet/dry mode (dg_swe_params.positivity, an extension for wet/dry fronts:
explicit stages on the conservative moments <N, U> with the depth limiter)
on the GPU against the oracle: dam breaks onto a 1 : 0.03 bed and onto a dry
bed (Ritter), which the primitive-variable stages cannot run, in 1D and 2D,
solo and batched, FP64, FP32 and the tensor-core volume pass."""

import numpy as np
import pytest

import synth
from helpers import both, rel_l2
from oracle import riemann
from oracle.run import run_explicit

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _case(dim, p):
    if dim == 1:
        return synth.dam_break_1d(n_el=100, order=p, hl=1.0, hr=0.03, reg=0, sigma0=0.0, eta=0.0, positivity=1)
    return synth.radial_dam_2d(n=12, order=p, reg=0, sigma0=0.0, eta=0.0, h_in=1.0, h_out=0.03, positivity=1)


def _limiter_active(d, V0, steps):
    """The oracle with and without the limiter must differ, or the case would
    not exercise it."""
    d.prm["positivity"] = 0
    try:
        Vu, _, _ = run_explicit(d, V0, steps)
    except (np.linalg.LinAlgError, FloatingPointError):
        return True
    finally:
        d.prm["positivity"] = 1
    Vl, _, _ = run_explicit(d, V0, steps)
    return not np.all(np.isfinite(Vu)) or rel_l2(Vu, Vl) > 1e-10


@pytest.mark.parametrize("dim,p,steps", [(1, 1, 40), (2, 1, 30), (2, 2, 4)])
def test_limited_dam_break_matches_oracle(dim, p, steps):
    c = _case(dim, p)
    d, V0, _, s = both(c)
    with np.errstate(all="ignore"):
        assert _limiter_active(d, V0, steps)
    Vo, dts, t = run_explicit(d, V0, steps)
    s.set_state(V0)
    st = s.run(steps)
    V, _ = s.get_state()
    assert abs(st["t"] - t) <= 1e-12 * t
    assert rel_l2(V, Vo) < 1e-12
    pts = d.check_points(d.to_modal(V)[0])
    assert pts.min() >= -1e-13
    s.close()


def test_limited_batch_bitwise_equals_solo_and_fp32_close():
    import paper_2301_11238_gb300 as G
    cases = [_case(1, 1), _case(2, 1), synth.radial_dam_2d(n=6, order=2, reg=1, sigma0=0.02)]
    B, _ = G.batch_from_cases(cases)
    B.run(15)
    B32, _ = G.batch_from_cases(cases, precision=G.PREC_FP32)
    B32.run(15)
    for i, c in enumerate(cases):
        s, V0, _ = G.solver_from_case(c)
        s.run(15)
        V = s.get_state(with_E=False)
        assert np.array_equal(B.get_state(i), V), i
        assert rel_l2(B32.get_state(i), V) < 1e-4, i
        s.close()
    B.close()
    B32.close()


def _dry_x_dam_2d(n=20, p=1):
    return synth.dry_dam_2d(n=n, order=p)


def test_ritter_dry_bed_1d_matches_oracle_and_exact():
    """Dam break onto a dry bed (depth exactly 0), p = 1, 200 elements, 700
    CFL steps (t about 0.049): the GPU state equals the oracle's to 1e-12
    relative L2 with the same time, the depth is non-negative, mass is
    conserved to round-off, and the L1 depth error against Ritter's exact
    solution is below 1.8e-3 (the oracle measures 1.5e-3 at t = 0.05)."""
    c = synth.dam_break_1d(n_el=200, order=1, hl=1.0, hr=0.0, x_dam=0.5, reg=0, sigma0=0.0, eta=0.0,
                           positivity=1)
    d, V0, _, s = both(c)
    Vo, _, t = run_explicit(d, V0, 700)
    s.set_state(V0)
    st = s.run(700)
    V, _ = s.get_state()
    s.close()
    assert abs(st["t"] - t) <= 1e-12 * t
    assert rel_l2(V, Vo) < 1e-12
    Vh = d.to_modal(V)
    assert d.check_points(Vh[0]).min() >= -1e-13
    assert abs(st["mass"] - st["mass0"]) <= 1e-13 * st["mass0"]
    xq = d.map_to_phys(d.rq)[:, :, 0]
    hq = np.einsum("qa,ka->kq", d.Phi, Vh[0])
    he, _ = riemann.ritter(xq.ravel(), st["t"], 0.5, 1.0, 9.81)
    assert float(np.sum(d.wJ * np.abs(hq - he.reshape(hq.shape)))) < 1.8e-3


def test_ritter_dry_bed_2d_matches_oracle():
    """The dry-bed dam break on 20 x 20 x 2 triangles, p = 1, 40 steps:
    FP64 GPU = oracle to 1e-12, depth non-negative, mass conserved."""
    c = _dry_x_dam_2d()
    d, V0, _, s = both(c)
    Vo, _, t = run_explicit(d, V0, 40)
    s.set_state(V0)
    st = s.run(40)
    V, _ = s.get_state()
    s.close()
    assert abs(st["t"] - t) <= 1e-12 * t
    assert rel_l2(V, Vo) < 1e-12
    assert d.check_points(d.to_modal(V)[0]).min() >= -1e-13
    assert abs(st["mass"] - st["mass0"]) <= 1e-13 * st["mass0"]


def test_dry_bed_batch_fp32_close_to_fp64():
    """Dry beds in a batch next to a wet instance: the FP64 batch equals the
    solo runs bit for bit, and the FP32 batch (whose wet/dry stages also run
    in FP64 from FP32 inputs) stays within 1e-4 of it after 60 steps."""
    import paper_2301_11238_gb300 as G
    cases = [synth.dam_break_1d(n_el=120, order=1, hl=1.0, hr=0.0, reg=0, sigma0=0.0, eta=0.0, positivity=1),
             _dry_x_dam_2d(n=12), synth.radial_dam_2d(n=6, order=2, reg=1, sigma0=0.02)]
    B, _ = G.batch_from_cases(cases)
    B.run(60)
    B32, _ = G.batch_from_cases(cases, precision=G.PREC_FP32)
    B32.run(60)
    for i, c in enumerate(cases):
        s, V0, _ = G.solver_from_case(c)
        s.run(60)
        V = s.get_state(with_E=False)
        assert np.array_equal(B.get_state(i), V), i
        assert rel_l2(B32.get_state(i), V) < 1e-4, (i, rel_l2(B32.get_state(i), V))
        s.close()
    B.close()
    B32.close()


def test_wet_dry_stage_in_tensor_core_pass():
    """The tensor-core volume pass (FP32 contexts, p >= 2) takes the same
    wet/dry stage: the 2D 1 : 0.03 dam break at p = 2, 4 steps, within the
    FP32 tolerance of the oracle."""
    import paper_2301_11238_gb300 as G
    c = _case(2, 2)
    d, V0, _, s = both(c, precision=G.PREC_FP32_TC)
    Vo, _, t = run_explicit(d, V0, 4)
    s.set_state(V0)
    st = s.run(4)
    V, _ = s.get_state()
    s.close()
    assert abs(st["t"] - t) <= 1e-6 * t
    assert rel_l2(V, Vo) < 1e-5


def test_wet_dry_groups_and_launch_count():
    """Wet/dry instances form groups of their own (a wet instance of the same
    dimension and order stays in a group without the stage kernel): 14
    launches per wet/dry group and step, 11 per other group; the persistent
    step, which has no wet/dry stage, is refused with DG_ERR_UNSUPPORTED."""
    import paper_2301_11238_gb300 as G
    wet = synth.dam_break_1d(n_el=50, order=1, reg=0, sigma0=0.0, eta=0.0)
    dry = synth.dam_break_1d(n_el=50, order=1, hl=1.0, hr=0.0, reg=0, sigma0=0.0, eta=0.0, positivity=1)
    B, _ = G.batch_from_cases([wet, dry])
    assert B.info()["groups"] == 2
    assert B.launches_per_step() == 11 + 14
    with pytest.raises(G.DGError) as ei:
        B.set_persistent(True)
    assert ei.value.status == G.DG_ERR_UNSUPPORTED
    B.run(5)
    s, _, _ = G.solver_from_case(dry)
    assert s.launches_per_step() == 14
    s.run(5)
    assert np.array_equal(B.get_state(1), s.get_state(with_E=False))
    s.close()
    B.close()
