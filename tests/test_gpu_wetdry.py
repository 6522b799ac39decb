"""Depth limiter (dg_swe_params.positivity, an extension for wet/dry fronts)
on the GPU against the oracle's positivity_limit: a dam break with depth
ratio 1 : 0.03 that the unlimited scheme cannot run, in 1D and 2D, solo and
batched, FP64 and FP32."""
import numpy as np
import pytest

import synth
from helpers import both, rel_l2
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
