"""Near-dry states in FP32 contexts against the FP64 oracle.

An FP32 element whose smallest nodal depth is below h_dry = 1000 h_floor
(1e-3 for the default floor 1e-6) assembles and solves its h-weighted mass
matrix in FP64 (dg_kernels.cuh: mass_solve_dispatch).  The cases put nodal depths between the floor and 1e-2:
  * a thin film (depth 1e-6 .. 5e-3) with a rotating velocity over a bed,
    tanh Bingham law, single residual, 1D and 2D, p = 1..3, at the FP32
    tolerance max(1e-5, 10 x the response to 2^-24 input rounding);
  * the dam break over the Gaussian bump with the downstream surface 1e-6
    above the bump's top (depth 1e-6 there), depth limiter on, 20 SSP-RK3
    steps, at the FP32 run tolerance 1e-4 of the limiter tests;
  * the same in the tensor-core mode (DG_PREC_FP32_TC)."""
import numpy as np
import pytest

import synth
from helpers import both, rel_l2, sensitivity
from oracle.run import build as oracle_build, residual_nodal, run_explicit

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _film(dim, p):
    if dim == 1:
        c = synth.dam_break_1d(n_el=60, order=p, reg=3, sigma0=0.01, eta=0.01, gamma=20.0)
        c.coords = np.linspace(-1.0, 1.0, 61).reshape(-1, 1)
        c.h_fn = lambda x, xc: 1e-6 + 5e-3 * 0.5 * (1 + np.cos(np.pi * x[:, 0]))
        c.u_fn = lambda x, xc: 0.05 * np.sin(np.pi * x[:, 0])[:, None]
        c.bed_fn = lambda x, xc=None: 0.01 * np.cos(2.0 * x[:, 0])
    else:
        c = synth.radial_dam_2d(n=12, order=p, reg=3, sigma0=0.01, eta=0.01, gamma=20.0)
        c.h_fn = lambda x, xc: 1e-6 + 5e-3 * 0.25 * (1 + np.cos(np.pi * x[:, 0])) * (1 + np.cos(np.pi * x[:, 1]))
        c.u_fn = lambda x, xc: 0.05 * np.stack([np.sin(np.pi * x[:, 1]), -np.sin(np.pi * x[:, 0])], axis=1)
        c.bed_fn = lambda x, xc=None: 0.01 * np.cos(2.0 * x[:, 0]) * np.sin(x[:, 1])
    return c


def _near_dry_fraction(V0, h_dry=1e-3):
    return float((V0[0].min(axis=1) < h_dry).mean())


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_thin_film_residual_fp32(dim, p):
    import paper_2301_11238_gb300 as G
    c = _film(dim, p)
    d, V0, _, s = both(c, precision=G.PREC_FP32)
    assert 0.05 < _near_dry_fraction(V0) < 0.95  # both branches are exercised
    dv_o, E_o = residual_nodal(d, V0)
    dv, E = s.residual(V0)
    sv, se = sensitivity(d, V0, eps=2.0 ** -24)
    ev, ee = rel_l2(dv.cpu().numpy(), dv_o), rel_l2(E.cpu().numpy(), E_o)
    assert ev < max(1e-5, 10 * sv) and ee < max(1e-5, 10 * se), (ev, ee, sv, se)
    s.close()


def _bump_near_dry(p):
    amp = 0.2
    c = synth.bump_dam_2d(n=12, order=p, amp=amp, width=0.3, s_down=amp + 1e-6, sigma0=0.0, eta=0.0, positivity=1)
    c.params["reg"] = 0
    return c


@pytest.mark.parametrize("prec_name,p", [("fp32", 1), ("fp32", 2), ("fp32tc", 2)])
def test_bump_near_dry_run(prec_name, p):
    import paper_2301_11238_gb300 as G
    prec = {"fp32": G.PREC_FP32, "fp32tc": G.PREC_FP32_TC}[prec_name]
    c = _bump_near_dry(p)
    d, V0, _ = oracle_build(c)
    assert _near_dry_fraction(V0) > 0.0
    s, _, _ = G.solver_from_case(c, precision=prec)
    st = s.run(20)
    Vg = s.get_state(with_E=False)
    Vo, _, t = run_explicit(d, V0, 20)
    assert abs(st["t"] - t) < 1e-5 * t
    assert rel_l2(Vg, Vo) < 1e-4, rel_l2(Vg, Vo)
    # depths stay non-negative at the nodes (limiter) and near-dry values stay finite
    assert np.all(np.isfinite(Vg)) and Vg[0].min() > -1e-6
    s.close()
