"""Tensor-core volume pass (DG_PREC_FP32_TC: tcgen05 TF32 with hi/lo
operand splits, FP32 accumulation) against the FP64 oracle, through the C
ABI.

The three contractions it moves to the tensor cores (interpolation to the
volume points, the test-function contraction of Eq. WeakForm51, the
h-weighted mass matrix of Appendix A) take operands split into two
round-to-nearest TF32 parts: about 22 significant bits each, against FP32's
24.  The tolerance follows the FP32 path's rule at that working precision:
max(1e-5, 10 x the problem's response to relative input perturbations of
2^-22).  (On the ill-conditioned smooth states here, where large flux and
source terms cancel, the response to 2^-24 perturbations is already
1e-5, and a split with truncated parts, about 20 bits, measured 2.7e-4.)  Cases cover p = 2 and 3, every regularization, a bed,
tiles with ragged ends (162 and 98 triangles), an exact multiple of the
128-element tile and a mesh with more tiles than SMs (each CTA walks
several tiles), the three output modes (stage update, dV/dt, raw residual
through dg_swe_residual_static), and a batch.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from helpers import both, rel_l2, sensitivity, smooth_case
from oracle.run import build as oracle_build, residual_nodal, run_explicit

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


TC_EPS = 2.0 ** -22


def _tol(d, V0):
    sv, se = sensitivity(d, V0, eps=TC_EPS)
    return max(FP32_TOL, 10.0 * sv), max(FP32_TOL, 10.0 * se)


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("reg", [0, 1, 2, 3, 4, 5])
def test_tc_residual_matches_oracle(p, reg):
    import paper_2301_11238_gb300 as G
    c = smooth_case(2, p, reg, n=9, seed=p + 10 * reg)  # 162 triangles: two tiles, the second ragged
    d, V0, _, s = both(c, precision=G.PREC_FP32_TC)
    dv_o, E_o = residual_nodal(d, V0)
    dv, E = s.residual(V0)
    tv, te = _tol(d, V0)
    ev, ee = rel_l2(dv.cpu().numpy(), dv_o), rel_l2(E.cpu().numpy(), E_o)
    assert ev < tv and ee < te, (ev, ee, tv, te)
    s.close()


@pytest.mark.parametrize("n,p", [(7, 3), (8, 2), (8, 3), (128, 2)])
def test_tc_residual_tile_shapes(n, p):
    """98 triangles (one ragged tile), 128 (exactly one tile) and 32,768
    (256 tiles: every CTA of the persistent grid walks several)."""
    import paper_2301_11238_gb300 as G
    c = smooth_case(2, p, 3, n=n, seed=5)
    d, V0, _, s = both(c, precision=G.PREC_FP32_TC)
    dv_o, _ = residual_nodal(d, V0)
    dv, _ = s.residual(V0)
    assert rel_l2(dv.cpu().numpy(), dv_o) < _tol(d, V0)[0]
    s.close()


@pytest.mark.parametrize("p", [2, 3])
def test_tc_close_to_cuda_core_fp32(p):
    import paper_2301_11238_gb300 as G
    c = smooth_case(2, p, 1, n=12, seed=21)
    d, V0, _, s32 = both(c, precision=G.PREC_FP32)
    _, _, _, stc = both(c, precision=G.PREC_FP32_TC)
    a = s32.residual(V0)[0].cpu().numpy()
    b = stc.residual(V0)[0].cpu().numpy()
    assert rel_l2(b, a) < _tol(d, V0)[0]
    s32.close()
    stc.close()


@pytest.mark.parametrize("case_fn", ["radial", "bump"])
def test_tc_run_matches_oracle(case_fn):
    """60 SSP-RK3 steps (stage-update mode, step size from the GPU's own
    FP64 reduction) against the oracle run with the same step sizes."""
    import paper_2301_11238_gb300 as G
    c = (synth.radial_dam_2d(n=10, order=2, reg=1, sigma0=0.02) if case_fn == "radial"
         else synth.bump_dam_2d(n=10, order=3))
    d, V0, _ = oracle_build(c)
    s, _, _ = G.solver_from_case(c, precision=G.PREC_FP32_TC)
    st = s.run(60)
    Vg = s.get_state(with_E=False)
    Vo, _, t = run_explicit(d, V0, 60)
    assert abs(st["t"] - t) < 1e-5 * t
    assert rel_l2(Vg, Vo) < 1e-5
    s.close()


def test_tc_static_residual_matches():
    """Raw-residual output mode (the allocation-free entry point's volume
    pass) in the tensor-core form."""
    import torch
    import paper_2301_11238_gb300 as G
    c = smooth_case(2, 3, 3, n=9, seed=31)
    d, V0, _, s = both(c, precision=G.PREC_FP32_TC)
    Vd = torch.from_numpy(np.ascontiguousarray(V0)).cuda()
    ref, _ = s.residual(Vd)
    out = torch.empty_like(Vd)
    with torch.cuda.stream(s.stream):
        st = s.L.dg_swe_residual_static(s.ctx, C.c_void_p(Vd.data_ptr()), C.c_void_p(out.data_ptr()), None)
    assert st == G.DG_OK, s.L.dg_swe_last_error(s.ctx)
    torch.cuda.synchronize()
    assert rel_l2(out.cpu().numpy(), ref.cpu().numpy()) < 1e-6
    s.close()


def test_tc_batch_equals_solo_and_oracle():
    import paper_2301_11238_gb300 as G
    cases = [synth.bump_dam_2d(n=9, order=3), synth.dam_break_1d(n_el=40, order=2),
             synth.radial_dam_2d(n=11, order=2, reg=3, sigma0=0.1, gamma=50.0)]
    B, V0s = G.batch_from_cases(cases, precision=G.PREC_FP32_TC)
    stB = B.run(20)
    for i, c in enumerate(cases):
        s, _, _ = G.solver_from_case(c, precision=G.PREC_FP32_TC)
        s.run(20)
        V = s.get_state(with_E=False)
        assert np.array_equal(V, B.get_state(i)), (i, rel_l2(B.get_state(i), V))
        s.close()
        d, V0, _ = oracle_build(c)
        Vo, _, t = run_explicit(d, V0, 20)
        assert abs(stB[i]["t"] - t) < 1e-5 * t
        assert rel_l2(B.get_state(i), Vo) < 1e-5, i
    B.close()
