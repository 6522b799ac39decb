"""Accuracy of the reduced-precision paths against what the scheme itself
achieves.

* Stated error against an exact solution: on the Newtonian dam break with
  its exact (Stoker) solution (eta = sigma0 = 0, 200 elements, p = 1,
  t = 0.1, fixed dt = 1e-4), the GPU's FP32 and FP64 paths have L1 depth
  errors against the exact solution of 1.11e-3 and 1.07e-3 (measured): the
  unlimited p = 1 solution oscillates at the shock, where rounding
  differences grow, so FP32 costs about 4 % of the discretization error
  there; the bound here is 10 %.
* Error horizon of the bump dam break (the p = 3, FP32 workload): relative L2
  distance to the FP64 oracle after 100 and 1000 SSP-RK3 steps on a 16x16x2
  jittered mesh, for the CUDA-core FP32 path and the tensor-core pass
  (measured 1.6e-6 and 1.25e-5 for both)."""
import numpy as np
import pytest

import synth
from helpers import rel_l2
from oracle import riemann
from oracle.run import build as oracle_build, run_explicit

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_fp32_and_fp64_share_the_discretization_error():
    import paper_2301_11238_gb300 as G
    c = synth.dam_break_1d(n_el=200, order=1, reg=0, eta=0.0, sigma0=0.0)
    d, V0, _ = oracle_build(c)
    xq = d.map_to_phys(d.rq)[..., 0]
    he, _ = riemann.sample(xq.ravel(), 0.1, 0.5, 1.0, 0.0, 0.5, 0.0, 9.81)
    errs, states = {}, {}
    for prec in (G.PREC_FP64, G.PREC_FP32):
        s, _, _ = G.solver_from_case(c, precision=prec)
        for _ in range(1000):  # fixed dt = 1e-4 (the step bound here is about 1.1e-4) to t = 0.1
            s.step(1e-4, sync=False)
        st = s.sync()
        assert abs(st["t"] - 0.1) < 1e-12
        V = s.get_state(with_E=False)
        hq = d.eval_at_quad(d.to_modal(V))[0]
        errs[prec] = float(np.sum(d.wJ.ravel() * np.abs(hq.ravel() - he)))
        states[prec] = V
        s.close()
    diff = rel_l2(states[G.PREC_FP32], states[G.PREC_FP64])
    print(f"L1 depth error vs exact: FP64 {errs[G.PREC_FP64]:.4e}, FP32 {errs[G.PREC_FP32]:.4e}; "
          f"FP32 vs FP64 states: {diff:.2e}")
    assert errs[G.PREC_FP64] < 2e-3
    assert abs(errs[G.PREC_FP32] - errs[G.PREC_FP64]) < 0.1 * errs[G.PREC_FP64], errs


@pytest.mark.parametrize("prec_name", ["fp32", "fp32tc"])
def test_bump_error_horizon(prec_name):
    import paper_2301_11238_gb300 as G
    prec = {"fp32": G.PREC_FP32, "fp32tc": G.PREC_FP32_TC}[prec_name]
    c = synth.bump_dam_2d(n=16, order=3)
    d, V0, _ = oracle_build(c)
    s, _, _ = G.solver_from_case(c, precision=prec)
    Vo = V0
    out = []
    for n in (100, 900):
        Vo, _, _ = run_explicit(d, Vo, n)
        s.run(n)
        out.append(rel_l2(s.get_state(with_E=False), Vo))
    s.close()
    print(f"{prec_name}: rel L2 vs FP64 oracle after 100 / 1000 steps: {out[0]:.2e} / {out[1]:.2e}")
    assert out[0] < 1e-5 and out[1] < 1e-4, out
