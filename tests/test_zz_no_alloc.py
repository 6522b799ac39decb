"""dg_swe_residual_static: the residual entry point for callers that must not
allocate device memory per call (an application that reserved its whole
device-memory budget at start-up, or a latency-critical path where cudaMalloc,
which may synchronize the device, is off limits).  Its scratch lives in the
library's file-scope device array instead of the workspace.

Checked through the C ABI against dg_swe_residual on two calls in a row (the
second with a different state, so stale scratch from the first call would
show), with and without the E output, in 1D and 2D, within the tolerances
the parity tests use; further calls must leave the device's free memory
unchanged; an oversize problem must be rejected with DG_ERR_ARG.  Collected last so that a first-failure
stop has already run every other test."""
import ctypes as C

import numpy as np
import pytest

import synth
from helpers import rel_l2, smooth_case
from oracle.run import build as oracle_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _solver(case, precision):
    import paper_2301_11238_gb300 as G
    _, V0, bed = oracle_build(case)
    s = G.Solver(case.dim, case.coords, case.etov, case.order, case.params["reg"], case.params,
                 face_bc=case.face_bc, bcs=case.bcs, bed=bed if case.bed_fn is not None else None,
                 precision=precision)
    return s, V0


def _static(s, Vd, dv, E):
    import torch
    with torch.cuda.stream(s.stream):
        return s.L.dg_swe_residual_static(s.ctx, C.c_void_p(Vd.data_ptr()), C.c_void_p(dv.data_ptr()),
                                          None if E is None else C.c_void_p(E.data_ptr()))


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_static_residual_matches_workspace_residual(dim, precision, tol):
    import torch
    import paper_2301_11238_gb300 as G
    case = smooth_case(dim, 2, 1, n=40 if dim == 1 else 16, seed=8)
    s, V0 = _solver(case, precision)
    assert s.L.dg_swe_static_scratch_need(s.ctx) <= 16 * 1024 * 1024
    rng = np.random.default_rng(2)
    states = [V0, V0 * (1.0 + 0.05 * rng.standard_normal(V0.shape))]
    for V in states:  # two calls in a row
        Vd = torch.from_numpy(np.ascontiguousarray(V)).cuda()
        ref_dv, ref_E = s.residual(Vd)
        dv = torch.empty_like(Vd)
        E = torch.empty_like(ref_E)
        st = _static(s, Vd, dv, E)
        assert st == G.DG_OK, s.L.dg_swe_last_error(s.ctx)
        torch.cuda.synchronize()
        assert rel_l2(dv.cpu().numpy(), ref_dv.cpu().numpy()) < tol
        assert rel_l2(E.cpu().numpy(), ref_E.cpu().numpy()) < tol
        # without the E output
        dv2 = torch.empty_like(Vd)
        assert _static(s, Vd, dv2, None) == G.DG_OK, s.L.dg_swe_last_error(s.ctx)
        torch.cuda.synchronize()
        assert rel_l2(dv2.cpu().numpy(), ref_dv.cpu().numpy()) < tol
    s.close()


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("precision", [0, 1])
def test_static_residual_allocates_nothing(dim, precision):
    """After a first call (which loads the kernels and looks up the array's
    address), further calls leave the device's free memory unchanged."""
    import torch
    import paper_2301_11238_gb300 as G
    case = smooth_case(dim, 2, 3, n=40 if dim == 1 else 16, seed=9)
    s, V0 = _solver(case, precision)
    Vd = torch.from_numpy(np.ascontiguousarray(V0)).cuda()
    dv = torch.empty_like(Vd)
    E = torch.empty((s.nE, s.K, s.Np), dtype=torch.float64, device="cuda")
    assert _static(s, Vd, dv, E) == G.DG_OK, s.L.dg_swe_last_error(s.ctx)
    assert _static(s, Vd, dv, None) == G.DG_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for out_E in (E, None, E):
        assert _static(s, Vd, dv, out_E) == G.DG_OK, s.L.dg_swe_last_error(s.ctx)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
    s.close()


def test_static_residual_rejects_oversize_problem():
    import torch
    import paper_2301_11238_gb300 as G
    case = synth.radial_dam_2d(n=200, order=3)
    s = G.Solver(case.dim, case.coords, case.etov, 3, 1, case.params, face_bc=case.face_bc, bcs=case.bcs)
    assert s.L.dg_swe_static_scratch_need(s.ctx) > 16 * 1024 * 1024
    Vd = torch.zeros((s.nV, s.K, s.Np), dtype=torch.float64, device="cuda")
    dv = torch.empty_like(Vd)
    st = s.L.dg_swe_residual_static(s.ctx, C.c_void_p(Vd.data_ptr()), C.c_void_p(dv.data_ptr()), None)
    assert st == G.DG_ERR_ARG
    assert b"static scratch" in s.L.dg_swe_last_error(s.ctx)
    s.close()
