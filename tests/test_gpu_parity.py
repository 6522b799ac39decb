"""GPU (sm_103a) explicit path vs the FP64 oracle, through the C ABI.

FP64 tolerance: 1e-12 relative L2 (nodal values), the bound the method's
FP64 target states, raised to 10x the problem's own rounding sensitivity
(the oracle's response to 1-ulp input perturbations, ``helpers.sensitivity``)
where that floor exceeds 1e-12: for stiff viscous/Bingham states on fine 1D
meshes no FP64 evaluation order can agree to 1e-12.  FP32 tolerances are
stated per test.
"""
import math

import numpy as np
import pytest

import synth
from helpers import both, rel_l2, sensitivity, smooth_case
from oracle.run import residual_nodal, run_explicit

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


FP32_TOL = 1e-5
FP32_EPS = 2.0 ** -24


def fp64_tol(d, V0):
    """(tolerance for dV/dt, tolerance for E)."""
    sv, se = sensitivity(d, V0)
    return max(FP64_TOL, 10.0 * sv), max(FP64_TOL, 10.0 * se)


def fp32_tol(d, V0):
    """FP32 inputs are rounded to single precision: the floor is the
    problem's response to relative perturbations of 2^-24."""
    sv, se = sensitivity(d, V0, eps=FP32_EPS)
    return max(FP32_TOL, 10.0 * sv), max(FP32_TOL, 10.0 * se)


def check(dv, E, dv_o, E_o, tols):
    ev = rel_l2(dv.cpu().numpy(), dv_o)
    ee = rel_l2(E.cpu().numpy(), E_o)
    assert ev < tols[0] and ee < tols[1], (ev, ee, tols)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("reg", [0, 1, 2, 3, 4, 5])
def test_residual_fp64_1d(p, reg):
    c = smooth_case(1, p, reg, n=150, seed=p + 10 * reg)
    d, V0, _, s = both(c)
    dv_o, E_o = residual_nodal(d, V0)
    dv, E = s.residual(V0)
    check(dv, E, dv_o, E_o, fp64_tol(d, V0))


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("reg", [0, 1, 2, 3, 4, 5])
def test_residual_fp64_2d(p, reg):
    c = smooth_case(2, p, reg, n=9, seed=p + 10 * reg)
    d, V0, _, s = both(c)
    dv_o, E_o = residual_nodal(d, V0)
    dv, E = s.residual(V0)
    check(dv, E, dv_o, E_o, fp64_tol(d, V0))


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("bc", ["wall", "dirichlet"])
def test_residual_fp64_boundary_conditions(dim, bc):
    c = smooth_case(dim, 2, 1, bc=bc, seed=3)
    d, V0, _, s = both(c)
    dv_o, E_o = residual_nodal(d, V0)
    dv, E = s.residual(V0)
    check(dv, E, dv_o, E_o, fp64_tol(d, V0))


def test_residual_fp64_radial_dam_full_size():
    """The 8192-triangle, p = 2 radial dam break at its initial state and at
    a smooth random state (single residual evaluation)."""
    c = synth.radial_dam_2d(n=64, order=2, reg=1, sigma0=0.02)
    d, V0, _, s = both(c)
    dv_o, E_o = residual_nodal(d, V0)
    dv, E = s.residual(V0)
    check(dv, E, dv_o, E_o, (FP64_TOL, FP64_TOL))
    h_fn, u_fn, _ = synth.random_smooth_fields(2, 5, u_amp=0.5)
    V1, _ = synth.Case.initial_state(
        synth.Case("x", 2, c.coords, c.etov, c.face_bc, c.bcs, 2, c.params, h_fn=h_fn, u_fn=u_fn),
        d.node_xyz)
    dv_o, E_o = residual_nodal(d, V1)
    dv, E = s.residual(V1)
    check(dv, E, dv_o, E_o, fp64_tol(d, V1))


def test_lake_at_rest_gpu():
    c = synth.bump_dam_2d(n=10, order=3)
    c.h_fn = lambda x, xc=None, b=c.bed_fn: 1.0 - b(x)
    d, V0, _, s = both(c)
    dv, _ = s.residual(V0)
    assert np.abs(dv.cpu().numpy()).max() < 1e-11


def test_run_1d_dam_break_fp64():
    """1D Bingham dam break, 200 elements, p = 1, exponential regularization,
    2000 CFL-limited SSP-RK3 steps: final state vs the oracle run."""
    c = synth.dam_break_1d()
    d, V0, _, s = both(c)
    Vo, dts, t = run_explicit(d, V0, 2000)
    s.set_state(V0)
    st = s.run(2000)
    V, _ = s.get_state()
    assert st["steps"] == 2000
    assert abs(st["t"] - t) < 1e-12 * t
    assert rel_l2(V, Vo) < FP64_TOL


def test_run_2d_radial_dam_fp64():
    c = synth.radial_dam_2d(n=12, order=2, reg=2, sigma0=0.1)
    d, V0, _, s = both(c)
    Vo, dts, t = run_explicit(d, V0, 60)
    s.set_state(V0)
    st = s.run(60)
    V, _ = s.get_state()
    assert abs(st["t"] - t) < 1e-12 * t
    assert rel_l2(V, Vo) < FP64_TOL


def test_step_fixed_dt_matches_oracle():
    c = smooth_case(2, 3, 3, n=6, seed=9)
    d, V0, _, s = both(c)
    dt = 1e-4
    Vo, _, _ = run_explicit(d, V0, 3, dt=dt)
    s.set_state(V0)
    for _ in range(3):
        assert s.step(dt) == dt
    V, _ = s.get_state()
    assert rel_l2(V, Vo) < FP64_TOL


def test_mass_conservation_walls_gpu():
    c = synth.radial_dam_2d(n=16, order=2, reg=3, sigma0=0.05, gamma=20.0)
    c.bcs = [([0, 2, 2, 0, 0, 0, 0], [0.0] * 7)]
    d, V0, _, s = both(c)
    s.set_state(V0)
    st = s.run(200)
    assert abs(st["mass"] - st["mass0"]) < 1e-13 * st["mass0"]
    assert abs(st["mass0"] - d.total_mass(d.to_modal(V0))) < 1e-13 * st["mass0"]


def test_nonfinite_state_is_reported():
    import paper_2301_11238_gb300 as G
    c = synth.dam_break_1d(n_el=40)
    d, V0, _, s = both(c)
    V = V0.copy()
    V[0, 3, 1] = np.nan
    s.set_state(V)
    with pytest.raises(G.DGError) as ei:
        s.run(2)
    assert ei.value.status == G.DG_ERR_NONFINITE


# ------------------------------------------------------------------ FP32

@pytest.mark.parametrize("dim,p", [(1, 1), (1, 3), (2, 2), (2, 3)])
def test_residual_fp32(dim, p):
    """FP32 state and arithmetic: relative L2 within max(1e-5, 10x the
    problem's response to 2^-24 input rounding) of the FP64 oracle."""
    c = smooth_case(dim, p, 3, seed=21)
    d, V0, _, s = both(c, precision=1)
    dv_o, E_o = residual_nodal(d, V0)
    dv, E = s.residual(V0)
    check(dv, E, dv_o, E_o, fp32_tol(d, V0))


def test_run_2d_radial_dam_fp32():
    c = synth.radial_dam_2d(n=12, order=2, reg=1, sigma0=0.02)
    d, V0, _, s = both(c, precision=1)
    Vo, _, t = run_explicit(d, V0, 60)
    s.set_state(V0)
    st = s.run(60)
    V, _ = s.get_state()
    assert abs(st["t"] - t) < 1e-5 * t
    assert rel_l2(V, Vo) < 1e-5


def test_residual_fp64_fine_1d_within_rounding_sensitivity():
    """150 elements on [0, 1], p = 3, bi-viscosity: the oracle's own rounding
    sensitivity is above 1e-12 here; the library must stay within a small
    multiple of it."""
    c = smooth_case(1, 3, 5, n=150, seed=4, length=1.0)
    d, V0, _, s = both(c)
    dv_o, _ = residual_nodal(d, V0)
    dv, _ = s.residual(V0)
    sens = sensitivity(d, V0)[0]
    assert sens > FP64_TOL
    assert rel_l2(dv.cpu().numpy(), dv_o) < 10.0 * sens


# ------------------------------------------------------------------ edge cases

@pytest.mark.parametrize("dim", [1, 2])
def test_single_element_and_smallest_meshes(dim):
    """Every face a boundary face (1D, one element) or two triangles sharing
    one face (2D, one square): residual and a few steps against the oracle."""
    if dim == 1:
        c = smooth_case(1, 3, 3, n=1, seed=2, bc="dirichlet")
    else:
        c = smooth_case(2, 2, 1, n=1, seed=2, bc="wall")
    d, V0, _, s = both(c)
    dv_o, E_o = residual_nodal(d, V0)
    dv, E = s.residual(V0)
    check(dv, E, dv_o, E_o, fp64_tol(d, V0))
    Vo, _, _ = run_explicit(d, V0, 3)
    s.set_state(V0)
    s.run(3)
    V, _ = s.get_state()
    assert rel_l2(V, Vo) < FP64_TOL


@pytest.mark.parametrize("reg", [1, 2, 3, 4, 5])
def test_zero_yield_stress_is_newtonian(reg):
    """sigma0 = 0 removes the Bingham term for every regularization: the
    library's residual equals its Newtonian residual bit for bit."""
    import paper_2301_11238_gb300 as G
    c = smooth_case(2, 2, reg, n=6, seed=4, sigma0=0.0)
    c0 = smooth_case(2, 2, 0, n=6, seed=4, sigma0=0.0)
    _, V0, bed, s = both(c)
    _, _, _, s0 = both(c0)
    dv, E = s.residual(V0)
    dv0, E0 = s0.residual(V0)
    assert np.array_equal(dv.cpu().numpy(), dv0.cpu().numpy())


def test_near_dry_state_uses_floor():
    """Depths below h_floor (1e-6) at some nodes: wave speeds and the
    h-weighted mass use max(h, h_floor); the result stays finite and matches
    the oracle."""
    c = smooth_case(2, 2, 3, n=6, seed=5, bed=False)
    c.params["h_floor"] = 1e-3
    d, V0, _, s = both(c)
    V = V0.copy()
    V[0, :5, :] = 2e-4  # five elements below the floor
    dv_o, E_o = residual_nodal(d, V)
    dv, E = s.residual(V)
    assert np.isfinite(dv.cpu().numpy()).all()
    check(dv, E, dv_o, E_o, fp64_tol(d, V))
