"""Batched ensembles on the GPU: every batched instance must evolve exactly
as the same instance run alone (FP64, bitwise), and, transitively, as the
oracle; the autotuner must not change results."""
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
    a = synth.dam_break_1d(n_el=70, order=1)
    b = synth.radial_dam_2d(n=10, order=2, reg=1, sigma0=0.02)
    c = synth.radial_dam_2d(n=7, order=2, reg=3, sigma0=0.1, gamma=50.0)
    d = smooth_case(1, 3, 2, n=40, seed=5, bc="dirichlet")
    e = smooth_case(2, 1, 5, n=6, seed=6, bc="wall")
    f = synth.bump_dam_2d(n=6, order=3)
    return [a, b, c, d, e, f]


def test_batch_matches_single_instances_bitwise():
    import paper_2301_11238_gb300 as G
    cases = _mixed_cases()
    B, V0s = G.batch_from_cases(cases)
    stB = B.run(25)
    for i, c in enumerate(cases):
        s, V0, _ = G.solver_from_case(c)
        st = s.run(25)
        V = s.get_state(with_E=False)
        VB = B.get_state(i)
        assert np.array_equal(V, VB), (i, rel_l2(VB, V))
        assert stB[i]["t"] == st["t"] and stB[i]["steps"] == 25
        assert abs(stB[i]["mass"] - st["mass"]) <= 1e-14 * abs(st["mass"])
        s.close()
    B.close()


def test_batch_instance_matches_oracle():
    import paper_2301_11238_gb300 as G
    c = synth.radial_dam_2d(n=8, order=2, reg=2, sigma0=0.1)
    other = synth.dam_break_1d(n_el=50, order=2)
    B, _ = G.batch_from_cases([other, c])
    d, V0, _ = oracle_build(c)
    Vo, _, t = run_explicit(d, V0, 20)
    st = B.run(20)
    assert abs(st[1]["t"] - t) < 1e-12 * t
    assert rel_l2(B.get_state(1), Vo) < 1e-12


def test_autotune_keeps_results():
    import paper_2301_11238_gb300 as G
    cases = _mixed_cases()[:3]
    B1, _ = G.batch_from_cases(cases)
    B2, _ = G.batch_from_cases(cases)
    tiles = B2.autotune(3)
    # the grid-stride E-step, the per-face flux and the staged volume forms
    # are reported as negative block sizes
    sizes = (32, 64, 128, 256)
    for g in tiles:
        assert abs(g[0]) in sizes and abs(g[1]) in sizes and abs(g[2]) in sizes
    B1.run(10)
    B2.run(10)
    for i in range(len(cases)):
        assert np.array_equal(B1.get_state(i), B2.get_state(i))


def test_batch_fp32_close_to_fp64():
    import paper_2301_11238_gb300 as G
    cases = _mixed_cases()[:3]
    B64, _ = G.batch_from_cases(cases)
    B32, _ = G.batch_from_cases(cases, precision=G.PREC_FP32)
    B64.run(20)
    B32.run(20)
    for i in range(3):
        assert rel_l2(B32.get_state(i), B64.get_state(i)) < 1e-5


def test_batch_nonfinite_names_instance():
    import paper_2301_11238_gb300 as G
    cases = _mixed_cases()[:2]
    B, V0s = G.batch_from_cases(cases)
    V = V0s[1].copy()
    V[0, 5, 0] = np.inf
    B.set_state(1, V)
    with pytest.raises(G.DGError) as ei:
        B.run(2)
    assert ei.value.status == G.DG_ERR_NONFINITE and "instance 1" in str(ei.value)


def _run_with_volume_tiles(cases, precision, vol_tile, steps):
    import paper_2301_11238_gb300 as G
    B, _ = G.batch_from_cases(cases, precision=precision)
    tiles = B.tiles()
    B.set_tiles([[t[0], t[1], vol_tile] for t in tiles])
    B.run(steps)
    out = [B.get_state(i) for i in range(len(cases))]
    B.close()
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_staged_volume_bitwise_equal_to_direct(prec):
    """The staged volume kernel (bulk copies into shared memory, negative
    block size) does the same arithmetic as the direct one: in FP64 bitwise
    equal states after 12 steps, for 1D/2D groups of every order, with and
    without a bed, through every RK stage (c0 = 0 and c0 != 0).  In FP32 the
    two kernels inline the same element code, but the compiler may fuse its
    multiply-adds differently in each (seen once the near-dry FP64 mass solve
    joined that code: 5.7e-11 relative after 12 steps on the p = 3 bump), so
    FP32 states agree to 1e-9 relative, far below FP32 rounding."""
    cases = _mixed_cases()
    ref = _run_with_volume_tiles(cases, prec, 64, 12)
    for T in (-32, -64, -128):
        got = _run_with_volume_tiles(cases, prec, T, 12)
        for i in range(len(cases)):
            if prec == 0:
                assert np.array_equal(got[i], ref[i]), (T, i, rel_l2(got[i], ref[i]))
            else:
                assert rel_l2(got[i], ref[i]) < 1e-9, (T, i, rel_l2(got[i], ref[i]))


@pytest.mark.parametrize("prec", [0, 1])
def test_staged_volume_persistent_loop(prec):
    """131,072 triangles: more tiles than resident blocks (4096 tiles of 32
    against at most about 1,800 resident blocks), so every block walks
    several tiles and the copy of its next tile overlaps the current one;
    T = 96 leaves a ragged last tile."""
    c = synth.radial_dam_2d(n=256, order=2, reg=1, sigma0=0.02)
    ref = _run_with_volume_tiles([c], prec, 128, 3)[0]
    for T in (-32, -96):
        got = _run_with_volume_tiles([c], prec, T, 3)[0]
        assert np.array_equal(got, ref), (T, rel_l2(got, ref))


def test_staged_volume_rejects_oversized_tile():
    import paper_2301_11238_gb300 as G
    B, _ = G.batch_from_cases([synth.bump_dam_2d(n=4, order=3)])
    t = B.tiles()[0]
    with pytest.raises(G.DGError) as ei:
        B.set_tiles([[t[0], t[1], -256]])  # 2 x 11 slots x 20 KB: beyond shared memory
    assert ei.value.status == G.DG_ERR_ARG
    B.set_tiles([[t[0], t[1], -32]])
    B.run(2)
    B.close()


def test_batch_mass_multiblock_instances():
    """Mass and initial mass of instances that span several 256-element
    reduction blocks (with ragged last blocks), next to small ones: equal to
    the single-context solver and to the oracle's integral of h of the same
    state to 1e-14, and reproducible bit for bit across stats calls."""
    import paper_2301_11238_gb300 as G
    cases = [synth.dam_break_1d(n_el=3001, order=2),
             synth.radial_dam_2d(n=4, order=1),
             synth.radial_dam_2d(n=40, order=2, reg=3, sigma0=0.02, gamma=50.0),
             synth.dam_break_1d(n_el=50, order=1),
             synth.radial_dam_2d(n=37, order=3)]
    B, V0s = G.batch_from_cases(cases)
    discs = [oracle_build(c)[0] for c in cases]
    st0 = B.stats()
    for i, d in enumerate(discs):
        m_ref = d.total_mass(d.to_modal(V0s[i]))
        assert abs(st0[i]["mass0"] - m_ref) <= 1e-14 * abs(m_ref), (i, st0[i]["mass0"], m_ref)
        assert abs(st0[i]["mass"] - m_ref) <= 1e-14 * abs(m_ref)
    st = B.run(4)
    again = B.stats()
    for i, (c, d) in enumerate(zip(cases, discs)):
        VB = B.get_state(i)
        m_ref = d.total_mass(d.to_modal(VB))
        assert abs(st[i]["mass"] - m_ref) <= 1e-14 * abs(m_ref), (i, st[i]["mass"], m_ref)
        assert st[i]["mass"] == again[i]["mass"] and st[i]["mass0"] == again[i]["mass0"]
        s, _, _ = G.solver_from_case(c)
        ss = s.run(4)
        assert abs(ss["mass"] - st[i]["mass"]) <= 1e-14 * abs(ss["mass"])
        assert abs(ss["mass0"] - st[i]["mass0"]) <= 1e-14 * abs(ss["mass0"])
        s.close()
    B.close()


def _run_with_tiles(cases, precision, tiles_fn, steps):
    import paper_2301_11238_gb300 as G
    B, _ = G.batch_from_cases(cases, precision=precision)
    B.set_tiles([tiles_fn(t) for t in B.tiles()])
    B.run(steps)
    out = [B.get_state(i) for i in range(len(cases))]
    B.close()
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_grid_stride_estep_and_face_forms_equal_direct(prec):
    """The grid-stride E-step (negative E-step block size) and the per-face
    flux form with connectivity prefetch (negative face block size) do the
    arithmetic of the direct kernels: FP64 states bitwise equal after 12
    steps on the mixed 1D/2D groups of every order, and after 3 steps on
    131,072 triangles, where every thread of the resident grid walks several
    elements and faces (block sizes 32 and 96 leave ragged ends).  FP32 to
    1e-9 relative (the compiler may fuse multiply-adds differently)."""
    cases = _mixed_cases()
    ref = _run_with_tiles(cases, prec, lambda t: [64, 64, 64], 12)
    for T in (-32, -64, -256):
        got = _run_with_tiles(cases, prec, lambda t: [T, T, 64], 12)
        for i in range(len(cases)):
            if prec == 0:
                assert np.array_equal(got[i], ref[i]), (T, i, rel_l2(got[i], ref[i]))
            else:
                assert rel_l2(got[i], ref[i]) < 1e-9, (T, i, rel_l2(got[i], ref[i]))
    big = [synth.radial_dam_2d(n=256, order=2, reg=1, sigma0=0.02)]
    ref = _run_with_tiles(big, prec, lambda t: [128, 128, 128], 3)[0]
    for T in (-32, -96, -128):
        got = _run_with_tiles(big, prec, lambda t: [T, T, 128], 3)[0]
        if prec == 0:
            assert np.array_equal(got, ref), (T, rel_l2(got, ref))
        else:
            assert rel_l2(got, ref) < 1e-9, (T, rel_l2(got, ref))
