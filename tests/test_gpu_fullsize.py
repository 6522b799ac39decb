"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (one batch, autotuned kernel forms, CUDA-graph replay): one SSP-RK3
step of the 8.4M-triangle slump (FP64 and FP32), the 524,288-triangle bump dam break
(p = 3, FP32) and the nine-instance radial sweep (FP64), checked on sampled
elements against the oracle, and whole instances of the 256-instance
ensemble (FP32).

The oracle cannot hold millions of elements, but one RK step of an element
depends only on elements within six face rings of it (three stages, each an
E-step and a flux exchange with face neighbours).  For each sampled element
the oracle therefore runs the step on the patch of elements within seven
vertex rings, from the same initial nodal state and with the step size the
GPU took (the only global quantity of the step)."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from helpers import rel_l2
from oracle.dg import Discretization
from oracle.run import node_coords

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _patch(etov, n_vertices, seeds, rings=7):
    """Elements within ``rings`` vertex rings of the seed elements."""
    K, nv = etov.shape
    A = sp.csr_matrix((np.ones(K * nv), (np.repeat(np.arange(K), nv), etov.ravel())), shape=(K, n_vertices))
    mask = np.zeros(K, dtype=bool)
    mask[seeds] = True
    At = A.T.tocsr()
    for _ in range(rings):
        vmask = (At @ mask.astype(np.float64)) > 0
        mask = (A @ vmask.astype(np.float64)) > 0
    return np.nonzero(mask)[0]


def _oracle_step_on_patch(case, V0, bed, elems, dt):
    etov = case.etov[elems]
    used, inv = np.unique(etov.ravel(), return_inverse=True)
    coords = case.coords[used]
    sub = inv.reshape(etov.shape)
    d = Discretization(case.dim, coords, sub, case.order, case.params, face_bc=np.zeros_like(sub, dtype=np.int64),
                       bcs=case.bcs, bed_nodal=None if case.bed_fn is None else bed[elems])
    Vh = d.to_modal(V0[:, elems, :])
    V1, _ = d.ssp_rk3_step(Vh, dt)
    return d.to_nodal(V1)


def _sampled_check(case, precision, n_samples, tol, seed=0):
    import paper_2301_11238_gb300 as G
    B, V0s = G.batch_from_cases([case], precision=precision)
    B.autotune(3)
    B.advance(1)
    st = B.stats()[0]
    V1 = B.get_state(0)
    B.close()
    assert st["steps"] == 1
    V0 = np.asarray(V0s[0])
    _, bed = case.initial_state(node_coords(case.dim, case.coords, case.etov, case.order))
    rng = np.random.default_rng(seed)
    K = case.etov.shape[0]
    picks = rng.choice(K, size=n_samples, replace=False)
    got, ref = [], []
    for e in picks:
        elems = _patch(case.etov, case.coords.shape[0], [e])
        Vp = _oracle_step_on_patch(case, V0, bed, elems, st["dt_last"])
        k = int(np.searchsorted(elems, e))
        got.append(V1[:, e, :])
        ref.append(Vp[:, k, :])
    err = rel_l2(np.array(got), np.array(ref))
    assert err < tol, err
    return err


def test_slump_full_size_fp32_sampled():
    """8,388,608 triangles, p = 2: 12 sampled elements after one step."""
    _sampled_check(synth.slump_2d(n=2048), 1, 12, 1e-5)


def test_bump_full_size_fp32_sampled():
    """524,288 jittered triangles, p = 3 (the staged volume kernel is among
    the autotuner's candidates for this group)."""
    _sampled_check(synth.bump_dam_2d(n=512), 1, 12, 1e-5)


def test_radial_sweep_full_size_fp64_sampled():
    """Nine 8192-triangle instances in one batch; instance by instance,
    8 sampled elements each, FP64 tolerance."""
    import paper_2301_11238_gb300 as G
    cases = [synth.radial_dam_2d(n=64, order=2, reg=reg, sigma0=s0, eta=0.01, gamma=1e3, beta=1e3)
             for s0 in (0.0, 0.02, 0.1) for reg in (1, 2, 3)]
    B, V0s = G.batch_from_cases(cases)
    B.autotune(3)
    B.advance(1)
    stats = B.stats()
    rng = np.random.default_rng(3)
    for i, c in enumerate(cases):
        V1 = B.get_state(i)
        V0 = np.asarray(V0s[i])
        got, ref = [], []
        for e in rng.choice(c.etov.shape[0], size=8, replace=False):
            elems = _patch(c.etov, c.coords.shape[0], [e])
            Vp = _oracle_step_on_patch(c, V0, None, elems, stats[i]["dt_last"])
            got.append(V1[:, e, :])
            ref.append(Vp[:, int(np.searchsorted(elems, e)), :])
        assert rel_l2(np.array(got), np.array(ref)) < 1e-12, i
    B.close()


def test_ensemble_full_size_fp32_whole_instances():
    """The 256-instance ensemble in one batch (FP32): after one step, the
    three smallest 1D and the two smallest 2D instances against whole-instance
    oracle steps."""
    import paper_2301_11238_gb300 as G
    from oracle.run import build
    cases = synth.ensemble_cases()
    B, V0s = G.batch_from_cases(cases, precision=G.PREC_FP32)
    B.autotune(3)
    B.advance(1)
    stats = B.stats()
    sizes = [(c.etov.shape[0], i) for i, c in enumerate(cases)]
    one = sorted((k, i) for k, i in sizes if cases[i].dim == 1)[:3]
    two = sorted((k, i) for k, i in sizes if cases[i].dim == 2)[:2]
    for _, i in one + two:
        d, V0, _ = build(cases[i])
        V1o, _ = d.ssp_rk3_step(d.to_modal(np.asarray(V0s[i])), stats[i]["dt_last"])
        assert rel_l2(B.get_state(i), d.to_nodal(V1o)) < 1e-5, i
    B.close()


def test_slump_full_size_fp64_sampled():
    """The benchmark's headline: 8,388,608 triangles, p = 2, FP64, one step
    in the benchmark's launch configuration; 12 sampled elements at the FP64
    tolerance."""
    _sampled_check(synth.slump_2d(n=2048), 0, 12, 1e-12, seed=1)
