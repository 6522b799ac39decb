"""CPU-side checks of the C ABI: the library builds, loads and exports every
entry point declared in include/*.h, and its host-only setup (reference
operators, connectivity, node layout, argument validation) behaves as
documented.  No GPU compute is called here."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

import synth
from oracle.run import node_coords

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(dg_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    import paper_2301_11238_gb300._lib as L
    lib = L.lib()
    names = _declared()
    assert "dg_swe_init" in names and "dg_swe_residual" in names and "dg_swe_run" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("dim,p", [(1, 1), (1, 2), (1, 3), (2, 1), (2, 2), (2, 3)])
def test_node_layout_matches_documented_convention(dim, p):
    import paper_2301_11238_gb300 as G
    c = synth.dam_break_1d(n_el=9, order=p) if dim == 1 else synth.bump_dam_2d(n=5, order=p)
    s = G.Solver(c.dim, c.coords, c.etov, p, c.params["reg"], c.params, face_bc=c.face_bc, bcs=c.bcs,
                 allocate=False)
    assert np.abs(s.node_coords() - node_coords(dim, c.coords, c.etov, p)).max() < 1e-14
    K = c.etov.shape[0]
    np_ = p + 1 if dim == 1 else (p + 1) * (p + 2) // 2
    assert (s.K, s.Np, s.nV, s.nE) == (K, np_, dim + 1, dim * dim)
    nf_expected = K + 1 if dim == 1 else 3 * 5 * 5 + 2 * 5  # 3n^2 + 2n edges of an n x n grid
    assert s.n_faces == nf_expected
    assert s.workspace_bytes % 256 == 0 and s.workspace_bytes > 0
    assert s.launches_per_step() == 11
    s.close()


def test_invalid_arguments_are_rejected():
    import paper_2301_11238_gb300 as G
    c = synth.radial_dam_2d(n=3)
    bad = []
    et = c.etov.copy()
    et[2] = et[2][::-1]  # clockwise triangle
    bad.append(dict(etov=et))
    bad.append(dict(order=4))
    bad.append(dict(reg=7))
    bad.append(dict(reg=2, prm=dict(c.params, sigma0=1e-4)))  # 0 < sigma0 < 1/(2 beta)
    bad.append(dict(prm=dict(c.params, h_floor=0.0)))
    fb = c.face_bc.copy()
    fb[0, 0] = 3  # tag beyond n_bc = 1 on a boundary face
    bad.append(dict(face_bc=fb))
    et2 = c.etov.copy()
    et2[0, 0] = 10 ** 6
    bad.append(dict(etov=et2))
    for kw in bad:
        args = dict(dim=2, coords=c.coords, etov=c.etov, order=2, reg=1, prm=c.params, face_bc=c.face_bc)
        args.update(kw)
        with pytest.raises(G.DGError) as ei:
            G.Solver(args["dim"], args["coords"], args["etov"], args["order"], args["reg"], args["prm"],
                     face_bc=args["face_bc"], allocate=False)
        assert ei.value.status == G.DG_ERR_ARG


def test_wall_mode_only_on_velocity_slots():
    import paper_2301_11238_gb300 as G
    c = synth.radial_dam_2d(n=3)
    with pytest.raises(G.DGError):
        G.Solver(2, c.coords, c.etov, 2, 1, c.params, bcs=[([2, 0, 0, 0, 0, 0, 0], [0.0] * 7)],
                 allocate=False)


def test_calls_without_workspace_fail_cleanly():
    import paper_2301_11238_gb300 as G
    c = synth.dam_break_1d(n_el=4)
    s = G.Solver(1, c.coords, c.etov, 1, 4, c.params, face_bc=c.face_bc, bcs=c.bcs, allocate=False)
    st = s.L.dg_swe_step(s.ctx, 0.0, None)
    assert st == G.DG_ERR_WORKSPACE
    st = s.L.dg_swe_set_workspace(s.ctx, C.c_void_p(0x1001), s.workspace_bytes)
    assert st == G.DG_ERR_WORKSPACE  # misaligned
    s.close()


def test_empty_mesh_rejected():
    import paper_2301_11238_gb300 as G
    coords = np.array([[0.0], [1.0]])
    with pytest.raises(G.DGError) as ei:
        G.Solver(1, coords, np.zeros((0, 2), dtype=np.int32), 1, 0, synth.cases.default_params(), allocate=False)
    assert ei.value.status == G.DG_ERR_ARG


def test_fma_probe_rejects_bad_arguments():
    import paper_2301_11238_gb300._lib as L
    lib = L.lib()
    out = C.c_double()
    fake = C.c_void_p(0x1000)  # never dereferenced: the arguments are rejected first
    assert lib.dg_probe_fma_rate(7, 5, fake, None, C.byref(out)) == L.DG_ERR_ARG
    assert lib.dg_probe_fma_rate(0, 0, fake, None, C.byref(out)) == L.DG_ERR_ARG
    assert lib.dg_probe_fma_rate(0, 5, None, None, C.byref(out)) == L.DG_ERR_ARG
    assert lib.dg_probe_fma_rate(0, 5, fake, None, None) == L.DG_ERR_ARG
