"""Host-side checks of the batch ABI (no GPU work): grouping by (dim, order),
totals, launch accounting and per-instance validation."""
import numpy as np
import pytest

import synth


def _spec(c):
    return dict(dim=c.dim, coords=c.coords, etov=c.etov, order=c.order, reg=c.params["reg"], prm=c.params,
                face_bc=c.face_bc, bcs=c.bcs)


def test_batch_groups_and_totals():
    import paper_2301_11238_gb300 as G
    cases = [synth.dam_break_1d(n_el=30, order=1), synth.radial_dam_2d(n=4, order=2),
             synth.radial_dam_2d(n=5, order=2, reg=3), synth.dam_break_1d(n_el=12, order=3)]
    b = G.Batch([_spec(c) for c in cases], allocate=False)
    info = b.info()
    assert info["groups"] == 3
    assert info["elements"] == 30 + 32 + 50 + 12
    assert info["dofs"] == 30 * 2 * 2 + 32 * 6 * 3 + 50 * 6 * 3 + 12 * 4 * 2
    assert b.launches_per_step() == 33
    assert b.tiles() == [[128, 128, 128]] * 3
    b.close()


def test_batch_rejects_bad_instance_and_mixed_precision():
    import paper_2301_11238_gb300 as G
    good = synth.radial_dam_2d(n=3)
    bad = synth.radial_dam_2d(n=3)
    et = bad.etov.copy()
    et[0] = et[0][::-1]
    specs = [_spec(good), dict(_spec(bad), etov=et)]
    with pytest.raises(G.DGError) as ei:
        G.Batch(specs, allocate=False)
    assert ei.value.status == G.DG_ERR_ARG and "instance 1" in str(ei.value)
