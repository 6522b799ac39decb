"""Shared test helpers: build the oracle and the library on the same seeded case."""
import numpy as np

import synth
from oracle.run import build as oracle_build


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0))


def smooth_case(dim, p, reg, n=None, seed=0, bed=True, alpha=0.05, sigma0=0.5, gamma=1.0, beta=5.0,
                eta=0.05, pap_m=1.0, bc="copy", length=10.0):
    """A case with seeded smooth random fields on a jittered mesh; parameters
    chosen so that |E| crosses the regularizations' branch points."""
    if dim == 1:
        c = synth.dam_break_1d(n_el=n or 150, order=p, reg=reg, sigma0=sigma0, eta=eta, pap_m=pap_m)
        c.coords = np.linspace(0.0, length, c.etov.shape[0] + 1).reshape(-1, 1)
    else:
        c = synth.radial_dam_2d(n=n or 9, order=p, reg=reg, sigma0=sigma0, eta=eta)
        c.coords, c.etov = synth.rect_tri_mesh(n or 9, n or 9, jitter=0.1, seed=seed + 11)
        c.face_bc = np.zeros((c.etov.shape[0], 3), dtype=np.int8)
    c.params.update(gamma=gamma, beta=beta, alpha=alpha)
    h_fn, u_fn, b_fn = synth.random_smooth_fields(dim, seed, h_amp=0.3, u_amp=1.5,
                                                  bed_amp=0.1 if bed else 0.0)
    c.h_fn, c.u_fn, c.bed_fn = h_fn, u_fn, b_fn
    if bc == "wall":
        c.bcs = ([([0, 2, 0, 0, 0, 0, 0], [0.0] * 7)] * 2 if dim == 1
                 else [([0, 2, 2, 0, 0, 0, 0], [0.0] * 7)])
    elif bc == "dirichlet":
        c.bcs = [([1, 1, 1, 1, 0, 0, 0], [1.2, 0.3, -0.2, 0.1, 0, 0, 0]),
                 ([1, 0, 1, 0, 0, 0, 0], [0.9, 0.0, 0.0, 0.0, 0, 0, 0])]
        if dim == 2:
            c.face_bc = (np.arange(c.etov.shape[0] * 3).reshape(-1, 3) % 2).astype(np.int8)
    return c


def both(case, precision=0):
    """Oracle discretization, nodal V0 and bed, and a library Solver on the same inputs."""
    import paper_2301_11238_gb300 as G
    d, V0, bed = oracle_build(case)
    s = G.Solver(case.dim, case.coords, case.etov, case.order, case.params["reg"], case.params,
                 face_bc=case.face_bc, bcs=case.bcs, bed=bed if case.bed_fn is not None else None,
                 precision=precision)
    return d, V0, bed, s


def sensitivity(d, V0, trials=3, seed=1, eps=2.2e-16):
    """Relative L2 change of the oracle's (dV/dt, E) under random relative
    perturbations of size eps (default 1 ulp of FP64) of the input state: the
    rounding sensitivity of the problem itself, a floor no implementation
    working at that precision can beat.  Returns (s_dV, s_E)."""
    from oracle.run import residual_nodal
    dv, E = residual_nodal(d, V0)
    rng = np.random.default_rng(seed)
    sv = se = 0.0
    for _ in range(trials):
        V1 = V0 * (1 + eps * rng.uniform(-1, 1, V0.shape))
        dv1, E1 = residual_nodal(d, V1)
        sv = max(sv, rel_l2(dv1, dv))
        se = max(se, rel_l2(E1, E))
    return sv, se
