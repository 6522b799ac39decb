"""GB300 (sm_103a) DG solver for shallow-water flow with a regularized Bingham law.

Thin Python binding of the C ABI in include/dg_swe.h: it marshals arguments
and hands PyTorch-owned device memory (the workspace) and CUDA streams to the
library.  Every step of the method runs in the library's CUDA kernels; if the
library cannot be built or loaded, constructing a solver raises.
"""
import ctypes as C

import numpy as np

from . import _lib
from ._lib import (DG_OK, DG_ERR_ARG, DG_ERR_CUDA, DG_ERR_WORKSPACE, DG_ERR_NONFINITE,  # noqa: F401
                   DG_ERR_NEWTON, DG_ERR_UNSUPPORTED, DG_ERR_TIMEOUT, STATUS_NAMES)

PREC_FP64, PREC_FP32, PREC_FP32_TC = 0, 1, 2


class DGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _torch():
    import torch
    return torch


def make_params(prm, bcs=None, precision=PREC_FP64):
    """dg_swe_params from a dict with keys g, rho, alpha, eta, sigma0, gamma,
    beta, pap_m, h_floor, cfl and a list of (modes[7], values[7]) boundary
    descriptors."""
    p = _lib.Params()
    for k in ("g", "rho", "alpha", "eta", "sigma0", "gamma", "beta", "pap_m", "h_floor", "cfl"):
        setattr(p, k, float(prm[k]))
    p.precision = int(precision)
    p.positivity = int(prm.get("positivity", 0))
    p.flow_index = float(prm.get("flow_index", 1.0))
    p.rate_floor = float(prm.get("rate_floor", 0.0))
    bcs = bcs if bcs else [([0] * 7, [0.0] * 7)]
    if len(bcs) > _lib.MAX_BC:
        raise ValueError("too many boundary descriptors")
    p.n_bc = len(bcs)
    for i, (modes, vals) in enumerate(bcs):
        for s in range(7):
            p.bc[i].mode[s] = int(modes[s])
            p.bc[i].value[s] = float(vals[s])
    return p


class Solver:
    """One DG instance (mesh, order, regularization, parameters) on cuda:0.

    Arrays crossing the boundary are float64 in the [field][element][node]
    layout of include/dg_swe.h."""

    def __init__(self, dim, coords, etov, order, reg, prm, face_bc=None, bcs=None, bed=None,
                 precision=PREC_FP64, device="cuda", stream=None, allocate=True):
        self.L = _lib.lib()
        self.dim, self.order, self.reg, self.precision = int(dim), int(order), int(reg), int(precision)
        self._coords = np.ascontiguousarray(coords, dtype=np.float64).reshape(-1, dim)
        self._etov = np.ascontiguousarray(etov, dtype=np.int32)
        self._face_bc = None if face_bc is None else np.ascontiguousarray(face_bc, dtype=np.int8)
        self._bed = None if bed is None else np.ascontiguousarray(bed, dtype=np.float64)
        m = _lib.Mesh()
        m.dim = self.dim
        m.n_vertices = self._coords.shape[0]
        m.coords = self._coords.ctypes.data
        m.n_elements = self._etov.shape[0]
        m.elem_vertices = self._etov.ctypes.data
        m.face_bc = None if self._face_bc is None else self._face_bc.ctypes.data
        m.bed = None if self._bed is None else self._bed.ctypes.data
        self._params = make_params(prm, bcs, precision)
        ctx = C.c_void_p()
        st = self.L.dg_swe_init(C.byref(m), self.order, self.reg, C.byref(self._params), C.byref(ctx))
        self.ctx = ctx
        if st != DG_OK:
            msg = self.L.dg_swe_last_error(ctx).decode() if ctx.value else ""
            if ctx.value:
                self.L.dg_swe_destroy(ctx)
                self.ctx = C.c_void_p()
            raise DGError(st, msg)
        K, np_, nv, ne, nf = C.c_int64(), C.c_int32(), C.c_int32(), C.c_int32(), C.c_int64()
        self.L.dg_swe_sizes(self.ctx, C.byref(K), C.byref(np_), C.byref(nv), C.byref(ne), C.byref(nf))
        self.K, self.Np, self.nV, self.nE, self.n_faces = K.value, np_.value, nv.value, ne.value, nf.value
        self.workspace = None
        self.stream = None
        if allocate:
            self.allocate(device, stream)

    # -------------------------------------------------------------- setup
    def _check(self, st):
        if st != DG_OK:
            raise DGError(st, self.L.dg_swe_last_error(self.ctx).decode())

    def allocate(self, device="cuda", stream=None):
        torch = _torch()
        nbytes = int(self.L.dg_swe_workspace_size(self.ctx))
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.workspace.device)
        self._check(self.L.dg_swe_set_stream(self.ctx, C.c_void_p(self.stream.cuda_stream)))
        self._check(self.L.dg_swe_set_workspace(self.ctx, C.c_void_p(self.workspace.data_ptr()), nbytes))

    @property
    def workspace_bytes(self):
        return int(self.L.dg_swe_workspace_size(self.ctx))

    def node_coords(self):
        out = np.empty((self.K, self.Np, self.dim))
        self._check(self.L.dg_swe_node_coords(self.ctx, out.ctypes.data))
        return out

    def launches_per_step(self):
        return int(self.L.dg_swe_launches_per_step(self.ctx))

    # -------------------------------------------------------------- state
    def set_state(self, V):
        """V: numpy (nV, K, Np) float64 (host) or a CUDA float64 tensor."""
        if isinstance(V, np.ndarray):
            V = np.ascontiguousarray(V, dtype=np.float64)
            assert V.shape == (self.nV, self.K, self.Np)
            self._check(self.L.dg_swe_set_state(self.ctx, V.ctypes.data, 0))
        else:
            torch = _torch()
            assert V.dtype == torch.float64 and V.is_cuda and V.is_contiguous()
            assert tuple(V.shape) == (self.nV, self.K, self.Np)
            self._check(self.L.dg_swe_set_state(self.ctx, C.c_void_p(V.data_ptr()), 1))

    def get_state(self, with_E=True):
        V = np.empty((self.nV, self.K, self.Np))
        E = np.empty((self.nE, self.K, self.Np)) if with_E else None
        self._check(self.L.dg_swe_get_state(self.ctx, V.ctypes.data,
                                            None if E is None else E.ctypes.data, 0))
        return (V, E) if with_E else V

    def get_state_device(self, V_out):
        self._check(self.L.dg_swe_get_state(self.ctx, C.c_void_p(V_out.data_ptr()), None, 1))

    # -------------------------------------------------------------- compute
    def residual(self, V, with_E=True):
        """dV/dt (and E) for a state; V is a CUDA float64 tensor (nV, K, Np) or
        a numpy array (copied to the device)."""
        torch = _torch()
        if isinstance(V, np.ndarray):
            V = torch.from_numpy(np.ascontiguousarray(V, dtype=np.float64)).to(self.workspace.device)
        dV = torch.empty_like(V)
        E = torch.empty((self.nE, self.K, self.Np), dtype=torch.float64, device=V.device) if with_E else None
        self._check(self.L.dg_swe_residual(self.ctx, C.c_void_p(V.data_ptr()), C.c_void_p(dV.data_ptr()),
                                           None if E is None else C.c_void_p(E.data_ptr())))
        return (dV, E) if with_E else dV

    def step(self, dt=0.0, sync=True):
        if sync:
            out = C.c_double()
            self._check(self.L.dg_swe_step(self.ctx, float(dt), C.byref(out)))
            return out.value
        self._check(self.L.dg_swe_step(self.ctx, float(dt), None))
        return None

    def run(self, n_steps):
        st = _lib.Stats()
        self._check(self.L.dg_swe_run(self.ctx, int(n_steps), 0.0, C.byref(st)))
        return _stats_dict(st)

    def advance(self, n_steps):
        """Enqueue n_steps CFL-limited SSP-RK3 steps (no host synchronization)."""
        self._check(self.L.dg_swe_advance(self.ctx, int(n_steps)))

    def time_kernels(self, n_iter=20):
        """Average ms per launch: estep, face, volume, dt partial, mass partial."""
        ms = (C.c_double * 5)()
        self._check(self.L.dg_swe_time_kernels(self.ctx, int(n_iter), ms))
        return dict(zip(("estep", "face", "volume", "dt", "mass"), list(ms)))

    def sync(self):
        st = _lib.Stats()
        self._check(self.L.dg_swe_sync(self.ctx, C.byref(st)))
        return _stats_dict(st)

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            self.L.dg_swe_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Newton:
    """Backward Euler with a Jacobian-free Newton-Krylov solve on a Solver's
    state (FP64; include/dg_newton.h).  ``run(n)`` advances n steps of size
    dt and returns the solver statistics."""

    def __init__(self, solver, dt, max_newton=10, rtol=1e-10, atol=1e-12, krylov_dim=30, krylov_rtol=1e-6,
                 on_fail_continue=1):
        torch = _torch()
        self.L = solver.L
        self.solver = solver  # the context must outlive this object
        p = _lib.NewtonParams()
        p.dt, p.max_newton, p.rtol, p.atol = float(dt), int(max_newton), float(rtol), float(atol)
        p.krylov_dim, p.krylov_rtol, p.on_fail_continue = int(krylov_dim), float(krylov_rtol), int(on_fail_continue)
        self._p = p
        h = C.c_void_p()
        st = self.L.dg_newton_init(solver.ctx, C.byref(p), C.byref(h))
        if st != DG_OK:
            raise DGError(st, "dg_newton_init")
        self.h = h
        nbytes = int(self.L.dg_newton_workspace_size(h))
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=solver.workspace.device)
        self._check(self.L.dg_newton_set_workspace(h, C.c_void_p(self.workspace.data_ptr()), nbytes))

    def _check(self, st):
        if st != DG_OK:
            raise DGError(st, self.L.dg_newton_last_error(self.h).decode())

    def run(self, n_steps):
        st = _lib.NewtonStats()
        self._check(self.L.dg_newton_run(self.h, int(n_steps), C.byref(st)))
        return dict(steps=st.steps, newton_its=st.newton_its, krylov_its=st.krylov_its,
                    failed_steps=st.failed_steps, t=st.t, last_res=st.last_res, last_newton=st.last_newton,
                    status=st.status)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.L.dg_newton_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stats_dict(st):
    return dict(steps=st.steps, t=st.t, dt_last=st.dt_last, dt_min=st.dt_min, dt_max=st.dt_max,
                mass=st.mass, mass0=st.mass0, status=st.status)


def fma_rate(precision=PREC_FP64, repeats=5, stream=None):
    """Measured fused multiply-add rate (flop/s, FMA = 2) of the current
    GPU's FP64 or FP32 pipe (include/dg_probe.h)."""
    torch = _torch()
    L = _lib.lib()
    scratch = torch.empty(int(L.dg_probe_scratch_bytes()), dtype=torch.uint8, device="cuda")
    s = stream if stream is not None else torch.cuda.current_stream()
    out = C.c_double()
    st = L.dg_probe_fma_rate(int(precision), int(repeats), C.c_void_p(scratch.data_ptr()),
                             C.c_void_p(s.cuda_stream), C.byref(out))
    if st != DG_OK:
        raise DGError(st, "dg_probe_fma_rate failed")
    return out.value


def solver_from_case(case, precision=PREC_FP64, order=None, with_state=True, stream=None):
    """Build a Solver for a synthetic case; sets the initial state sampled at
    the library's own node coordinates."""
    p = case.order if order is None else order
    s = Solver(case.dim, case.coords, case.etov, p, case.params["reg"], case.params,
               face_bc=case.face_bc, bcs=case.bcs, bed=None, precision=precision, allocate=False)
    xyz = s.node_coords()
    V0, bed = case.initial_state(xyz)
    if case.bed_fn is not None:
        s.close()
        s = Solver(case.dim, case.coords, case.etov, p, case.params["reg"], case.params,
                   face_bc=case.face_bc, bcs=case.bcs, bed=bed, precision=precision, allocate=False)
    s.allocate(stream=stream)
    if with_state:
        s.set_state(V0)
    return s, V0, bed


class Batch:
    """Many independent instances advanced together (include/dg_batch.h).

    ``specs`` is a list of dicts with keys dim, coords, etov, order, reg, prm
    and optionally face_bc, bcs, bed.  All instances share ``precision``."""

    def __init__(self, specs, precision=PREC_FP64, device="cuda", stream=None, allocate=True):
        self.L = _lib.lib()
        n = len(specs)
        self.n = n
        self._keep = []
        meshes = (_lib.Mesh * n)()
        params = (_lib.Params * n)()
        orders = (C.c_int * n)()
        regs = (C.c_int * n)()
        self.shapes = []
        for i, sp in enumerate(specs):
            dim = int(sp["dim"])
            coords = np.ascontiguousarray(sp["coords"], dtype=np.float64).reshape(-1, dim)
            etov = np.ascontiguousarray(sp["etov"], dtype=np.int32)
            fb = sp.get("face_bc")
            fb = None if fb is None else np.ascontiguousarray(fb, dtype=np.int8)
            bed = sp.get("bed")
            bed = None if bed is None else np.ascontiguousarray(bed, dtype=np.float64)
            self._keep += [coords, etov, fb, bed]
            m = meshes[i]
            m.dim = dim
            m.n_vertices = coords.shape[0]
            m.coords = coords.ctypes.data
            m.n_elements = etov.shape[0]
            m.elem_vertices = etov.ctypes.data
            m.face_bc = None if fb is None else fb.ctypes.data
            m.bed = None if bed is None else bed.ctypes.data
            params[i] = make_params(sp["prm"], sp.get("bcs"), precision)
            orders[i] = int(sp["order"])
            regs[i] = int(sp["reg"])
            p = int(sp["order"])
            np_ = p + 1 if dim == 1 else (p + 1) * (p + 2) // 2
            self.shapes.append((dim + 1, etov.shape[0], np_))
        ctx = C.c_void_p()
        st = self.L.dg_batch_init(n, meshes, orders, regs, params, C.byref(ctx))
        self.ctx = ctx
        if st != DG_OK:
            msg = self.L.dg_batch_last_error(ctx).decode() if ctx.value else ""
            if ctx.value:
                self.L.dg_batch_destroy(ctx)
                self.ctx = C.c_void_p()
            raise DGError(st, msg)
        self.workspace = None
        if allocate:
            self.allocate(device, stream)

    def allocate(self, device="cuda", stream=None):
        torch = _torch()
        nbytes = int(self.L.dg_batch_workspace_size(self.ctx))
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.workspace.device)
        self._check(self.L.dg_batch_set_stream(self.ctx, C.c_void_p(self.stream.cuda_stream)))
        self._check(self.L.dg_batch_set_workspace(self.ctx, C.c_void_p(self.workspace.data_ptr()), nbytes))

    def _check(self, st):
        if st != DG_OK:
            raise DGError(st, self.L.dg_batch_last_error(self.ctx).decode())

    def set_state(self, i, V):
        if isinstance(V, np.ndarray):
            V = np.ascontiguousarray(V, dtype=np.float64)
            assert V.shape == self.shapes[i]
            self._check(self.L.dg_batch_set_state(self.ctx, int(i), V.ctypes.data, 0))
        else:
            assert tuple(V.shape) == self.shapes[i] and V.is_cuda and V.is_contiguous()
            self._check(self.L.dg_batch_set_state(self.ctx, int(i), C.c_void_p(V.data_ptr()), 1))

    def get_state(self, i):
        V = np.empty(self.shapes[i])
        self._check(self.L.dg_batch_get_state(self.ctx, int(i), V.ctypes.data, 0))
        return V

    def get_state_device(self, i, V_out):
        self._check(self.L.dg_batch_get_state(self.ctx, int(i), C.c_void_p(V_out.data_ptr()), 1))

    def advance(self, n_steps):
        self._check(self.L.dg_batch_advance(self.ctx, int(n_steps)))

    def run(self, n_steps):
        st = (_lib.Stats * self.n)()
        self._check(self.L.dg_batch_run(self.ctx, int(n_steps), st))
        return [_stats_dict(s) for s in st]

    def stats(self):
        st = (_lib.Stats * self.n)()
        self._check(self.L.dg_batch_stats(self.ctx, st))
        return [_stats_dict(s) for s in st]

    def autotune(self, n_iter=10):
        self._check(self.L.dg_batch_autotune(self.ctx, int(n_iter)))
        return self.tiles()

    def time_kernels(self, n_iter=20):
        """Per group: average ms per launch of estep, face, volume, dt."""
        ng = len(self.tiles())
        ms = (C.c_double * (4 * ng))()
        self._check(self.L.dg_batch_time_kernels(self.ctx, int(n_iter), ms, 4 * ng))
        return [dict(zip(("estep", "face", "volume", "dt"), list(ms[4 * g:4 * g + 4]))) for g in range(ng)]

    def tiles(self):
        ng = C.c_int32()
        self.L.dg_batch_tiles(self.ctx, None, 0, C.byref(ng))
        out = (C.c_int32 * (3 * ng.value))()
        self.L.dg_batch_tiles(self.ctx, out, 3 * ng.value, C.byref(ng))
        return [list(out[3 * g:3 * g + 3]) for g in range(ng.value)]

    def set_tiles(self, tiles):
        flat = [int(t) for g in tiles for t in g]
        arr = (C.c_int32 * len(flat))(*flat)
        self._check(self.L.dg_batch_set_tiles(self.ctx, arr, len(flat)))

    def info(self):
        K, D, G_ = C.c_int64(), C.c_int64(), C.c_int32()
        self._check(self.L.dg_batch_info(self.ctx, C.byref(K), C.byref(D), C.byref(G_)))
        return dict(elements=K.value, dofs=D.value, groups=G_.value)

    def set_persistent(self, on=True):
        """One persistent launch per group and step instead of 11 launches
        (include/dg_batch.h: dg_batch_set_persistent)."""
        self._check(self.L.dg_batch_set_persistent(self.ctx, 1 if on else 0))

    def launches_per_step(self):
        return int(self.L.dg_batch_launches_per_step(self.ctx))

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            self.L.dg_batch_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_from_cases(cases, precision=PREC_FP64, stream=None):
    """Batch for synthetic cases; initial states sampled at the library's own
    node coordinates (from host-only single-instance set-ups)."""
    specs, V0s = [], []
    for c in cases:
        probe = Solver(c.dim, c.coords, c.etov, c.order, c.params["reg"], c.params, face_bc=c.face_bc,
                       bcs=c.bcs, precision=precision, allocate=False)
        xyz = probe.node_coords()
        probe.close()
        V0, bed = c.initial_state(xyz)
        specs.append(dict(dim=c.dim, coords=c.coords, etov=c.etov, order=c.order, reg=c.params["reg"],
                          prm=c.params, face_bc=c.face_bc, bcs=c.bcs,
                          bed=bed if c.bed_fn is not None else None))
        V0s.append(V0)
    b = Batch(specs, precision=precision, stream=stream)
    for i, V0 in enumerate(V0s):
        b.set_state(i, V0)
    return b, V0s


class Implicit:
    """Backward Euler + Newton, 1D (include/dg_implicit.h)."""

    def __init__(self, coords, etov, order, reg, prm, dt, m3=-1, face_bc=None, bcs=None, bed=None,
                 max_it=10, on_fail_continue=True, rtol=1e-10, atol=1e-13, xtol=1e-14, device="cuda",
                 stream=None, allocate=True, mixed=False, n_gamma=1, gamma0=0.0):
        self.L = _lib.lib()
        self.order = int(order)
        self._coords = np.ascontiguousarray(coords, dtype=np.float64).reshape(-1, 1)
        self._etov = np.ascontiguousarray(etov, dtype=np.int32)
        self._face_bc = None if face_bc is None else np.ascontiguousarray(face_bc, dtype=np.int8)
        self._bed = None if bed is None else np.ascontiguousarray(bed, dtype=np.float64)
        m = _lib.Mesh()
        m.dim = 1
        m.n_vertices = self._coords.shape[0]
        m.coords = self._coords.ctypes.data
        m.n_elements = self._etov.shape[0]
        m.elem_vertices = self._etov.ctypes.data
        m.face_bc = None if self._face_bc is None else self._face_bc.ctypes.data
        m.bed = None if self._bed is None else self._bed.ctypes.data
        self._params = make_params(prm, bcs, PREC_FP64)
        ip = _lib.ImplicitParams(dt=float(dt), m3=int(m3), max_it=int(max_it),
                                 on_fail_continue=1 if on_fail_continue else 0, rtol=rtol, atol=atol, xtol=xtol,
                                 linear_solver=1 if mixed else 0, n_gamma=int(n_gamma), gamma0=float(gamma0))
        ctx = C.c_void_p()
        st = self.L.dg_implicit_init(C.byref(m), self.order, int(reg), C.byref(self._params), C.byref(ip),
                                     C.byref(ctx))
        self.ctx = ctx
        if st != DG_OK:
            msg = self.L.dg_implicit_last_error(ctx).decode() if ctx.value else ""
            if ctx.value:
                self.L.dg_implicit_destroy(ctx)
                self.ctx = C.c_void_p()
            raise DGError(st, msg)
        self.K = self._etov.shape[0]
        self.Np = self.order + 1
        self.NpE = (self.order if m3 < 0 else int(m3)) + 1
        self.workspace = None
        if allocate:
            torch = _torch()
            nbytes = int(self.L.dg_implicit_workspace_size(self.ctx))
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.workspace.device)
            self._check(self.L.dg_implicit_set_stream(self.ctx, C.c_void_p(self.stream.cuda_stream)))
            self._check(self.L.dg_implicit_set_workspace(self.ctx, C.c_void_p(self.workspace.data_ptr()), nbytes))

    def _check(self, st):
        if st != DG_OK:
            raise DGError(st, self.L.dg_implicit_last_error(self.ctx).decode())

    def node_coords(self):
        out = np.empty((self.K, self.Np, 1))
        self._check(self.L.dg_implicit_node_coords(self.ctx, out.ctypes.data))
        return out

    def set_state(self, V):
        V = np.ascontiguousarray(V, dtype=np.float64)
        assert V.shape == (2, self.K, self.Np)
        self._check(self.L.dg_implicit_set_state(self.ctx, V.ctypes.data, 0))

    def get_state(self):
        V = np.empty((2, self.K, self.Np))
        E = np.empty((self.K, self.NpE))
        self._check(self.L.dg_implicit_get_state(self.ctx, V.ctypes.data, E.ctypes.data, 0))
        return V, E

    def run(self, n_steps):
        st = _lib.ImplicitStats()
        self._check(self.L.dg_implicit_run(self.ctx, int(n_steps), C.byref(st)))
        return dict(steps=st.steps, newton_its=st.newton_its, failed_steps=st.failed_steps, t=st.t,
                    last_its=st.last_its, status=st.status)

    def active_percent(self):
        v = C.c_double()
        self._check(self.L.dg_implicit_active_percent(self.ctx, C.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            self.L.dg_implicit_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def implicit_from_case(case, dt=None, **kw):
    """Implicit integrator for a 1D synthetic case with its state set."""
    probe = Implicit(case.coords, case.etov, case.order, case.params["reg"], case.params, dt or case.dt or 1e-3,
                     m3=case.m3, face_bc=case.face_bc, bcs=case.bcs, allocate=False)
    V0, bed = case.initial_state(probe.node_coords())
    probe.close()
    s = Implicit(case.coords, case.etov, case.order, case.params["reg"], case.params, dt or case.dt,
                 m3=case.m3, face_bc=case.face_bc, bcs=case.bcs,
                 bed=bed if case.bed_fn is not None else None, **kw)
    s.set_state(V0)
    return s, V0
