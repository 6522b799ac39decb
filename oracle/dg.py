"""Discontinuous Galerkin space discretization for the oracle (Sec. 3, Sec. 5).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

For each element e this evaluates, with the fixed quadrature of refelem.py,
  E-step (Eq. WeakForm52):  <N_E, E> = <N_E^-, G_bar . n>_Gamma - <grad N_E, G>_Omega
      with G the velocity components (Eq. Gterm) and the central flux
      G_bar = (G^- + G^+)/2;
  residual (Eq. WeakForm51, without the time term):
      r_V = <N^-, F_bar . n> - <grad N, F> - <N^-, Q_bar . n> + <grad N, Q> - <N, S>
      with F (Eq. Fterm), Q = h sigma / rho (Eq. Qterm), S (Eq. Sterm), the HLL
      flux F_bar (Eq. HLLSolver) and the central Q_bar;
  time derivative: <N, dU/dt> = -r_V with U = (h, h u) (Eq. Uterm), i.e.
      M dh/dt = -r_h and M_h du/dt = -r_u - M_u dh/dt, where
      M_h = <psi, h psi>, M_u = <psi, u psi> (dU/dV of Appendix A); in
      wet/dry mode the explicit stages update the moments <N, U> instead
      (ssp_rk3_step).

Unknowns are modal coefficients of V = (h, u) and E (Sec. 5).  Exterior
(neighbour) values at face points are obtained by mapping the physical point
into the neighbour and evaluating its expansion there; boundary faces use
ghost values (Sec. 5.2): copy (homogeneous Neumann), Dirichlet value, or a
reflecting wall for the velocity (an extension).

Readings where the paper is silent: HLL wave speeds use sqrt(g_c h) in the
face-normal frame; wave speeds and M_h use max(h, h_floor).
"""
import math
import numpy as np

from . import refelem as R
from . import constitutive as C

BC_COPY, BC_DIRICHLET, BC_WALL = 0, 1, 2


class Discretization:
    """Geometry, basis tables and connectivity for one mesh and order."""

    def __init__(self, dim, coords, etov, order, prm, face_bc=None, bcs=None, bed_nodal=None,
                 m3=None):
        self.dim = dim
        self.p = order
        self.m3 = order if (m3 is None or m3 < 0) else m3
        self.prm = dict(prm)
        self.coords = np.asarray(coords, dtype=float).reshape(-1, dim)
        self.etov = np.asarray(etov, dtype=np.int64)
        K = self.K = self.etov.shape[0]
        self.nV = dim + 1
        self.nE = dim * dim
        self.nf = dim + 1
        self.Np = R.n_modes(dim, order)
        self.NpE = R.n_modes(dim, self.m3)
        self.face_bc = (np.zeros((K, self.nf), dtype=np.int64) if face_bc is None
                        else np.asarray(face_bc, dtype=np.int64))
        self.bcs = bcs if bcs is not None else [([0] * 7, [0.0] * 7)]
        g = self.prm["g"]
        a = self.prm["alpha"]
        self.gc = g * math.cos(a)
        self.gs = g * math.sin(a)

        # ---- volume quadrature and basis tables
        self.rq, self.wq = R.vol_rule(dim, order)
        self.Nq = self.wq.size
        self.Phi, dref = R.basis(dim, order, self.rq)
        self.PhiE, drefE = R.basis(dim, self.m3, self.rq)

        # ---- affine geometry
        X = self.coords[self.etov]  # (K, dim+1, dim)
        if dim == 1:
            J = 0.5 * (X[:, 1, 0] - X[:, 0, 0])
            if np.any(J <= 0):
                raise ValueError("1D elements must have x1 > x0")
            self.J = J
            self.Ginv = (1.0 / J).reshape(K, 1, 1)  # dr/dx
        else:
            xr = 0.5 * (X[:, 1] - X[:, 0])
            xs = 0.5 * (X[:, 2] - X[:, 0])
            J = xr[:, 0] * xs[:, 1] - xs[:, 0] * xr[:, 1]
            if np.any(J <= 0):
                raise ValueError("triangles must be counter-clockwise")
            self.J = J
            G = np.empty((K, 2, 2))  # G[k, a, i] = d r_a / d x_i
            G[:, 0, 0] = xs[:, 1] / J
            G[:, 0, 1] = -xs[:, 0] / J
            G[:, 1, 0] = -xr[:, 1] / J
            G[:, 1, 1] = xr[:, 0] / J
            self.Ginv = G
        self.wJ = self.wq[None, :] * self.J[:, None]  # (K, Nq)
        # physical derivatives of basis at volume points: dPhix[i] (K, Nq, Np)
        self.dPhix = [sum(self.Ginv[:, a, i][:, None, None] * dref[a][None] for a in range(dim))
                      for i in range(dim)]
        self.dPhiEx = [sum(self.Ginv[:, a, i][:, None, None] * drefE[a][None] for a in range(dim))
                       for i in range(dim)]
        # mass matrices <psi, psi> (K, Np, Np)
        self.M = np.einsum("kq,qa,qb->kab", self.wJ, self.Phi, self.Phi)
        self.ME = np.einsum("kq,qa,qb->kab", self.wJ, self.PhiE, self.PhiE)

        # ---- faces
        fref, self.tf, self.wf = R.face_points_ref(dim, order)
        self.Nfq = self.wf.size
        self.Phif = np.stack([R.basis(dim, order, fref[f])[0] for f in range(self.nf)])
        self.PhiEf = np.stack([R.basis(dim, self.m3, fref[f])[0] for f in range(self.nf)])
        self.n = np.empty((K, self.nf, dim))
        self.sJ = np.empty((K, self.nf))
        if dim == 1:
            self.n[:, 0, 0] = -1.0
            self.n[:, 1, 0] = 1.0
            self.sJ[:] = 1.0
        else:
            for f in range(3):
                t = X[:, (f + 1) % 3] - X[:, f]
                ln = np.sqrt((t ** 2).sum(axis=1))
                self.n[:, f, 0] = t[:, 1] / ln
                self.n[:, f, 1] = -t[:, 0] / ln
                self.sJ[:, f] = 0.5 * ln
        # physical face points
        self.xf = np.stack([self.map_to_phys(fref[f]) for f in range(self.nf)], axis=1)
        # connectivity by shared vertices
        keys = {}
        for e in range(K):
            for f in range(self.nf):
                key = self._face_key(e, f)
                keys.setdefault(key, []).append((e, f))
        self.nbr = -np.ones((K, self.nf), dtype=np.int64)
        for lst in keys.values():
            if len(lst) == 2:
                (e1, f1), (e2, f2) = lst
                self.nbr[e1, f1] = e2
                self.nbr[e2, f2] = e1
            elif len(lst) > 2:
                raise ValueError("non-manifold face")
        # neighbour basis values at this element's face points
        self.Phinb = np.zeros((K, self.nf, self.Nfq, self.Np))
        self.PhiEnb = np.zeros((K, self.nf, self.Nfq, self.NpE))
        for e in range(K):
            for f in range(self.nf):
                e2 = self.nbr[e, f]
                if e2 < 0:
                    continue
                rr = self.map_to_ref(e2, self.xf[e, f])
                self.Phinb[e, f] = R.basis(dim, order, rr)[0]
                self.PhiEnb[e, f] = R.basis(dim, self.m3, rr)[0]
        self.nbr_safe = np.where(self.nbr >= 0, self.nbr, np.arange(K)[:, None])
        self.is_bnd = self.nbr < 0

        # ---- nodes, Vandermonde, bed
        self.rnodes = R.ref_nodes(dim, order)
        self.Vand = R.basis(dim, order, self.rnodes)[0]
        self.node_xyz = self.map_to_phys(self.rnodes)  # (K, Np, dim)
        if bed_nodal is None:
            self.Hh = np.zeros((K, self.Np))
        else:
            self.Hh = self.to_modal(np.asarray(bed_nodal, dtype=float))
        self.dHq = np.stack([np.einsum("kqa,ka->kq", self.dPhix[i], self.Hh)
                             for i in range(dim)])  # (dim, K, Nq)
        # element size for the time-step bound: length (1D), 2 x inradius (2D)
        if dim == 1:
            self.dx = 2.0 * self.J
        else:
            area = 2.0 * self.J  # reference triangle has area 2
            perim = 2.0 * self.sJ.sum(axis=1)
            self.dx = 4.0 * area / perim

    # ------------------------------------------------------------ helpers
    def _face_key(self, e, f):
        if self.dim == 1:
            return (int(self.etov[e, f]),)
        a, b = int(self.etov[e, f]), int(self.etov[e, (f + 1) % 3])
        return (min(a, b), max(a, b))

    def map_to_phys(self, rpts):
        """Reference points (n, dim) -> physical points (K, n, dim)."""
        X = self.coords[self.etov]
        rpts = np.atleast_2d(rpts)
        if self.dim == 1:
            lam = 0.5 * (1.0 + rpts[:, 0])
            return (X[:, 0, None, :] * (1 - lam)[None, :, None]
                    + X[:, 1, None, :] * lam[None, :, None])
        l1 = 0.5 * (1.0 + rpts[:, 0])
        l2 = 0.5 * (1.0 + rpts[:, 1])
        l0 = 1.0 - l1 - l2
        return (X[:, 0, None, :] * l0[None, :, None] + X[:, 1, None, :] * l1[None, :, None]
                + X[:, 2, None, :] * l2[None, :, None])

    def map_to_ref(self, e, xpts):
        """Physical points (n, dim) -> reference coordinates in element e."""
        X = self.coords[self.etov[e]]
        if self.dim == 1:
            lam = (xpts[:, 0] - X[0, 0]) / (X[1, 0] - X[0, 0])
            return (2.0 * lam - 1.0).reshape(-1, 1)
        A = np.stack([X[1] - X[0], X[2] - X[0]], axis=1)  # columns
        lam = np.linalg.solve(A, (xpts - X[0]).T).T
        return 2.0 * lam - 1.0

    def to_modal(self, nodal):
        """Nodal values (..., K, Np) at the equispaced nodes -> modal coefficients."""
        return np.einsum("ab,...kb->...ka", np.linalg.inv(self.Vand), nodal)

    def to_nodal(self, modal):
        return np.einsum("ab,...kb->...ka", self.Vand, modal)

    def E_to_nodal(self, Eh):
        """E modal (nE, K, NpE) -> values at the equispaced nodes of degree p."""
        PhiE_nodes = R.basis(self.dim, self.m3, self.rnodes)[0]
        return np.einsum("ab,...kb->...ka", PhiE_nodes, Eh)

    def E_to_modal(self, En):
        """E nodal at the degree-p nodes (requires m3 == p)."""
        assert self.m3 == self.p
        return self.to_modal(En)

    # ------------------------------------------------------------ traces
    def traces(self, Vh, Eh=None):
        """Interior and exterior values at face points.

        Returns Vm, Vp (nV, K, nf, Nfq) and, if Eh is given, Em, Ep (nE, ...)."""
        Vm = np.einsum("fqa,vka->vkfq", self.Phif, Vh)
        Vnb = Vh[:, self.nbr_safe]  # (nV, K, nf, Np)
        Vp = np.einsum("kfqa,vkfa->vkfq", self.Phinb, Vnb)
        Em = Ep = None
        if Eh is not None:
            Em = np.einsum("fqa,vka->vkfq", self.PhiEf, Eh)
            Enb = Eh[:, self.nbr_safe]
            Ep = np.einsum("kfqa,vkfa->vkfq", self.PhiEnb, Enb)
        Vp, Ep = self.ghosts(Vm, Vp, Em, Ep)
        return Vm, Vp, Em, Ep

    def ghosts(self, Vm, Vp, Em, Ep):
        """Exterior values at boundary faces (Sec. 5.2)."""
        Vp = Vp.copy()
        if Ep is not None:
            Ep = Ep.copy()
        d = self.dim
        for (k, f) in zip(*np.nonzero(self.is_bnd)):
            modes, vals = self.bcs[self.face_bc[k, f]]
            for v in range(self.nV):
                Vp[v, k, f] = Vm[v, k, f] if modes[v] != BC_DIRICHLET else vals[v]
            if any(modes[1 + j] == BC_WALL for j in range(d)):
                nn = self.n[k, f]
                un = sum(Vm[1 + j, k, f] * nn[j] for j in range(d))
                for j in range(d):
                    Vp[1 + j, k, f] = Vm[1 + j, k, f] - 2.0 * un * nn[j]
            if Ep is not None:
                for c in range(self.nE):
                    slot = self.nV + c
                    Ep[c, k, f] = Em[c, k, f] if modes[slot] != BC_DIRICHLET else vals[slot]
        return Vp, Ep

    # ------------------------------------------------------------ E-step
    def e_step(self, Vh):
        """E = grad u in the weak sense of Eq. WeakForm52 (modal, (nE, K, NpE))."""
        d = self.dim
        uq = np.einsum("qa,jka->jkq", self.Phi, Vh[1:])
        Vm, Vp, _, _ = self.traces(Vh)
        Gbar = 0.5 * (Vm[1:] + Vp[1:])  # (d, K, nf, Nfq)
        rhs = np.empty((self.nE, self.K, self.NpE))
        for i in range(d):
            for j in range(d):
                vol = -np.einsum("kq,kqa,kq->ka", self.wJ, self.dPhiEx[i], uq[j])
                face = np.einsum("q,kf,fqa,kf,kfq->ka", self.wf, self.sJ, self.PhiEf,
                                 self.n[:, :, i], Gbar[j])
                rhs[d * i + j] = vol + face
        return np.linalg.solve(self.ME[None], rhs[..., None])[..., 0]

    # ------------------------------------------------------------ pointwise physics
    def flux_F(self, V):
        """F_i (Eq. Fterm) as (dim, nV, ...) for V = (h, u_1[, u_2])."""
        d = self.dim
        h = V[0]
        u = V[1:]
        F = np.empty((d, self.nV) + h.shape)
        for i in range(d):
            F[i, 0] = h * u[i]
            for j in range(d):
                F[i, 1 + j] = h * u[i] * u[j]
            F[i, 1 + i] += 0.5 * self.gc * h * h
        return F

    def flux_Q(self, V, E):
        """Q_i = h sigma_{j i} / rho in momentum rows (Eq. Qterm), (dim, nV, ...)."""
        d = self.dim
        sig = C.stress(E, d, self.prm)
        h = V[0]
        Q = np.zeros((d, self.nV) + h.shape)
        for i in range(d):
            for j in range(d):
                Q[i, 1 + j] = h * sig[j, i] / self.prm["rho"]
        return Q

    def hll(self, Vm, Vp, n):
        """HLL normal flux F_bar . n (Eq. HLLSolver) in the face-normal frame."""
        d = self.dim
        hf = self.prm["h_floor"]
        hm, hp = Vm[0], Vp[0]
        unm = sum(Vm[1 + j] * n[j] for j in range(d))
        unp = sum(Vp[1 + j] * n[j] for j in range(d))
        cm = np.sqrt(self.gc * np.maximum(hm, hf))
        cp = np.sqrt(self.gc * np.maximum(hp, hf))
        SL = np.minimum(unm - cm, unp - cp)
        SR = np.maximum(unm + cm, unp + cp)

        def fn(V, h, un):
            out = np.empty((self.nV,) + h.shape)
            out[0] = h * un
            for j in range(d):
                out[1 + j] = h * V[1 + j] * un + 0.5 * self.gc * h * h * n[j]
            return out

        def cons(V, h):
            out = np.empty((self.nV,) + h.shape)
            out[0] = h
            for j in range(d):
                out[1 + j] = h * V[1 + j]
            return out

        Fm, Fp = fn(Vm, hm, unm), fn(Vp, hp, unp)
        Um, Up = cons(Vm, hm), cons(Vp, hp)
        mid = (SR * Fm - SL * Fp + SL * SR * (Up - Um)) / (SR - SL)
        return np.where(SL >= 0, Fm, np.where(SR <= 0, Fp, mid))

    # ------------------------------------------------------------ residual
    def spatial_residual(self, Vh, Eh):
        """r_V of Eq. WeakForm51 without the time term, (nV, K, Np)."""
        d = self.dim
        Vq = np.einsum("qa,vka->vkq", self.Phi, Vh)
        Eq = np.einsum("qa,cka->ckq", self.PhiE, Eh)
        F = self.flux_F(Vq)
        Q = self.flux_Q(Vq, Eq)
        S = np.zeros((self.nV, self.K, self.Nq))
        h = Vq[0]
        S[1] = -self.gs * h - self.gc * h * self.dHq[0]
        if d == 2:
            S[2] = -self.gc * h * self.dHq[1]
        r = np.zeros((self.nV, self.K, self.Np))
        for i in range(d):
            r += np.einsum("kq,kqa,vkq->vka", self.wJ, self.dPhix[i], Q[i] - F[i])
        r -= np.einsum("kq,qa,vkq->vka", self.wJ, self.Phi, S)
        Vm, Vp, Em, Ep = self.traces(Vh, Eh)
        nn = np.moveaxis(self.n, 2, 0)[:, :, :, None]  # (d, K, nf, 1)
        Fn = self.hll(Vm, Vp, nn)
        Qm = self.flux_Q(Vm, Em)
        Qp = self.flux_Q(Vp, Ep)
        Qn = 0.5 * sum((Qm[i] + Qp[i]) * nn[i][None] for i in range(d))
        r += np.einsum("q,kf,fqa,vkfq->vka", self.wf, self.sJ, self.Phif, Fn - Qn)
        return r

    def mass_solve(self, Vh, r):
        """Solve <N, (dU/dV) N> dV/dt = -r (dU/dV of Appendix A)."""
        d = self.dim
        dV = np.empty_like(r)
        dV[0] = np.linalg.solve(self.M, -r[0][..., None])[..., 0]
        Vq = np.einsum("qa,vka->vkq", self.Phi, Vh)
        hq = np.maximum(Vq[0], self.prm["h_floor"])
        hdq = np.einsum("qa,ka->kq", self.Phi, dV[0])
        Mh = np.einsum("kq,kq,qa,qb->kab", self.wJ, hq, self.Phi, self.Phi)
        for j in range(d):
            rhs = -r[1 + j] - np.einsum("kq,kq,kq,qa->ka", self.wJ, Vq[1 + j], hdq, self.Phi)
            dV[1 + j] = np.linalg.solve(Mh, rhs[..., None])[..., 0]
        return dV

    def rhs(self, Vh):
        """dV/dt (modal) and E for state Vh."""
        Eh = self.e_step(Vh)
        r = self.spatial_residual(Vh, Eh)
        return self.mass_solve(Vh, r), Eh

    # ------------------------------------------------------------ time stepping
    def max_diffusivity(self):
        return (4.0 * C.max_viscosity(self.prm) + C.max_slope(self.prm)) / self.prm["rho"]

    def stable_dt(self, Vh):
        """Explicit step bound (reading of the paper's silence on explicit
        stepping): per element
            dt_e = cfl * dx_e / ((2p+1) lam_e + (2p+1)^2 * 2 nu / dx_e)
        with lam_e the largest |u| + sqrt(g_c max(h, h_floor)) over the
        element's nodes and nu = (4 eta_max + max d sigma_B/dE) / rho (eta_max
        the largest viscous slope / 4: eta, or the Herschel-Bulkley
        eta rate_floor^(n-1)); dt is the
        minimum over elements."""
        Vn = self.to_nodal(Vh)
        sp = np.sqrt(sum(Vn[1 + j] ** 2 for j in range(self.dim)))
        lam = (sp + np.sqrt(self.gc * np.maximum(Vn[0], self.prm["h_floor"]))).max(axis=1)
        q = 2 * self.p + 1
        nu = self.max_diffusivity()
        dte = self.prm["cfl"] * self.dx / (q * lam + q * q * 2.0 * nu / self.dx)
        return float(dte.min())

    def ssp_rk3_step(self, Vh, dt=None):
        """One Shu-Osher SSP-RK3 step (explicit integrator for the
        benchmark workloads; the paper itself integrates implicitly).
        Without prm["positivity"] the stages are taken on V = (h, u) with
        dV/dt from rhs (method of lines through dU/dV).  With it (wet/dry
        fronts) they are taken on the moments <N, U(V)> of U = (h, h u), the
        quantity whose difference the paper's time term (Eq. WeakForm7)
        holds: each Euler substep is <N, U(V')> = <N, U(V)> - dt r_V(V), the
        stage results are the same convex combinations of moments, and V is
        recovered from the moments by recover_from_moments (depth limited
        before the velocity is solved for).  The two forms agree to O(dt^2)
        per step; only the second stays finite where the depth at the start
        of a stage is zero, since it divides the new momentum by the new
        depth instead of the momentum change by the old one."""
        if dt is None:
            dt = self.stable_dt(Vh)
        if self.prm.get("positivity", 0):
            m0 = self.moments(Vh)
            V1 = self.recover_from_moments(m0 - dt * self.residual(Vh))
            V2 = self.recover_from_moments(0.75 * m0 + 0.25 * (self.moments(V1) - dt * self.residual(V1)))
            V3 = self.recover_from_moments(m0 / 3.0 + 2.0 / 3.0 * (self.moments(V2) - dt * self.residual(V2)))
            return V3, dt
        k1, _ = self.rhs(Vh)
        V1 = Vh + dt * k1
        k2, _ = self.rhs(V1)
        V2 = 0.75 * Vh + 0.25 * (V1 + dt * k2)
        k3, _ = self.rhs(V2)
        return Vh / 3.0 + 2.0 / 3.0 * (V2 + dt * k3), dt

    def residual(self, Vh):
        """r_V of Eq. WeakForm51 (without the time term) with E from the E-step."""
        return self.spatial_residual(Vh, self.e_step(Vh))

    def moments(self, Vh):
        """<N, U(V)> per element: the test-function moments of the
        conservative unknowns U = (h, h u_1, ..., h u_d) (Eq. Uterm), with the
        products h u_j formed at the volume quadrature points; (nV, K, Np)."""
        Vq = np.einsum("qa,vka->vkq", self.Phi, Vh)
        m = np.empty_like(Vh)
        m[0] = np.einsum("kq,qa,kq->ka", self.wJ, self.Phi, Vq[0])
        for j in range(self.dim):
            m[1 + j] = np.einsum("kq,qa,kq->ka", self.wJ, self.Phi, Vq[0] * Vq[1 + j])
        return m

    def recover_from_moments(self, m):
        """V from moments m = <N, U>: h from M h = m_h; h through the depth
        limiter (positivity_limit's scaling); u_j from M_h u_j = m_u_j with
        M_h = <psi, max(h, h_floor) psi> of the limited depth; u = 0 in
        elements whose mean depth is below h_floor."""
        V = np.empty_like(m)
        V[0] = np.linalg.solve(self.M, m[0][..., None])[..., 0]
        V[0], hbar = self._limit_depth(V[0])
        hq = np.maximum(np.einsum("qa,ka->kq", self.Phi, V[0]), self.prm["h_floor"])
        Mh = np.einsum("kq,kq,qa,qb->kab", self.wJ, hq, self.Phi, self.Phi)
        for j in range(self.dim):
            V[1 + j] = np.linalg.solve(Mh, m[1 + j][..., None])[..., 0]
        dry = hbar < self.prm["h_floor"]
        for j in range(self.dim):
            V[1 + j][dry] = 0.0
        return V

    # ------------------------------------------------------------ wet/dry (extension)
    def check_points(self, Vh_field):
        """Values of one field at every point the depth limiter checks:
        the equispaced nodes, the volume quadrature points and the face
        quadrature points of every face; shape (K, n_points)."""
        at_nodes = self.to_nodal(Vh_field)
        at_vol = np.einsum("qa,ka->kq", self.Phi, Vh_field)
        at_faces = np.einsum("fqa,ka->kfq", self.Phif, Vh_field).reshape(self.K, -1)
        return np.concatenate([at_nodes, at_vol, at_faces], axis=1)

    def positivity_limit(self, Vh):
        """Depth limiter for wet/dry fronts.  Dry beds are left to future work
        in the paper (Sec. 7); this is the scaling limiter of Zhang and Shu
        (J. Comput. Phys. 229, 2010) applied to h, with the velocity set to
        zero in dry elements.  Per element, with hbar the cell average of h
        and m its minimum over check_points:
          hbar <= 0:        h = 0;
          m < 0 < hbar:     h <- hbar + theta (h - hbar), theta = hbar / (hbar - m)
                            (the scaled polynomial has minimum 0 and the same mean);
          otherwise:        h unchanged;
        and u = 0 in elements with hbar < h_floor."""
        V = Vh.copy()
        V[0], hbar = self._limit_depth(Vh[0])
        dry = hbar < self.prm["h_floor"]
        for j in range(self.dim):
            V[1 + j] = np.where(dry[:, None], 0.0, Vh[1 + j])
        return V

    def _limit_depth(self, h):
        """The depth part of positivity_limit: (limited h, cell averages)."""
        w = self.wJ
        hbar = np.einsum("kq,kq->k", w, np.einsum("qa,ka->kq", self.Phi, h)) / w.sum(axis=1)
        m = self.check_points(h).min(axis=1)
        hn = self.to_nodal(h)
        with np.errstate(divide="ignore", invalid="ignore"):
            theta = np.where(m < 0.0, hbar / (hbar - m), 1.0)
        scaled = hbar[:, None] + theta[:, None] * (hn - hbar[:, None])
        hn_new = np.where((hbar <= 0.0)[:, None], 0.0, np.where((m < 0.0)[:, None], scaled, hn))
        changed = (hbar <= 0.0) | (m < 0.0)
        return np.where(changed[:, None], self.to_modal(hn_new), h), hbar

    def total_mass(self, Vh):
        """Sum over elements of the integral of h (compensated summation)."""
        per = np.einsum("kq,qa,ka->k", self.wJ, self.Phi, Vh[0])
        return math.fsum(per.tolist())

    def eval_at_quad(self, Vh):
        return np.einsum("qa,vka->vkq", self.Phi, Vh)
