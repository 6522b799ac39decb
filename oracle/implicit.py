"""Backward Euler + Newton-Raphson for the 1D scheme (Sec. 5.1, Appendix A).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Unknowns per element e (modal coefficients, Sec. 5): x_e = [h_e, u_e, E_e]
with h, u of degree p and E of degree m3.  The residual at time level k is
Eq. WeakForm7:
  R_V = (1/dt) <N_V, U(V^k) - U(V^{k-1})> + <N_V^-, F_bar.n> - <dN_V/dx, F>
        - <N_V^-, Q_bar.n> + <dN_V/dx, Q> - <N_V, S>
  R_E = <N_E, E> - <N_E^-, G_bar.n> + <dN_E/dx, G>
Newton (Eq. Newton): J dx = -R with the tangent blocks of Appendix A: dU/dV,
dF/dV, the HLL flux derivative with the wave speeds S_L, S_R held fixed,
dQ/dV = sigma/rho (h column), dQ/dE = h sigma'(E)/rho, dS/dV, dG/dV, and
dR_E/dE = <N_E, N_E>.  Boundary ghost values (Sec. 5.2) enter through
dV+/dV- (copy: 1, Dirichlet: 0, wall on u: -1).

The global Jacobian is assembled densely and solved with a library solve
(numpy); at most 10 Newton iterations per step (Sec. 6).  Stopping rule (the
paper does not give one): ||R||_2 <= rtol ||R^0||_2, or ||R||_2 <= atol, or
||dx||_inf <= xtol (1 + ||x||_inf).
"""
import numpy as np

from . import constitutive as C
from .dg import Discretization, BC_COPY, BC_DIRICHLET, BC_WALL


class Implicit1D:
    def __init__(self, disc: Discretization, dt):
        assert disc.dim == 1, "the implicit integrator is one-dimensional"
        self.d = disc
        self.dt = float(dt)
        d = disc
        self.Np, self.NpE, self.K = d.Np, d.NpE, d.K
        self.nb = 2 * d.Np + d.NpE
        self.prm = d.prm
        self.gc, self.gs = d.gc, d.gs
        self.rho = self.prm["rho"]
        # derivative of basis at volume points (K, Nq, Np) and E basis
        self.dPhi = d.dPhix[0]
        self.dPhiE = d.dPhiEx[0]

    # ------------------------------------------------------------ packing
    def pack(self, Vh, Eh):
        return np.concatenate([Vh[0], Vh[1], Eh[0]], axis=1)  # (K, nb)

    def unpack(self, X):
        Np = self.Np
        return np.stack([X[:, :Np], X[:, Np:2 * Np]]), X[:, 2 * Np:][None]

    # ------------------------------------------------------------ residual
    def old_term(self, Vh_old):
        """<N_V, U(V^{k-1})> per element, (2, K, Np)."""
        d = self.d
        Vq = np.einsum("qa,vka->vkq", d.Phi, Vh_old)
        U = np.stack([Vq[0], Vq[0] * Vq[1]])
        return np.einsum("kq,qa,vkq->vka", d.wJ, d.Phi, U)

    def face_states(self, Vh, Eh):
        d = self.d
        Vm, Vp, Em, Ep = d.traces(Vh, Eh)
        return Vm[:, :, :, 0], Vp[:, :, :, 0], Em[:, :, :, 0], Ep[:, :, :, 0]  # (nV|nE, K, 2)

    def speeds(self, Vm, Vp, n):
        hf = self.prm["h_floor"]
        unm, unp = Vm[1] * n, Vp[1] * n
        cm = np.sqrt(self.gc * np.maximum(Vm[0], hf))
        cp = np.sqrt(self.gc * np.maximum(Vp[0], hf))
        return np.minimum(unm - cm, unp - cp), np.maximum(unm + cm, unp + cp)

    def hll_frozen(self, Vm, Vp, n, SL, SR):
        """HLL flux F_bar.n (Eq. HLLSolver) with given wave speeds."""
        def fn(V):
            h, u = V
            return np.stack([h * u * n, (h * u * u + 0.5 * self.gc * h * h) * n])

        def cons(V):
            return np.stack([V[0], V[0] * V[1]])

        Fm, Fp = fn(Vm), fn(Vp)
        mid = (SR * Fm - SL * Fp + SL * SR * (cons(Vp) - cons(Vm))) / (SR - SL)
        return np.where(SL >= 0, Fm, np.where(SR <= 0, Fp, mid))

    def residual(self, X, Uold, speeds=None):
        """R (K, nb) at X; ``speeds`` = (S_L, S_R) to hold the HLL speeds fixed."""
        d = self.d
        Vh, Eh = self.unpack(X)
        Np = self.Np
        Vq = np.einsum("qa,vka->vkq", d.Phi, Vh)
        Eq = np.einsum("qa,cka->ckq", d.PhiE, Eh)
        h, u, e = Vq[0], Vq[1], Eq[0]
        sig = C.stress(Eq, 1, self.prm)[0, 0]
        U = np.stack([h, h * u])
        F = np.stack([h * u, h * u * u + 0.5 * self.gc * h * h])
        Q = np.stack([np.zeros_like(h), h * sig / self.rho])
        S = np.stack([np.zeros_like(h), -self.gs * h - self.gc * h * d.dHq[0]])
        R = np.zeros((self.K, self.nb))
        RV = (np.einsum("kq,qa,vkq->vka", d.wJ, d.Phi, U) - Uold) / self.dt
        RV += np.einsum("kq,kqa,vkq->vka", d.wJ, self.dPhi, Q - F)
        RV -= np.einsum("kq,qa,vkq->vka", d.wJ, d.Phi, S)
        RE = np.einsum("kq,qc,kq->kc", d.wJ, d.PhiE, e) + np.einsum("kq,kqc,kq->kc", d.wJ, self.dPhiE, u)
        Vm, Vp, Em, Ep = self.face_states(Vh, Eh)
        n = d.n[:, :, 0]
        SL, SR = self.speeds(Vm, Vp, n) if speeds is None else speeds
        Fb = self.hll_frozen(Vm, Vp, n, SL, SR)
        sm = C.stress(Em, 1, self.prm)[0, 0]
        sp = C.stress(Ep, 1, self.prm)[0, 0]
        Qb = 0.5 * (Vm[0] * sm + Vp[0] * sp) / self.rho * n
        Gb = 0.5 * (Vm[1] + Vp[1]) * n
        phif = d.Phif[:, 0, :]   # (2 faces, Np)
        phiEf = d.PhiEf[:, 0, :]
        RV[0] += np.einsum("fa,kf->ka", phif, Fb[0])
        RV[1] += np.einsum("fa,kf->ka", phif, Fb[1] - Qb)
        RE -= np.einsum("fc,kf->kc", phiEf, Gb)
        R[:, :Np] = RV[0]
        R[:, Np:2 * Np] = RV[1]
        R[:, 2 * Np:] = RE
        return R

    # ------------------------------------------------------------ Jacobian
    def jacobian(self, X):
        """Dense dR/dX (K*nb, K*nb) from the Appendix A tangent terms, with
        the HLL wave speeds held fixed at their values at X."""
        d = self.d
        K, Np, NpE, nb = self.K, self.Np, self.NpE, self.nb
        Vh, Eh = self.unpack(X)
        Vq = np.einsum("qa,vka->vkq", d.Phi, Vh)
        Eq = np.einsum("qa,cka->ckq", d.PhiE, Eh)
        h, u, e = Vq[0], Vq[1], Eq[0]
        sig = C.stress(Eq, 1, self.prm)[0, 0]
        dsig = C.dsigma_dE_1d(e, self.prm)
        J = np.zeros((K * nb, K * nb))
        ih = lambda k: slice(k * nb, k * nb + Np)  # noqa: E731
        iu = lambda k: slice(k * nb + Np, k * nb + 2 * Np)  # noqa: E731
        iE = lambda k: slice(k * nb + 2 * Np, k * nb + nb)  # noqa: E731
        Phi, PhiE = d.Phi, d.PhiE
        for k in range(K):
            w = d.wJ[k]
            dP, dPE = self.dPhi[k], self.dPhiE[k]

            def vol(test, coef, trial):
                return np.einsum("q,qa,q,qb->ab", w, test, coef, trial)
            # time term (1/dt) <N, dU/dV N>
            J[ih(k), ih(k)] += vol(Phi, np.ones_like(h[k]), Phi) / self.dt
            J[iu(k), ih(k)] += vol(Phi, u[k], Phi) / self.dt
            J[iu(k), iu(k)] += vol(Phi, h[k], Phi) / self.dt
            # -<dN/dx, dF/dV N>
            J[ih(k), ih(k)] -= vol(dP, u[k], Phi)
            J[ih(k), iu(k)] -= vol(dP, h[k], Phi)
            J[iu(k), ih(k)] -= vol(dP, u[k] ** 2 + self.gc * h[k], Phi)
            J[iu(k), iu(k)] -= vol(dP, 2 * h[k] * u[k], Phi)
            # +<dN/dx, dQ/dV N>, +<dN/dx, dQ/dE N_E>
            J[iu(k), ih(k)] += vol(dP, sig[k] / self.rho, Phi)
            J[iu(k), iE(k)] += vol(dP, h[k] * dsig[k] / self.rho, PhiE)
            # -<N, dS/dV N>
            J[iu(k), ih(k)] -= vol(Phi, -self.gs - self.gc * d.dHq[0][k], Phi)
            # R_E: <N_E, N_E> and +<dN_E/dx, dG/du N>
            J[iE(k), iE(k)] += vol(PhiE, np.ones_like(h[k]), PhiE)
            J[iE(k), iu(k)] += vol(dPE, np.ones_like(h[k]), Phi)
        # faces
        Vm, Vp, Em, Ep = self.face_states(Vh, Eh)
        n = d.n[:, :, 0]
        SL, SR = self.speeds(Vm, Vp, n)
        for k in range(K):
            for f in range(2):
                nn = n[k, f]
                hm, um, hp, up = Vm[0, k, f], Vm[1, k, f], Vp[0, k, f], Vp[1, k, f]
                em, ep = Em[0, k, f], Ep[0, k, f]
                sl, sr = SL[k, f], SR[k, f]
                dFn_m = np.array([[um * nn, hm * nn], [(um * um + self.gc * hm) * nn, 2 * hm * um * nn]])
                dFn_p = np.array([[up * nn, hp * nn], [(up * up + self.gc * hp) * nn, 2 * hp * up * nn]])
                dU_m = np.array([[1.0, 0.0], [um, hm]])
                dU_p = np.array([[1.0, 0.0], [up, hp]])
                if sl >= 0:
                    A_m, A_p = dFn_m, np.zeros((2, 2))
                elif sr <= 0:
                    A_m, A_p = np.zeros((2, 2)), dFn_p
                else:
                    A_m = (sr * dFn_m - sl * sr * dU_m) / (sr - sl)
                    A_p = (-sl * dFn_p + sl * sr * dU_p) / (sr - sl)
                # -Q_bar.n on the u row
                sm = C.stress(np.array([[em]]), 1, self.prm)[0, 0][0]
                sp = C.stress(np.array([[ep]]), 1, self.prm)[0, 0][0]
                dsm = C.dsigma_dE_1d(np.array([em]), self.prm)[0]
                dsp = C.dsigma_dE_1d(np.array([ep]), self.prm)[0]
                A_m = A_m.copy()
                A_p = A_p.copy()
                A_m[1, 0] -= 0.5 * sm / self.rho * nn
                A_p[1, 0] -= 0.5 * sp / self.rho * nn
                BE_m = -0.5 * hm * dsm / self.rho * nn   # d(R_u flux)/dE-
                BE_p = -0.5 * hp * dsp / self.rho * nn
                GV_m = -0.5 * nn                          # d(R_E flux)/du-
                GV_p = -0.5 * nn
                phi = d.Phif[f, 0, :]
                phiE = d.PhiEf[f, 0, :]
                k2 = d.nbr[k, f]
                if k2 >= 0:
                    pts_p = d.Phinb[k, f, 0, :]
                    ptsE_p = d.PhiEnb[k, f, 0, :]
                    tgt = k2
                    dVp = np.eye(2)
                    dEp = 1.0
                else:
                    modes, _ = d.bcs[d.face_bc[k, f]]
                    pts_p, ptsE_p, tgt = phi, phiE, k
                    dVp = np.diag([0.0 if modes[0] == BC_DIRICHLET else 1.0,
                                   0.0 if modes[1] == BC_DIRICHLET else (-1.0 if modes[1] == BC_WALL else 1.0)])
                    dEp = 0.0 if modes[2] == BC_DIRICHLET else 1.0
                    A_p = A_p @ dVp
                    BE_p *= dEp
                    GV_p *= dVp[1, 1]
                # rows h, u of element k
                rows = [ih(k), iu(k)]
                colm = [ih(k), iu(k)]
                colp = [ih(tgt), iu(tgt)]
                for r in range(2):
                    for c in range(2):
                        J[rows[r], colm[c]] += np.outer(phi, phi) * A_m[r, c]
                        J[rows[r], colp[c]] += np.outer(phi, pts_p) * A_p[r, c]
                J[iu(k), iE(k)] += np.outer(phi, phiE) * BE_m
                J[iu(k), iE(tgt)] += np.outer(phi, ptsE_p) * BE_p
                J[iE(k), iu(k)] += np.outer(phiE, phi) * GV_m
                J[iE(k), iu(tgt)] += np.outer(phiE, pts_p) * GV_p
        return J

    # ------------------------------------------------------------ Newton
    def initial_E(self, Vh):
        """E consistent with V: solve R_E = 0 for E (it is linear in E)."""
        return self.d.e_step(Vh)

    def step(self, X, max_it=10, rtol=1e-10, atol=1e-13, xtol=1e-14, Vh_old=None):
        """One backward-Euler step from X (K, nb); returns (X_new, iterations,
        converged).  ``Vh_old`` overrides the previous time level (continuation
        stages start from a later iterate)."""
        if Vh_old is None:
            Vh_old, _ = self.unpack(X)
        Uold = self.old_term(Vh_old)
        Xk = X.copy()
        R = self.residual(Xk, Uold)
        r0 = np.linalg.norm(R)
        for it in range(1, max_it + 1):
            if np.linalg.norm(R) <= atol:
                return Xk, it - 1, True
            Jm = self.jacobian(Xk)
            dx = np.linalg.solve(Jm, -R.ravel()).reshape(Xk.shape)
            Xk = Xk + dx
            R = self.residual(Xk, Uold)
            rn = np.linalg.norm(R)
            if rn <= rtol * r0 or rn <= atol or np.abs(dx).max() <= xtol * (1 + np.abs(Xk).max()):
                return Xk, it, True
        return Xk, max_it, False

    def step_continuation(self, X, n_gamma, gamma0, **kw):
        """One step with continuation in the regularization parameter
        (Sec. 6.3): Newton is solved in turn for
        gamma_i = gamma0 + (i - 1)(gamma - gamma0)/(n_gamma - 1), i = 1..n_gamma,
        each stage starting from the previous stage's solution; the time term
        keeps U(V^{k-1}).  Returns (X, total iterations, all stages converged)."""
        if n_gamma <= 1:
            return self.step(X, **kw)
        gamma = self.prm["gamma"]
        Vh_old, _ = self.unpack(X)
        total, ok_all = 0, True
        Xk = X
        try:
            for i in range(1, n_gamma + 1):
                self.prm["gamma"] = gamma0 + (i - 1) * (gamma - gamma0) / (n_gamma - 1)
                Xk, it, ok = self.step(Xk, Vh_old=Vh_old, **kw)
                total += it
                ok_all = ok_all and ok
        finally:
            self.prm["gamma"] = gamma
        return Xk, total, ok_all

    def run(self, Vh0, n_steps, **kw):
        X = self.pack(Vh0, self.initial_E(Vh0))
        its, fails = [], 0
        for _ in range(n_steps):
            X, it, ok = self.step(X, **kw)
            its.append(it)
            fails += 0 if ok else 1
        return X, its, fails

    def active_percent(self, X):
        """Sec. 6: 100/|Omega| int H(|E| - sigma0/gamma) at the quadrature points."""
        d = self.d
        _, Eh = self.unpack(X)
        Eq = np.einsum("qa,cka->ckq", d.PhiE, Eh)[0]
        thr = self.prm["sigma0"] / self.prm["gamma"]
        act = (np.abs(Eq) - thr >= 0).astype(float)
        return 100.0 * np.sum(d.wJ * act) / np.sum(d.wJ)
