"""Backward Euler + Newton with the auxiliary variable eliminated, in one or
two dimensions: the paper's time discretization (Sec. 5.1, Eq. WeakForm7 and
Eq. Newton) carried to the two-dimensional scheme, for which the paper gives
no tangent blocks (its Appendix A is one-dimensional).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The E equation of Eq. WeakForm7 is linear in E and u, so E = E(u) is the
E-step of the explicit scheme (Eq. WeakForm52) and the system reduces to the
V unknowns (modal coefficients, Sec. 5):
    R(V) = (1/dt) <N_V, U(V) - U(V_old)> + r_V(V, E(V)),
with U = (h, h u) (Eq. Uterm) and r_V the spatial residual of Eq. WeakForm51.
Newton: J dV = -R, V <- V + dV, with the Jacobian J = dR/dV built column by
column by central differences.  Columns of elements that are more than four
faces apart never touch the same rows (R of an element reads E of its
neighbours, and E reads u of theirs), so such columns are perturbed together
(a distance-4 colouring of the element graph); the assembled sparse matrix
is solved with a library sparse solve.  Stopping rule: ||R||_2 <= rtol
||R^0||_2 or ||R||_2 <= atol, at most max_it iterations (the paper uses 10,
Sec. 6).  The converged state solves R = 0 whatever the accuracy of J.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


class ImplicitReduced:
    def __init__(self, disc, dt, fd_eps=1e-6):
        self.d = disc
        self.dt = float(dt)
        self.fd_eps = float(fd_eps)
        d = disc
        self.shape = (d.nV, d.K, d.Np)
        self.n = d.nV * d.K * d.Np
        self.colors = self._colouring()

    # ------------------------------------------------------------ residual
    def conserved_term(self, Vh):
        """<N_V, U(V)> per element, (nV, K, Np): U = (h, h u_1, ..., h u_d)."""
        d = self.d
        Vq = np.einsum("qa,vka->vkq", d.Phi, Vh)
        U = np.concatenate([Vq[:1], Vq[:1] * Vq[1:]])
        return np.einsum("kq,qa,vkq->vka", d.wJ, d.Phi, U)

    def residual(self, Vh, Uold):
        """R(V) of Eq. WeakForm7 with E = E(u); Uold = conserved_term(V_old)."""
        d = self.d
        Eh = d.e_step(Vh)
        return (self.conserved_term(Vh) - Uold) / self.dt + d.spatial_residual(Vh, Eh)

    # ------------------------------------------------------------ Jacobian
    def _colouring(self):
        d = self.d
        K = d.K
        nbr = [set(int(x) for x in d.nbr[e] if x >= 0) for e in range(K)]
        ball = [{e} for e in range(K)]
        for _ in range(4):  # elements within four faces
            ball = [set().union(*(nbr[x] | {x} for x in b)) for b in ball]
        colour = -np.ones(K, dtype=np.int64)
        for e in range(K):
            used = {int(colour[x]) for x in ball[e] if colour[x] >= 0}
            c = 0
            while c in used:
                c += 1
            colour[e] = c
        return colour

    def jacobian(self, Vh, Uold):
        d = self.d
        nV, K, Np = self.shape
        rows, cols, vals = [], [], []
        idx = np.arange(self.n).reshape(self.shape)
        for c in range(int(self.colors.max()) + 1):
            els = np.nonzero(self.colors == c)[0]
            for v in range(nV):
                for a in range(Np):
                    h = self.fd_eps * np.maximum(1.0, np.abs(Vh[v, els, a]))
                    Vp = Vh.copy()
                    Vm = Vh.copy()
                    Vp[v, els, a] += h
                    Vm[v, els, a] -= h
                    dR = self.residual(Vp, Uold) - self.residual(Vm, Uold)
                    hk = np.zeros(K)
                    hk[els] = h
                    # column of element e lives in the rows of e's distance-2 ball
                    for i, e in enumerate(els):
                        near = [e] + [int(x) for x in d.nbr[e] if x >= 0]
                        near = sorted(set(near + [int(y) for x in near for y in d.nbr[x] if y >= 0]))
                        blk = dR[:, near, :] / (2.0 * h[i])
                        r = idx[:, near, :].ravel()
                        keep = blk.ravel() != 0.0
                        rows.append(r[keep])
                        cols.append(np.full(int(keep.sum()), idx[v, e, a]))
                        vals.append(blk.ravel()[keep])
        return sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.n, self.n))

    # ------------------------------------------------------------ stepping
    def step(self, Vh, max_it=10, rtol=1e-10, atol=1e-12):
        """One backward-Euler step from Vh; returns (V_new, iterations, ||R||_2)."""
        Uold = self.conserved_term(Vh)
        V = Vh.copy()
        R = self.residual(V, Uold)
        r0 = np.linalg.norm(R)
        res = r0
        its = 0
        while its < max_it and res > max(rtol * r0, atol):
            J = self.jacobian(V, Uold)
            dV = spla.spsolve(J, -R.ravel()).reshape(self.shape)
            V = V + dV
            R = self.residual(V, Uold)
            res = np.linalg.norm(R)
            its += 1
        return V, its, res

    def run(self, Vh, n_steps, **kw):
        its = []
        for _ in range(n_steps):
            Vh, k, _ = self.step(Vh, **kw)
            its.append(k)
        return Vh, its
