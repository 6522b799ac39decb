"""Manufactured solutions with a forcing term, for the oracle's solution-level
convergence pin.

The exact solution is a compactly supported smooth pulse on a still layer:
    h = 1 + a_h phi(x) (1 + sin(2 t) / 2),
    u_1 = a_1 phi(x) cos(3 t),  u_2 = a_2 phi(x) sin(2 t)  (2D),
with phi = (1 - |x - c|^2 / R^2)^8 inside the disc |x - c| < R and 0 outside
(seven continuous derivatives), so that the state is exactly (1, 0) on and
near the boundary and the copy boundary condition is exact there.  The
forcing is the residual of the exact solution in the conservative system of
Eq. shallowR2/3 (U = (h, h u), E = grad u):
    f = dU/dt + sum_i dF_i/dx_i - sum_i dQ_i/dx_i - S,
written here symbolically (sympy) from the PDE, independently of the
oracle's weak form; the discrete scheme with this forcing added to its
source must converge to the exact solution.
"""
import numpy as np
import sympy as sp

PULSE_POWER = 8


def _residual_exprs(dim, prm, X, t, phi):
    """Symbolic (h, u) and the forcing f of the conservative system for a
    pulse profile phi (an expression in X, or 0 for the still layer)."""
    g, rho, alpha = prm["g"], prm["rho"], prm["alpha"]
    eta, s0, gam = prm["eta"], prm["sigma0"], prm["gamma"]
    gc = g * sp.cos(alpha)
    gs = g * sp.sin(alpha)
    amps = (0.1, 0.2, 0.1)
    h = 1 + amps[0] * phi * (1 + sp.sin(2 * t) / 2)
    u = [amps[1] * phi * sp.cos(3 * t)]
    if dim == 2:
        u.append(amps[2] * phi * sp.sin(2 * t))
    E = [[sp.diff(u[j], X[i]) for j in range(dim)] for i in range(dim)]
    bingham = prm["reg"] == 3 and s0 > 0 and not (isinstance(phi, sp.Integer) and phi == 0)
    if dim == 1:
        e = E[0][0]
        sig = [[4 * eta * e + (2 * s0 * sp.tanh(gam * e) if bingham else 0)]]
    else:
        d11, d22 = E[0][0], E[1][1]
        d12 = (E[0][1] + E[1][0]) / 2
        t11, t22, t12 = 2 * d11 + d22, d11 + 2 * d22, d12
        mu = 2 * eta
        if bingham:
            s = sp.sqrt((d11 ** 2 + 2 * d12 ** 2 + d22 ** 2 + (d11 + d22) ** 2) / 2)
            mu = mu + s0 * sp.tanh(gam * s) / s
        sig = [[mu * t11, mu * t12], [mu * t12, mu * t22]]
    f = [sp.diff(h, t) + sum(sp.diff(h * u[i], X[i]) for i in range(dim))]
    for j in range(dim):
        m = sp.diff(h * u[j], t)
        for i in range(dim):
            F = h * u[i] * u[j] + (gc * h * h / 2 if i == j else 0)
            Q = h * sig[j][i] / rho
            m += sp.diff(F, X[i]) - sp.diff(Q, X[i])
        if j == 0:
            m += gs * h  # - S with S_1 = -g_s h (flat bed)
        f.append(m)
    return [h] + u, f


def forced_problem(dim, prm, radius=1.0, center=(0.1, -0.07)):
    """(exact, forcing): functions of (t, x) with x of shape (..., dim)
    returning arrays of shape (dim + 1, ...).

    The pulse enters the symbolic work as an undefined function phi(x) whose
    value and first and second derivatives are substituted numerically (from
    the closed form of phi), which keeps the expressions small."""
    t = sp.symbols("t")
    X = list(sp.symbols("x y")[:dim])
    phi = sp.Function("phi")(*X)
    V_in, f_in = _residual_exprs(dim, prm, X, t, phi)
    V_out, f_out = _residual_exprs(dim, prm, X, t, sp.Integer(0))
    # plain symbols for phi and its derivatives (second derivatives replaced first)
    pairs = [(sp.Derivative(phi, X[i], X[j]), sp.Symbol(f"p{i}{j}")) for i in range(dim) for j in range(i, dim)]
    pairs += [(sp.Derivative(phi, X[i]), sp.Symbol(f"p{i}")) for i in range(dim)]
    pairs += [(phi, sp.Symbol("p"))]
    psyms = [b for _, b in pairs]

    def to_syms(ex):
        ex = sp.sympify(ex).doit()
        for a, b in pairs:
            ex = ex.subs(a, b)
        return ex

    lam = lambda ex: sp.lambdify([t] + psyms, to_syms(ex), "numpy", cse=True)  # noqa: E731
    lam_out = lambda ex: sp.lambdify([t] + X, ex, "numpy")  # noqa: E731
    parts = [([lam(c) for c in V_in], [lam_out(c) for c in V_out]),
             ([lam(c) for c in f_in], [lam_out(c) for c in f_out])]
    # closed form of the pulse and its derivatives, in the same order as psyms
    r2 = sum((X[i] - center[i]) ** 2 for i in range(dim)) / radius ** 2
    prof = (1 - r2) ** PULSE_POWER
    pexpr = [sp.diff(prof, X[i], X[j]) for i in range(dim) for j in range(i, dim)]
    pexpr += [sp.diff(prof, X[i]) for i in range(dim)] + [prof]
    pfun = [sp.lambdify(X, e, "numpy") for e in pexpr]
    cen = np.asarray(center[:dim])

    def evaluate(which, tt, x):
        fin, fout = parts[which]
        m = (((x - cen) ** 2).sum(axis=-1) / radius ** 2) < 1.0
        cols = [x[..., i] for i in range(dim)]
        pv = [np.broadcast_to(f(*cols), m.shape) for f in pfun]
        out = np.empty((dim + 1,) + x.shape[:-1])
        with np.errstate(all="ignore"):
            for v in range(dim + 1):
                a = np.broadcast_to(fin[v](tt, *pv), m.shape)
                b = np.broadcast_to(fout[v](tt, *cols), m.shape)
                out[v] = np.where(m, a, b)
        return out

    return (lambda tt, x: evaluate(0, tt, x)), (lambda tt, x: evaluate(1, tt, x))
