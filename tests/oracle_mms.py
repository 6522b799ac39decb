"""Closed-form time derivatives of smooth states for the oracle's consistency pin.

For a smooth state (h, u) with bed H the exact right-hand side of
Eq. shallowR2/3 (with E = grad u) is
    dh/dt = -div(h u),
    d(h u_j)/dt = -sum_i d F_i[1+j]/dx_i + sum_i d Q_i[1+j]/dx_i + S[1+j],
    du_j/dt = (d(h u_j)/dt - u_j dh/dt) / h,
written here symbolically (sympy) from the PDE, independently of the oracle's
weak form.  The tanh regularization (Eq. sigmaTwoC) keeps the stress smooth.
"""
import sympy as sp


def exact_rhs(dim, prm, with_bed=True):
    g, rho, alpha = prm["g"], prm["rho"], prm["alpha"]
    eta, s0, gam = prm["eta"], prm["sigma0"], prm["gamma"]
    gc = g * sp.cos(alpha)
    gs = g * sp.sin(alpha)
    if dim == 1:
        x = sp.symbols("x")
        X = [x]
        h = 1 + sp.Rational(1, 5) * sp.sin(sp.pi * x) + sp.Rational(1, 10) * x
        u = [sp.Rational(3, 10) * sp.cos(sp.pi * x) + sp.Rational(1, 5) * x]
        H = sp.Rational(1, 10) * sp.cos(2 * x) if with_bed else sp.Integer(0)
    else:
        x, y = sp.symbols("x y")
        X = [x, y]
        h = 1 + sp.Rational(1, 5) * sp.sin(sp.pi * x / 2) * sp.cos(sp.pi * y / 3)
        u = [sp.Rational(3, 10) * sp.cos(x + y / 2) + sp.Rational(1, 4) * x,
             sp.Rational(1, 5) * sp.sin(x - y) - sp.Rational(1, 5) * y]
        H = (sp.Rational(1, 10) * sp.cos(x) * sp.sin(y / 2)) if with_bed else sp.Integer(0)
    E = [[sp.diff(u[j], X[i]) for j in range(dim)] for i in range(dim)]
    if dim == 1:
        e = E[0][0]
        s = sp.sqrt(e ** 2)
        sig = [[4 * eta * e + 2 * s0 * sp.tanh(gam * e)]]
    else:
        d11, d22 = E[0][0], E[1][1]
        d12 = (E[0][1] + E[1][0]) / 2
        t11, t22, t12 = 2 * d11 + d22, d11 + 2 * d22, d12
        nc2 = d11 ** 2 + 2 * d12 ** 2 + d22 ** 2 + (d11 + d22) ** 2
        s = sp.sqrt(nc2 / 2)
        mu = 2 * eta + s0 * sp.tanh(gam * s) / s
        sig = [[mu * t11, mu * t12], [mu * t12, mu * t22]]
    ht = -sum(sp.diff(h * u[i], X[i]) for i in range(dim))
    uts = []
    for j in range(dim):
        mom = 0
        for i in range(dim):
            F = h * u[i] * u[j] + (gc * h * h / 2 if i == j else 0)
            Q = h * sig[j][i] / rho
            mom += -sp.diff(F, X[i]) + sp.diff(Q, X[i])
        src = -gc * h * sp.diff(H, X[j])
        if j == 0:
            src += -gs * h
        mom += src
        uts.append((mom - u[j] * ht) / h)
    f = lambda ex: sp.lambdify(X, ex, "numpy")  # noqa: E731
    return dict(h=f(h), u=[f(c) for c in u], H=f(H), ht=f(ht), ut=[f(c) for c in uts])
