"""Regularized Bingham stress for the oracle (Sec. 4, Appendix A).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The stress splits into a Newtonian and a Bingham part (Eq. binghamR):
sigma = 2 eta (D + tr D I) + sigma_B, with D = (E + E^T)/2 (Eq. DtensorE).
In 1D this is 4 eta E + sigma_B(E) (Eq. sigma11D, bingham1D).

The paper regularizes the 1D Bingham term sigma_B = 2 sigma0 sign(E) with a
scalar function phi(|E|):
  1 smooth max  (Eq. sigmaTwoA/AA), phi = 2 sigma0 gamma s / max_beta(gamma s, sigma0)
                with max_beta(a, b) read as max_beta(a - b, 0) + b (the form the
                appendix differentiates);
  2 local quadratic (Eq. sigmaTwoB);
  3 tanh (Eq. sigmaTwoC), phi = 2 sigma0 tanh(gamma s).
Extensions the paper does not define: 4 exponential (Papanastasiou),
phi = 2 sigma0 (1 - exp(-m s)); 5 bi-viscosity, phi = min(2 gamma s, 2 sigma0).

2D reading (the paper gives the regularizations in 1D only): with
s = ||D||_c / sqrt(2) (||.||_c of Eq. bingham; s = |E| in 1D) the Bingham part
is sigma_B = phi(s) / (2 s) (D + tr D I).  This equals Eq. bingham2 when phi is
the unregularized 2 sigma0, and reduces to the paper's 1D functions in 1D.
sigma0 = 0 gives sigma_B = 0 for every regularization.

Herschel-Bulkley extension (the paper's introduction cites the law; its
scheme is Bingham): with prm["flow_index"] = n in (0, 1) the Newtonian
viscosity eta becomes the power law eta max(s, prm["rate_floor"])^(n - 1)
(eta read as the consistency, s as above); n = 1 (or absent) is the paper's
Newtonian part.
"""
import numpy as np


def max_beta0(x, beta):
    """max_beta(x, 0) of Eq. sigmaTwoAA."""
    e = 1.0 / (2.0 * beta)
    return np.where(x >= e, x, np.where(x <= -e, 0.0, 0.5 * beta * (x + e) ** 2))


def dmax_beta0(x, beta):
    """Derivative of max_beta(x, 0) (Appendix A)."""
    e = 1.0 / (2.0 * beta)
    return np.where(x >= e, 1.0, np.where(x <= -e, 0.0, beta * (x + e)))


def phi(s, prm):
    """phi_k(s) for s >= 0: the regularized 1D Bingham stress at E = s."""
    s = np.asarray(s, dtype=float)
    reg, s0, g, b, m = prm["reg"], prm["sigma0"], prm["gamma"], prm["beta"], prm["pap_m"]
    if reg == 0 or s0 == 0.0:
        return np.zeros_like(s)
    if reg == 1:
        den = max_beta0(g * s - s0, b) + s0
        return 2.0 * s0 * g * s / den
    if reg == 2:
        e = 1.0 / (2.0 * b)
        x = g * s
        mid = 2.0 * s0 - b * (s0 - x + e) ** 2
        return np.where(x >= s0 + e, 2.0 * s0, np.where(x <= s0 - e, 2.0 * x, mid))
    if reg == 3:
        return 2.0 * s0 * np.tanh(g * s)
    if reg == 4:
        return -2.0 * s0 * np.expm1(-m * s)  # 2 sigma0 (1 - exp(-m s)), without cancellation at small s
    if reg == 5:
        return np.minimum(2.0 * g * s, 2.0 * s0)
    raise ValueError(reg)


def dphi(s, prm):
    """d phi_k / ds for s >= 0 (Appendix A; for regularization 2 the lowest
    branch is read as 2 gamma, the derivative of 2 gamma E)."""
    s = np.asarray(s, dtype=float)
    reg, s0, g, b, m = prm["reg"], prm["sigma0"], prm["gamma"], prm["beta"], prm["pap_m"]
    if reg == 0 or s0 == 0.0:
        return np.zeros_like(s)
    if reg == 1:
        x = g * s - s0
        den = max_beta0(x, b) + s0
        return 2.0 * s0 * g / den - 2.0 * s0 * g * g * s * dmax_beta0(x, b) / den ** 2
    if reg == 2:
        e = 1.0 / (2.0 * b)
        x = g * s
        return np.where(x >= s0 + e, 0.0,
                        np.where(x <= s0 - e, 2.0 * g, 2.0 * b * g * (s0 - x + e)))
    if reg == 3:
        x = np.minimum(g * s, 350.0)  # sech^2 underflows to 0 long before cosh overflows
        return 2.0 * s0 * g / np.cosh(x) ** 2
    if reg == 4:
        return 2.0 * s0 * m * np.exp(-m * s)
    if reg == 5:
        return np.where(g * s < s0, 2.0 * g, 0.0)
    raise ValueError(reg)


def phi_over_2s(s, prm):
    """phi_k(s) / (2 s), with its limit phi_k'(0) / 2 at s = 0."""
    s = np.asarray(s, dtype=float)
    with np.errstate(divide="ignore", invalid="ignore"):
        q = phi(s, prm) / (2.0 * s)
    lim = 0.5 * dphi(np.zeros_like(s), prm)
    return np.where(s > 0.0, q, lim)


def flow_index(prm):
    n = float(prm.get("flow_index", 1.0))
    return 1.0 if n == 0.0 else n


def viscosity(s, prm):
    """Viscosity of the Newtonian part at strain-rate measure s: eta, or
    eta max(s, rate_floor)^(n - 1) for the Herschel-Bulkley extension."""
    s = np.asarray(s, dtype=float)
    n = flow_index(prm)
    if n == 1.0:
        return np.full_like(s, prm["eta"])
    return prm["eta"] * np.maximum(s, prm["rate_floor"]) ** (n - 1.0)


def max_viscosity(prm):
    """Largest d sigma_N / dE over E, divided by 4 (1D): eta, or
    eta rate_floor^(n - 1) for 0 < n < 1, where the slope below the floor,
    4 eta rate_floor^(n - 1), exceeds the slope 4 eta n E^(n - 1) above it."""
    n = flow_index(prm)
    return prm["eta"] if n == 1.0 else prm["eta"] * prm["rate_floor"] ** (n - 1.0)


def max_slope(prm):
    """Largest d sigma_B / dE over E (attained at E = 0 for every
    regularization here)."""
    return float(dphi(np.array([0.0]), prm)[0])


def stress(E, dim, prm):
    """Depth-averaged stress sigma (Eq. binghamR) from E.

    E has shape (dim*dim, ...) with component 2*i + j (1D: 0) equal to
    E_ij = d u_j / d x_i (Eq. gradientVel).  Returns sigma as (dim, dim, ...)
    (symmetric)."""
    if dim == 1:
        e = E[0]
        s = np.abs(e)
        mu = 2.0 * viscosity(s, prm) + phi_over_2s(s, prm)
        return (mu * 2.0 * e)[None, None]
    d11 = E[0]
    d22 = E[3]
    d12 = 0.5 * (E[1] + E[2])
    t11 = 2.0 * d11 + d22
    t22 = d11 + 2.0 * d22
    t12 = d12
    nc2 = d11 ** 2 + 2.0 * d12 ** 2 + d22 ** 2 + (d11 + d22) ** 2
    s = np.sqrt(0.5 * nc2)
    mu = 2.0 * viscosity(s, prm) + phi_over_2s(s, prm)
    sig = np.empty((2, 2) + np.shape(d11))
    sig[0, 0] = mu * t11
    sig[1, 1] = mu * t22
    sig[0, 1] = mu * t12
    sig[1, 0] = mu * t12
    return sig


def dsigma_dE_1d(e, prm):
    """d sigma / dE in 1D: 4 eta + phi'(|E|) (Appendix A; Newtonian viscous
    part only)."""
    assert flow_index(prm) == 1.0, "the Appendix A tangent covers the Newtonian viscous part"
    return 4.0 * prm["eta"] + dphi(np.abs(e), prm)
