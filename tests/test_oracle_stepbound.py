"""Pins of the oracle's explicit step bound (Discretization.stable_dt) against
the spectrum of the oracle's own linearized space operator.

The paper integrates implicitly (Sec. 5.1) and gives no explicit step bound;
the benchmark workloads step with SSP-RK3.  The bound in use reads
    dt_e = cfl dx_e / ((2p+1) lam_e + (2p+1)^2 2 nu / dx_e),
with nu = (4 eta + max d sigma_B/dE) / rho (the largest slope of the
regularized stress of Sec. 4 is at E = 0).

What fixes it independently of that formula: the linearization of
dV/dt = rhs(V) about a state, J = d rhs / dV, built here column by column by
finite differences of the full nonlinear residual.  SSP-RK3 is stable for a
mode lambda when |R(dt lambda)| <= 1 with R(z) = 1 + z + z^2/2 + z^3/6.

Two properties are checked for every dimension and order:
1. stability: at dt = stable_dt no eigenvalue that sets the explicit limit
   (modulus above 1 % of the spectral radius) is amplified by a step more
   than the linearized ODE itself amplifies it, |R(dt lambda)| <=
   max(1, |exp(dt lambda)|): for the dissipative modes this is the stability
   region, and the few modes whose real part is slightly positive (about
   1e-3 of the spectral radius, from the face terms at the boundaries) are
   held to their exact growth;
2. calibration: in a viscous-dominated state the product rho(J) dt / cfl is
   the measured spectral radius over the bound's viscous term, and in a
   state with no stress it is the same ratio for the wave-speed term.  Both
   must lie in a stated band.  The band is narrow enough that a wrong
   constant fails for some order: a factor 2 in either term, (2p+1) in place
   of (2p+1)^2, the inradius in place of twice the inradius (a factor 4 in
   the viscous term), eta in place of 4 eta, or the slope of another
   regularization.

The boundaries hold the velocity at zero (Dirichlet u = 0 with h and E
copied), which makes the discrete viscous operator dissipative; with copy
(zero-gradient) boundaries the central flux of the stress adds a few
slightly growing boundary modes that say nothing about the step bound.
"""
import numpy as np
import pytest

import synth
from oracle.run import build

# ratio rho(J) * dt / cfl: measured spectral radius over the bound's term
VISCOUS_BAND = (0.7, 2.0)
WAVE_BAND = (1.5, 3.5)


def _fd_jacobian(d, Vh, eps=1e-7):
    x0 = Vh.ravel().copy()
    f0 = d.rhs(Vh)[0].ravel()
    J = np.empty((f0.size, x0.size))
    for i in range(x0.size):
        x = x0.copy()
        x[i] += eps
        J[:, i] = (d.rhs(x.reshape(Vh.shape))[0].ravel() - f0) / eps
    return J


def _case(dim, p, kind):
    """A state at rest (h = 1, u = 0) on a uniform mesh; kind selects the
    stress: 'newtonian' (eta = 1), 'reg1' / 'reg3' / 'reg4' / 'reg5' (Bingham
    sigma0 = 0.1 with parameter 1e3, eta = 0.01) or 'wave' (no stress)."""
    reg = {"newtonian": 0, "reg1": 1, "reg3": 3, "reg4": 4, "reg5": 5, "wave": 0}[kind]
    sigma0 = 0.0 if kind in ("newtonian", "wave") else 0.1
    eta = {"newtonian": 1.0, "wave": 0.0}.get(kind, 0.01)
    if dim == 1:
        c = synth.dam_break_1d(n_el=12, order=p, reg=reg, sigma0=sigma0, eta=eta, pap_m=1e3)
    else:
        c = synth.radial_dam_2d(n=3, order=p, reg=reg, sigma0=sigma0, eta=eta, gamma=1e3, beta=1e3)
    c.params.update(gamma=1e3, beta=1e3, pap_m=1e3)
    c.h_fn = lambda x, xc: np.ones(x.shape[0])
    c.u_fn = lambda x, xc: np.zeros((x.shape[0], dim))
    c.bcs = [([0, 1, 1, 1, 0, 0, 0], [0.0] * 7)] * len(c.bcs)
    return c


def _spectrum(dim, p, kind):
    d, V0, _ = build(_case(dim, p, kind))
    Vh = d.to_modal(V0)
    lam = np.linalg.eigvals(_fd_jacobian(d, Vh))
    return d, Vh, lam


def _rk3_amplification(z):
    return np.abs(1.0 + z + z * z / 2.0 + z ** 3 / 6.0)


def test_rk3_amplification_reference_values():
    # the real-axis limit of 3-stage third-order RK is about 2.5127 and the
    # imaginary-axis limit sqrt(3) (textbook values of the stability polynomial)
    assert _rk3_amplification(np.array([-2.5127])) <= 1.0
    assert _rk3_amplification(np.array([-2.52])) > 1.0
    assert _rk3_amplification(np.array([1j * np.sqrt(3.0)]))[0] == pytest.approx(1.0, abs=1e-12)
    assert _rk3_amplification(np.array([1.8j])) > 1.0


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_step_bound_stable_and_calibrated(dim, p):
    for kind in ("newtonian", "reg1", "reg3", "wave"):
        d, Vh, lam = _spectrum(dim, p, kind)
        rho = np.abs(lam).max()
        dt = d.stable_dt(Vh)
        big = lam[np.abs(lam) >= 0.01 * rho]
        amp = (_rk3_amplification(dt * big) - np.maximum(1.0, np.abs(np.exp(dt * big)))).max()
        assert amp <= 1e-12, f"{kind} dim={dim} p={p}: |R(dt lambda)| - max(1, |exp|) = {amp}"
        ratio = rho * dt / d.prm["cfl"]
        lo, hi = WAVE_BAND if kind == "wave" else VISCOUS_BAND
        assert lo <= ratio <= hi, f"{kind} dim={dim} p={p}: rho dt / cfl = {ratio:.3f} outside [{lo}, {hi}]"


@pytest.mark.parametrize("kind", ["reg4", "reg5"])
def test_step_bound_extension_regularizations(kind):
    # the extensions' slopes at E = 0 (2 sigma0 m and 2 gamma) enter the same way
    for p in (1, 2, 3):
        d, Vh, lam = _spectrum(1, p, kind)
        rho = np.abs(lam).max()
        dt = d.stable_dt(Vh)
        big = lam[np.abs(lam) >= 0.01 * rho]
        assert (_rk3_amplification(dt * big) - np.maximum(1.0, np.abs(np.exp(dt * big)))).max() <= 1e-12
        ratio = rho * dt / d.prm["cfl"]
        assert VISCOUS_BAND[0] <= ratio <= VISCOUS_BAND[1], f"{kind} p={p}: {ratio:.3f}"


def test_step_bound_planted_mistakes_fail():
    """The calibration band rejects the plausible mistakes named above: the
    same spectra checked against a step bound with one constant changed."""
    rows = []
    for dim in (1, 2):
        for p in (1, 2, 3):
            dv, Vv, lv = _spectrum(dim, p, "newtonian")
            dw, Vw, lw = _spectrum(dim, p, "wave")
            rows.append((p, np.abs(lv).max() * dv.stable_dt(Vv) / dv.prm["cfl"],
                         np.abs(lw).max() * dw.stable_dt(Vw) / dw.prm["cfl"]))
    # dt scales by 1/f for a viscous term f times too large (viscous-dominated
    # states) and for a wave term f times too large (wave states)
    viscous_mistakes = {"factor 2 high": 2.0, "factor 2 low": 0.5, "inradius for 2 x inradius": 4.0,
                        "eta for 4 eta": 0.25, "(2p+1) for (2p+1)^2": None}
    for name, f in viscous_mistakes.items():
        caught = False
        for p, rv, _ in rows:
            ff = f if f is not None else 1.0 / (2 * p + 1)
            caught |= not (VISCOUS_BAND[0] <= rv / ff <= VISCOUS_BAND[1])
        assert caught, f"viscous mistake not caught: {name}"
    wave_mistakes = {"factor 2 high": 2.0, "factor 2 low": 0.5, "(p+1) for (2p+1)": None}
    for name, f in wave_mistakes.items():
        caught = False
        for p, _, rw in rows:
            ff = f if f is not None else (p + 1) / (2 * p + 1)
            caught |= not (WAVE_BAND[0] <= rw / ff <= WAVE_BAND[1])
        assert caught, f"wave mistake not caught: {name}"
