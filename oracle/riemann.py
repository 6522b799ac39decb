"""Exact solutions of the 1D shallow-water dam break: the Riemann problem on
a wet bed (Stoker) and the dam break onto a dry bed (Ritter).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Used for the Newtonian limit (eta = sigma0 = 0) of the dam break, which the
paper compares against the analytic dam-break solution on a wet bed
(Sec. 6.3, Stoker).  The star depth h* solves
    f(h*, h_L) + f(h*, h_R) + u_R - u_L = 0,
with f(h, h_K) = 2 (sqrt(g h) - sqrt(g h_K)) for a rarefaction (h <= h_K)
and (h - h_K) sqrt(g (h + h_K) / (2 h h_K)) for a shock (h > h_K); it is
found by bisection (f is monotone in h).
"""
import math
import numpy as np


def _f(h, hk, g):
    if h <= hk:
        return 2.0 * (math.sqrt(g * h) - math.sqrt(g * hk))
    return (h - hk) * math.sqrt(0.5 * g * (h + hk) / (h * hk))


def star_state(hl, ul, hr, ur, g):
    lo, hi = 1e-14, 10.0 * max(hl, hr) + (ul - ur) ** 2 / g + 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if _f(mid, hl, g) + _f(mid, hr, g) + ur - ul > 0:
            hi = mid
        else:
            lo = mid
    hs = 0.5 * (lo + hi)
    us = 0.5 * (ul + ur) + 0.5 * (_f(hs, hr, g) - _f(hs, hl, g))
    return hs, us


def sample(x, t, x0, hl, ul, hr, ur, g):
    """(h, u) of the exact solution at points x and time t > 0."""
    hs, us = star_state(hl, ul, hr, ur, g)
    cl, cr, cs = math.sqrt(g * hl), math.sqrt(g * hr), math.sqrt(g * hs)
    xi = (np.asarray(x, dtype=float) - x0) / t
    h = np.empty_like(xi)
    u = np.empty_like(xi)
    for k, s in enumerate(xi):
        if s <= us:  # left of contact: left wave
            if hs > hl:  # left shock
                sl = ul - cl * math.sqrt(0.5 * hs * (hs + hl)) / hl
                h[k], u[k] = (hl, ul) if s < sl else (hs, us)
            else:  # left rarefaction
                head, tail = ul - cl, us - cs
                if s <= head:
                    h[k], u[k] = hl, ul
                elif s >= tail:
                    h[k], u[k] = hs, us
                else:
                    c = (ul + 2.0 * cl - s) / 3.0
                    h[k], u[k] = c * c / g, (ul + 2.0 * cl + 2.0 * s) / 3.0
        else:  # right wave
            if hs > hr:  # right shock
                sr = ur + cr * math.sqrt(0.5 * hs * (hs + hr)) / hr
                h[k], u[k] = (hs, us) if s < sr else (hr, ur)
            else:  # right rarefaction
                head, tail = ur + cr, us + cs
                if s >= head:
                    h[k], u[k] = hr, ur
                elif s <= tail:
                    h[k], u[k] = hs, us
                else:
                    c = (-ur + 2.0 * cr + s) / 3.0
                    h[k], u[k] = c * c / g, (ur - 2.0 * cr + 2.0 * s) / 3.0
    return h, u


def ritter(x, t, x0, hl, g):
    """(h, u) of the dam break onto a dry bed (Ritter): still water of depth hl
    left of x0, dry bed right of it, t > 0.  With c = sqrt(g hl) and
    xi = (x - x0) / t the rarefaction fan -c <= xi <= 2c carries
    h = (2c - xi)^2 / (9 g), u = 2 (c + xi) / 3; left of it h = hl, u = 0,
    right of the front xi = 2c the bed is dry (h = u = 0)."""
    c = math.sqrt(g * hl)
    xi = (np.asarray(x, dtype=float) - x0) / t
    fan = (xi >= -c) & (xi <= 2.0 * c)
    h = np.where(xi < -c, hl, np.where(fan, (2.0 * c - xi) ** 2 / (9.0 * g), 0.0))
    u = np.where(fan, 2.0 * (c + xi) / 3.0, 0.0)
    return h, u
