"""Exact solution of the Riemann problem for the 1D Euler equations of an
ideal gas (the textbook construction: Newton iteration for the star-region
pressure on the sum of the two wave functions, then sampling of the
self-similar fan).  Used only as an external reference in the tests."""
import math

import numpy as np


def _wave(p, rho, pk, ck, g):
    """Velocity jump across one wave and its derivative with respect to p."""
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    # rarefaction
    r = (p / pk) ** ((g - 1.0) / (2.0 * g))
    return 2.0 * ck / (g - 1.0) * (r - 1.0), 1.0 / (rho * ck) * (p / pk) ** (-(g + 1.0) / (2.0 * g))


def star_state(WL, WR, g=1.4):
    rl, ul, pl = WL
    rr, ur, pr = WR
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    p = max(1e-8, 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr))
    for _ in range(100):
        fl, dl = _wave(p, rl, pl, cl, g)
        fr, dr = _wave(p, rr, pr, cr, g)
        dp = (fl + fr + ur - ul) / (dl + dr)
        pn = max(1e-10, p - dp)
        if abs(pn - p) < 1e-14 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _wave(p, rl, pl, cl, g)
    fr, _ = _wave(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(WL, WR, xi, g=1.4):
    """Primitive (rho, u, p) at similarity coordinate xi = (x - x0)/t."""
    rl, ul, pl = WL
    rr, ur, pr = WR
    ps, us = star_state(WL, WR, g)
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    gm = (g - 1.0) / (g + 1.0)
    if xi <= us:  # left of the contact
        if ps > pl:
            rs = rl * (ps / pl + gm) / (gm * ps / pl + 1.0)
            sl = ul - cl * math.sqrt((g + 1.0) / (2 * g) * ps / pl + (g - 1.0) / (2 * g))
            return (rl, ul, pl) if xi <= sl else (rs, us, ps)
        rs = rl * (ps / pl) ** (1.0 / g)
        cs = cl * (ps / pl) ** ((g - 1.0) / (2 * g))
        if xi <= ul - cl:
            return (rl, ul, pl)
        if xi >= us - cs:
            return (rs, us, ps)
        u = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + xi)
        c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - xi))
        rho = rl * (c / cl) ** (2.0 / (g - 1.0))
        return (rho, u, pl * (c / cl) ** (2.0 * g / (g - 1.0)))
    if ps > pr:
        rs = rr * (ps / pr + gm) / (gm * ps / pr + 1.0)
        sr = ur + cr * math.sqrt((g + 1.0) / (2 * g) * ps / pr + (g - 1.0) / (2 * g))
        return (rr, ur, pr) if xi >= sr else (rs, us, ps)
    rs = rr * (ps / pr) ** (1.0 / g)
    cs = cr * (ps / pr) ** ((g - 1.0) / (2 * g))
    if xi >= ur + cr:
        return (rr, ur, pr)
    if xi <= us + cs:
        return (rs, us, ps)
    u = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + xi)
    c = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - xi))
    rho = rr * (c / cr) ** (2.0 / (g - 1.0))
    return (rho, u, pr * (c / cr) ** (2.0 * g / (g - 1.0)))


def density_profile(WL, WR, x, x0, t, g=1.4):
    return np.array([sample(WL, WR, (xx - x0) / t, g)[0] for xx in x])
