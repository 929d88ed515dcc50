"""Exact solution of the Riemann problem of the 1D Euler equations for an ideal gas.

Test helper only.  Pressure in the star region from Newton iteration on
f(p) = f_L(p) + f_R(p) + (u_R - u_L) = 0 with the shock / rarefaction branch functions of the
textbook solution (e.g. Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics", ch. 4),
then sampling of the self-similar solution at x/t.
"""
import math

import numpy as np


def _branch(p, rho, pk, gamma):
    a = math.sqrt(gamma * pk / rho)
    if p > pk:  # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        q = math.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (p + B))
    pr = p / pk  # rarefaction
    f = 2.0 * a / (gamma - 1.0) * (pr ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)
    df = 1.0 / (rho * a) * pr ** (-(gamma + 1.0) / (2.0 * gamma))
    return f, df


def star_state(left, right, gamma):
    """(p*, u*) for left/right = (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    p = max(1e-8, 0.5 * (pl + pr))
    for _ in range(100):
        fl, dfl = _branch(p, rl, pl, gamma)
        fr, dfr = _branch(p, rr, pr, gamma)
        f = fl + fr + (ur - ul)
        pn = max(1e-12, p - f / (dfl + dfr))
        if abs(pn - p) < 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _branch(p, rl, pl, gamma)
    fr, _ = _branch(p, rr, pr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, gamma, xi):
    """Primitive (rho, u, p) of the exact solution at similarity coordinates xi = (x - x0)/t."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, gamma)
    g = gamma
    out = np.zeros((3, len(xi)))
    al, ar = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    for n, s in enumerate(xi):
        if s <= us:  # left of contact
            if ps > pl:
                rs = rl * ((ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1))
                sh = ul - al * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                st = (rl, ul, pl) if s < sh else (rs, us, ps)
            else:
                rs = rl * (ps / pl) ** (1 / g)
                ash = al * (ps / pl) ** ((g - 1) / (2 * g))
                hd, tl = ul - al, us - ash
                if s < hd:
                    st = (rl, ul, pl)
                elif s > tl:
                    st = (rs, us, ps)
                else:
                    u = 2 / (g + 1) * (al + (g - 1) / 2 * ul + s)
                    c = 2 / (g + 1) * (al + (g - 1) / 2 * (ul - s))
                    r = rl * (c / al) ** (2 / (g - 1))
                    st = (r, u, pl * (c / al) ** (2 * g / (g - 1)))
        else:
            if ps > pr:
                rs = rr * ((ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1))
                sh = ur + ar * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                st = (rr, ur, pr) if s > sh else (rs, us, ps)
            else:
                rs = rr * (ps / pr) ** (1 / g)
                ash = ar * (ps / pr) ** ((g - 1) / (2 * g))
                hd, tl = ur + ar, us + ash
                if s > hd:
                    st = (rr, ur, pr)
                elif s < tl:
                    st = (rs, us, ps)
                else:
                    u = 2 / (g + 1) * (-ar + (g - 1) / 2 * ur + s)
                    c = 2 / (g + 1) * (ar - (g - 1) / 2 * (ur - s))
                    r = rr * (c / ar) ** (2 / (g - 1))
                    st = (r, u, pr * (c / ar) ** (2 * g / (g - 1)))
        out[:, n] = st
    return out
