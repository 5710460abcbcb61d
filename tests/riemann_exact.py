"""Exact solution of the Riemann problem of the 1D ideal-gas Euler equations (the textbook
construction: star pressure from the two-wave pressure function by Newton iteration, then
sampling of the self-similar solution at x/t).  Test infrastructure for the Sod checks."""
import numpy as np


def _wave(p, rho, pk, ck, g):
    """Pressure function f_k(p) and its derivative for one side (shock if p > pk)."""
    if p > pk:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = np.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    r = p / pk
    f = 2.0 * ck / (g - 1.0) * (r ** ((g - 1.0) / (2.0 * g)) - 1.0)
    return f, 1.0 / (rho * ck) * r ** (-(g + 1.0) / (2.0 * g))


def star_state(L, R, g=1.4):
    rl, ul, pl = L
    rr, ur, pr = R
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    p = max(1e-10, 0.5 * (pl + pr))
    for _ in range(100):
        fl, dl = _wave(p, rl, pl, cl, g)
        fr, dr = _wave(p, rr, pr, cr, g)
        step = (fl + fr + ur - ul) / (dl + dr)
        p = max(1e-12, p - step)
        if abs(step) < 1e-14 * p:
            break
    fl, _ = _wave(p, rl, pl, cl, g)
    fr, _ = _wave(p, rr, pr, cr, g)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(L, R, xi, g=1.4):
    """Primitive (rho, u, p) at similarity coordinates xi = (x - x_c)/t."""
    rl, ul, pl = L
    rr, ur, pr = R
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    ps, us = star_state(L, R, g)
    out = np.zeros((len(xi), 3))
    for i, s in enumerate(xi):
        if s <= us:                                  # left of the contact
            if ps > pl:                              # left shock
                rs = rl * (ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1)
                sh = ul - cl * np.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                out[i] = (rl, ul, pl) if s < sh else (rs, us, ps)
            else:                                    # left rarefaction
                rs = rl * (ps / pl) ** (1 / g)
                cs = cl * (ps / pl) ** ((g - 1) / (2 * g))
                if s < ul - cl:
                    out[i] = (rl, ul, pl)
                elif s > us - cs:
                    out[i] = (rs, us, ps)
                else:
                    u = 2 / (g + 1) * (cl + (g - 1) / 2 * ul + s)
                    c = 2 / (g + 1) * (cl + (g - 1) / 2 * (ul - s))
                    rho = rl * (c / cl) ** (2 / (g - 1))
                    out[i] = (rho, u, pl * (c / cl) ** (2 * g / (g - 1)))
        else:                                        # right of the contact
            if ps > pr:                              # right shock
                rs = rr * (ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1)
                sh = ur + cr * np.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                out[i] = (rs, us, ps) if s < sh else (rr, ur, pr)
            else:                                    # right rarefaction
                rs = rr * (ps / pr) ** (1 / g)
                cs = cr * (ps / pr) ** ((g - 1) / (2 * g))
                if s > ur + cr:
                    out[i] = (rr, ur, pr)
                elif s < us + cs:
                    out[i] = (rs, us, ps)
                else:
                    u = 2 / (g + 1) * (-cr + (g - 1) / 2 * ur + s)
                    c = 2 / (g + 1) * (cr - (g - 1) / 2 * (ur - s))
                    rho = rr * (c / cr) ** (2 / (g - 1))
                    out[i] = (rho, u, pr * (c / cr) ** (2 * g / (g - 1)))
    return out
