"""Exact Riemann solver for the ideal gas (textbook two-rarefaction/two-shock
star-state solution), used to pin the oracle's ideal-gas limit (a = b = 0)."""
import numpy as np
from scipy.optimize import brentq


def _wave_fn(p, rk, pk, ck, g):
    if p > pk:
        A = 2.0 / ((g + 1.0) * rk)
        B = (g - 1.0) / (g + 1.0) * pk
        return (p - pk) * np.sqrt(A / (p + B))
    return 2.0 * ck / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)


def solve(rL, uL, pL, rR, uR, pR, g, x, t, x0):
    """Exact (rho, u, p) at positions x and time t for a diaphragm at x0."""
    cL, cR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    f = lambda p: _wave_fn(p, rL, pL, cL, g) + _wave_fn(p, rR, pR, cR, g) + uR - uL
    ps = brentq(f, 1e-14, 100.0 * max(pL, pR), xtol=1e-15)
    us = 0.5 * (uL + uR) + 0.5 * (_wave_fn(ps, rR, pR, cR, g) - _wave_fn(ps, rL, pL, cL, g))
    gm = (g - 1.0) / (g + 1.0)
    out = np.zeros((3, len(x)))
    for k, xx in enumerate(x):
        S = (xx - x0) / t
        if S <= us:
            if ps > pL:
                rs = rL * (ps / pL + gm) / (gm * ps / pL + 1.0)
                SL = uL - cL * np.sqrt((g + 1.0) / (2.0 * g) * ps / pL + (g - 1.0) / (2.0 * g))
                st = (rL, uL, pL) if S < SL else (rs, us, ps)
            else:
                rs = rL * (ps / pL) ** (1.0 / g)
                cs = cL * (ps / pL) ** ((g - 1.0) / (2.0 * g))
                if S < uL - cL:
                    st = (rL, uL, pL)
                elif S > us - cs:
                    st = (rs, us, ps)
                else:
                    u = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * uL + S)
                    c = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * (uL - S))
                    st = (rL * (c / cL) ** (2.0 / (g - 1.0)), u, pL * (c / cL) ** (2.0 * g / (g - 1.0)))
        else:
            if ps > pR:
                rs = rR * (ps / pR + gm) / (gm * ps / pR + 1.0)
                SR = uR + cR * np.sqrt((g + 1.0) / (2.0 * g) * ps / pR + (g - 1.0) / (2.0 * g))
                st = (rR, uR, pR) if S > SR else (rs, us, ps)
            else:
                rs = rR * (ps / pR) ** (1.0 / g)
                cs = cR * (ps / pR) ** ((g - 1.0) / (2.0 * g))
                if S > uR + cR:
                    st = (rR, uR, pR)
                elif S < us + cs:
                    st = (rs, us, ps)
                else:
                    u = 2.0 / (g + 1.0) * (-cR + 0.5 * (g - 1.0) * uR + S)
                    c = 2.0 / (g + 1.0) * (cR - 0.5 * (g - 1.0) * (uR - S))
                    st = (rR * (c / cR) ** (2.0 / (g - 1.0)), u, pR * (c / cR) ** (2.0 * g / (g - 1.0)))
        out[:, k] = st
    return out
