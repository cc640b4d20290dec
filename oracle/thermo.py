"""Closed-form thermodynamics of the van der Waals fluid (test infrastructure only).

Used to build initial conditions of the synthetic workloads and as pins:
  - vdW pressure, internal energy e = C_v T - a rho (Eq. SM vdW internal energy)
  - isentropic sound speed (Eq. SM speed of sound formula, vdW form)
  - Maxwell's equal-area rule for coexistence densities (main text, Fig. 2)
  - Rankine-Hugoniot post-shock state in closed form (SM "Rankine-Hugoniot
    conditions"), with the velocity formula read with the pre-shock sound speed
    (the printed formula names the post-shock one; only the pre-shock reading
    satisfies the jump conditions)
  - Rankine-Hugoniot state by a direct root solve of the jump conditions (pin)
"""
from __future__ import annotations

import math

import numpy as np
from scipy import optimize

A_VDW = 2.0 / 49.0
B_VDW = 2.0 / 21.0
R_GAS = 1.0


def critical(a=A_VDW, b=B_VDW, R=R_GAS):
    """rho_cr = 1/(3b), T_cr = 8a/(27 R b), p_cr = a/(27 b^2) (main text)."""
    return 1.0 / (3.0 * b), 8.0 * a / (27.0 * R * b), a / (27.0 * b * b)


def pressure(rho, T, a=A_VDW, b=B_VDW, R=R_GAS):
    return rho * R * T / (1.0 - b * rho) - a * rho * rho


def energy(rho, T, delta, a=A_VDW, R=R_GAS):
    return (R / delta) * T - a * rho


def dp_drho_T(rho, T, a=A_VDW, b=B_VDW, R=R_GAS):
    return R * T / (1.0 - b * rho) ** 2 - 2.0 * a * rho


def sound_speed(rho, T, delta, a=A_VDW, b=B_VDW, R=R_GAS):
    """Isentropic vdW sound speed sqrt(R T (1 + delta)/(1 - b rho)^2 - 2 a rho)."""
    return math.sqrt(R * T * (1.0 + delta) / (1.0 - b * rho) ** 2 - 2.0 * a * rho)


def _helmholtz_mu(rho, T, a=A_VDW, b=B_VDW, R=R_GAS):
    """Chemical potential up to a T-only constant: mu = f + p/rho with
    f = -R T ln((1 - b rho)/rho) - a rho (isothermal part of the vdW free energy)."""
    return -R * T * math.log((1.0 - b * rho) / rho) - a * rho + pressure(rho, T, a, b, R) / rho


def maxwell(Tr: float, a=A_VDW, b=B_VDW, R=R_GAS):
    """Coexisting (rho_v, rho_l) at T = Tr*T_cr by equal pressure and equal chemical
    potential, which is Maxwell's equal-area rule."""
    rc, Tc, pc = critical(a, b, R)
    T = Tr * Tc
    # spinodal densities bracket the roots
    sp = np.sort(np.roots([-2.0 * a * b * b, 4.0 * a * b, -2.0 * a, R * T]).real)
    sp = [s for s in sp if 0 < s < 1.0 / b]
    lo, hi = sp[0], sp[-1]

    def resid(x):
        rv, rl = x
        return [pressure(rv, T, a, b, R) - pressure(rl, T, a, b, R),
                _helmholtz_mu(rv, T, a, b, R) - _helmholtz_mu(rl, T, a, b, R)]

    guess = [rc * max(1e-3, 1.0 - 2.0 * math.sqrt(1.0 - Tr)) * 0.8, rc * (1.0 + 2.0 * math.sqrt(1.0 - Tr))]
    guess = [min(guess[0], 0.9 * lo), max(guess[1], 1.1 * hi)]
    sol = optimize.fsolve(resid, guess, xtol=1e-14, full_output=True)
    rv, rl = sol[0]
    if not (0 < rv < lo and hi < rl < 1.0 / b):
        raise RuntimeError("Maxwell construction failed at Tr=%g" % Tr)
    return float(rv), float(rl)


def rh_closed_form(rho0: float, p0: float, rho1: float, delta: float,
                   a=A_VDW, b=B_VDW, R=R_GAS):
    """Post-shock (Mach M0 w.r.t. the pre-shock sound speed, u1, p1) for a shock moving
    into still fluid, from the reduced closed form (SM "Rankine-Hugoniot conditions")."""
    rc, Tc, pc = critical(a, b, R)
    vc = 1.0 / rc
    scale = math.sqrt(pc * vc)
    r0, r1, pt0 = rho0 / rc, rho1 / rc, p0 / pc
    T0 = (p0 + a * rho0 * rho0) * (1.0 - b * rho0) / (rho0 * R)
    c0 = sound_speed(rho0, T0, delta, a, b, R) / scale
    num = pt0 * (1.0 + delta) + r0 * r1 * (r0 + r1 + 3.0 * delta - 3.0)
    den = r0 * (2.0 * r0 * (3.0 - r1) + 3.0 * delta * (r0 - r1))
    M0 = math.sqrt(6.0 * r1 * num / den) / c0
    u1 = c0 * M0 * (r1 - r0) / r1
    p1 = pt0 + c0 * c0 * M0 * M0 * r0 * (r1 - r0) / r1
    return M0, u1 * scale, p1 * pc


def rh_root_solve(rho0: float, p0: float, rho1: float, delta: float,
                  a=A_VDW, b=B_VDW, R=R_GAS):
    """Same state from the jump conditions -s<M> + <N> = 0 solved numerically
    for (s, u1, p1) with u0 = 0."""
    def e_of(rho, p):
        T = (p + a * rho * rho) * (1.0 - b * rho) / (rho * R)
        return energy(rho, T, delta, a, R)

    def resid(x):
        s, u1, p1 = x
        E0 = e_of(rho0, p0)
        E1 = e_of(rho1, p1) + 0.5 * u1 * u1
        return [-s * (rho1 - rho0) + rho1 * u1,
                -s * rho1 * u1 + (p1 + rho1 * u1 * u1 - p0),
                -s * (rho1 * E1 - rho0 * E0) + u1 * (rho1 * E1 + p1)]

    T0 = (p0 + a * rho0 * rho0) * (1.0 - b * rho0) / (rho0 * R)
    c0 = sound_speed(rho0, T0, delta, a, b, R)
    M_guess, u_guess, p_guess = rh_closed_form(rho0, p0, rho1, delta, a, b, R)
    x = optimize.fsolve(resid, [M_guess * c0 * 1.01, u_guess * 0.99, p_guess * 1.01], xtol=1e-14)
    s, u1, p1 = x
    return s / c0, u1, p1


def post_shock_for_mach(rho0: float, T0: float, Mach: float, delta: float,
                        a=A_VDW, b=B_VDW, R=R_GAS):
    """Post-shock (rho1, u1, p1, T1) for a shock of the given Mach number (w.r.t. the
    pre-shock sound speed) into still fluid at (rho0, T0)."""
    p0 = pressure(rho0, T0, a, b, R)
    f = lambda r1: rh_closed_form(rho0, p0, r1, delta, a, b, R)[0] - Mach
    rc = critical(a, b, R)[0]
    r0 = rho0 / rc
    # the closed form's denominator vanishes at the strong-shock compression limit
    hi = rc * r0 * (6.0 + 3.0 * delta) / (2.0 * r0 + 3.0 * delta) * (1.0 - 1e-9)
    lo = rho0 * (1.0 + 1e-9)
    r1 = optimize.brentq(f, lo, hi, xtol=1e-15, rtol=1e-15)
    M0, u1, p1 = rh_closed_form(rho0, p0, r1, delta, a, b, R)
    T1 = (p1 + a * r1 * r1) * (1.0 - b * r1) / (r1 * R)
    return float(r1), float(u1), float(p1), float(T1)


# ---------------------------------------------------------------------------------------
# Dieterici fluid (SM "Coexistence curve", used isothermally there):
#   p = rho R T / (1 - b rho) exp(-a rho / (R T)),
# critical point rho_cr = 1/(2b), T_cr = a/(4 R b), p_cr = a / (2 e b)^2.  The workloads
# take b = 1/7, a = 32/441, which put the critical point at rho_cr = 3.5, T_cr = 8/63 as
# for the van der Waals constants above.
A_DIE = 32.0 / 441.0
B_DIE = 1.0 / 7.0


def dieterici_critical(a=A_DIE, b=B_DIE, R=R_GAS):
    return 1.0 / (2.0 * b), a / (4.0 * R * b), a / (2.0 * math.e * b) ** 2


def dieterici_pressure(rho, T, a=A_DIE, b=B_DIE, R=R_GAS):
    return rho * R * T / (1.0 - b * rho) * np.exp(-a * rho / (R * T))


def dieterici_dp_drho_T(rho, T, a=A_DIE, b=B_DIE, R=R_GAS):
    """(dp/drho)_T = p (1/rho + b/(1 - b rho) - a/(R T))."""
    return dieterici_pressure(rho, T, a, b, R) * (1.0 / rho + b / (1.0 - b * rho) - a / (R * T))


def dieterici_spinodals(T, a=A_DIE, b=B_DIE, R=R_GAS):
    """Densities where (dp/drho)_T = 0: roots of rho^2 - rho/b + R T/(a b) = 0."""
    disc = 1.0 / (b * b) - 4.0 * R * T / (a * b)
    if disc <= 0.0:
        raise ValueError("no spinodal above the critical temperature")
    r = math.sqrt(disc)
    return 0.5 * (1.0 / b - r), 0.5 * (1.0 / b + r)


def dieterici_maxwell(Tr: float, a=A_DIE, b=B_DIE, R=R_GAS):
    """Coexisting (rho_v, rho_l) at T = Tr T_cr: equal pressure p_s and equal areas,
    integral_{rho_v}^{rho_l} p / rho^2 drho = p_s (1/rho_v - 1/rho_l) (Maxwell's rule in
    the p-v plane), the saturation pressure found between the spinodal pressures."""
    from scipy import integrate
    rc, Tc, pc = dieterici_critical(a, b, R)
    T = Tr * Tc
    lo, hi = dieterici_spinodals(T, a, b, R)
    p_max = dieterici_pressure(lo, T, a, b, R)   # local maximum (vapour spinodal)
    p_min = dieterici_pressure(hi, T, a, b, R)   # local minimum (liquid spinodal)

    def roots(ps):
        rv = optimize.brentq(lambda r: dieterici_pressure(r, T, a, b, R) - ps, 1e-12 * lo, lo,
                             xtol=1e-15, rtol=1e-15)
        rl = optimize.brentq(lambda r: dieterici_pressure(r, T, a, b, R) - ps, hi,
                             (1.0 - 1e-12) / b, xtol=1e-15, rtol=1e-15)
        return rv, rl

    def area(ps):
        rv, rl = roots(ps)
        val, _ = integrate.quad(lambda r: dieterici_pressure(r, T, a, b, R) / (r * r), rv, rl,
                                epsabs=0.0, epsrel=1e-13, limit=200)
        return val - ps * (1.0 / rv - 1.0 / rl)

    span = p_max - p_min
    ps = optimize.brentq(area, p_min + 1e-9 * span, p_max - 1e-9 * span, xtol=1e-16, rtol=1e-15)
    rv, rl = roots(ps)
    return float(rv), float(rl)


# ---------------------------------------------------------------------------------------
# Non-classical gas dynamics (main text, Fig. 4; SM "Shock tube").
def temperature(rho, p, a=A_VDW, b=B_VDW, R=R_GAS):
    """T of the van der Waals fluid at (rho, p): (p + a rho^2)(1 - b rho)/(rho R)."""
    return (p + a * rho * rho) * (1.0 - b * rho) / (rho * R)


def fundamental_derivative(p, rho, delta, a=A_VDW, b=B_VDW):
    """Gamma = (v^3 / (2 c^2)) (d^2 p / d v^2)_s of the vdW fluid with C_v = R/delta, in
    the closed form of the SM (v = 1/rho; any consistent units)."""
    v = 1.0 / rho
    q = p + a / v ** 2
    num = (delta + 1.0) * (delta + 2.0) * q / (v - b) ** 2 - 6.0 * a / v ** 4
    den = 2.0 * (delta + 1.0) * q / (v * (v - b)) - 4.0 * a / v ** 4
    return num / den


# ---------------------------------------------------------------------------------------
# Simplified near-critical EoS (SM "Speed of sound"): free energy per volume
# E0 = beta (rho - rho_l)^2 (rho - rho_v)^2, p = p0 + rho dE0/drho - E0.  The printed form
# has no background pressure and gives p = 0 at both saturated densities, which leaves no
# gauge temperature theta = p/(rho T_L); a constant p0 changes neither the coexistence
# (equal pressure p0 and equal chemical potential at rho_v, rho_l) nor dp/drho.
SIMP = {"beta": 1e-3, "rho_l": 5.0, "rho_v": 0.5, "p0": 0.1}   # rho_l / rho_v = 10 as in the SM


def simplified_pressure(rho, beta=SIMP["beta"], rho_l=SIMP["rho_l"], rho_v=SIMP["rho_v"], p0=SIMP["p0"]):
    dl, dv = rho - rho_l, rho - rho_v
    return p0 + rho * 2.0 * beta * dl * dv * (dl + dv) - beta * dl * dl * dv * dv


def simplified_sound_speed(rho, beta=SIMP["beta"], rho_l=SIMP["rho_l"], rho_v=SIMP["rho_v"]):
    """sqrt(dp/drho) = sqrt(rho E0''); at rho_l, rho_v it is sqrt(2 beta rho) (rho_l - rho_v)."""
    dl, dv = rho - rho_l, rho - rho_v
    return math.sqrt(rho * 2.0 * beta * (dl * dl + 4.0 * dl * dv + dv * dv))
