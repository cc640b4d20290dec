"""Writes ``paper_2002_09217_gb300/workloads.json``: the thermodynamic constants
that the synthetic workloads are built from (coexistence densities by Maxwell's
rule, Rankine-Hugoniot post-shock states, the per-temperature time step, the time step of
uniform saturated states and of the critical state for the sound-pulse experiments, the
time steps of the coexistence-curve cases of Fig. 2, and the isothermal Dieterici
coexistence of the SM, the non-classical shock-tube states, the simplified near-critical
EoS).

Run: ``python -m oracle.write_workloads``.  It calls only ``oracle.thermo``; the
JSON file is data that the input generators read, so no product code executes
the oracle.

Time step rule (the paper keeps delta t symbolic with Delta x = 1): the explicit
step is stable in the dense phase only while the shortest waves (checkerboard
modes along x and along the diagonal) are carried by the stencil, which a 1-D
shortest-wave analysis of stream + relax puts at delta t <~ 1.25 sqrt(theta)/varsigma^2
and 2-D oracle runs at about 0.6 of that.  We take 0.45 sqrt(theta)/varsigma^2 at the
densest state of the workload, capped at 0.5.

A droplet hit by a shock is run at 3/4 of that step (``dt_droplet`` of the shock
rows): the interaction cools parts of the droplet well below the initial temperature
(to 0.69 T_cr from 0.8 T_cr in the 2048 x 1024 case), where the same bound is much
tighter (0.096 at 0.75 T_cr against 0.146 at 0.8 T_cr for the compressed liquid); at the
full step both forms of that case went non-finite before step 10,000, at 3/4 of it the
run stays finite.
"""
from __future__ import annotations

import json
import math
import os

from . import thermo

DELTA = 1.0 / 3.0
T_L = 1.0 / 3.0
OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2002_09217_gb300", "workloads.json")


def dt_rule(rho: float, T: float, delta: float = DELTA) -> float:
    p = thermo.pressure(rho, T)
    theta = p / (rho * T_L)
    c2 = thermo.sound_speed(rho, T, delta) ** 2
    return float(min(0.5, 0.45 * math.sqrt(theta) / c2))


def dt_rule_isothermal_dieterici(rho: float, T: float) -> float:
    """The same rule with the Dieterici pressure and its isothermal sound speed (the
    isothermal model carries sound at sqrt((dp/drho)_T))."""
    p = thermo.dieterici_pressure(rho, T)
    theta = p / (rho * T_L)
    return float(min(0.5, 0.45 * math.sqrt(theta) / thermo.dieterici_dp_drho_T(rho, T)))


def main() -> None:
    rc, Tc, pc = thermo.critical()
    coex = {}
    for k in range(70, 96):
        Tr = k / 100.0
        rv, rl = thermo.maxwell(Tr)
        coex["%.2f" % Tr] = {"rho_v": rv, "rho_l": rl, "dt": dt_rule(rl, Tr * Tc)}
    shocks = {}
    for k in range(70, 96):
        Tr = k / 100.0
        rv = coex["%.2f" % Tr]["rho_v"]
        row = {}
        for m in range(12, 31):
            Ma = m / 10.0
            r1, u1, p1, T1 = thermo.post_shock_for_mach(rv, Tr * Tc, Ma, DELTA)
            dt = min(coex["%.2f" % Tr]["dt"], dt_rule(r1, T1), 0.5 / (1.0 + abs(u1)))
            row["%.1f" % Ma] = {"rho1": r1, "u1": u1, "T1": T1, "dt": dt, "dt_droplet": 0.75 * dt}
        shocks["%.2f" % Tr] = row
    sup_rho = 2.0 * rc
    # isothermal Dieterici coexistence (SM "Coexistence curve"): constants, critical point,
    # Maxwell densities and time step per reduced temperature
    drc, dTc, dpc = thermo.dieterici_critical()
    dcoex = {}
    for k in range(70, 96):
        Tr = k / 100.0
        rv, rl = thermo.dieterici_maxwell(Tr)
        dcoex["%.2f" % Tr] = {"rho_v": rv, "rho_l": rl,
                              "dt": dt_rule_isothermal_dieterici(rl, Tr * dTc)}
    dieterici = {"a": thermo.A_DIE, "b": thermo.B_DIE, "critical": {"rho": drc, "T": dTc, "p": dpc},
                 "coexistence": dcoex}
    # shock tubes of non-classical gas dynamics: the anomalous case of the main text's
    # Fig. 4 and the SM's cases I, II, states given in reduced units (p/p_cr, rho/rho_cr);
    # snapshot times t* = (t / L) sqrt(p_cr / rho_cr)
    # the simplified near-critical EoS of the SM's speed-of-sound study (isothermal): its
    # constants and the time step by the usual rule at each saturated density
    sp = dict(thermo.SIMP)
    dts = []
    for rho in (sp["rho_l"], sp["rho_v"]):
        theta = thermo.simplified_pressure(rho) / (rho * T_L)
        dts.append(min(0.5, 0.45 * math.sqrt(theta) / thermo.simplified_sound_speed(rho) ** 2))
    simplified = dict(sp, dt=min(dts))
    nonclassical = {"U_ch": math.sqrt(pc / rc), "cases": {}}
    for name, (pl, rl_), (pr_, rr_), dlt, tstar in (
            ("fig4", (1.09, 0.879), (0.885, 0.562), 0.0125, 0.45),
            ("I", (1.6077, 1.01), (0.8957, 0.594), 0.329, 0.2),
            ("II", (3.00, 1.818), (0.575, 0.275), 0.0125, 0.15)):
        sides = {}
        for side, (pp, rr) in (("left", (pl, rl_)), ("right", (pr_, rr_))):
            rho = rr * rc
            sides[side] = {"rho": rho, "T": thermo.temperature(rho, pp * pc)}
        dt = min(dt_rule(sides[k]["rho"], sides[k]["T"], dlt) for k in sides)
        nonclassical["cases"][name] = dict(sides, delta=dlt, t_star=tstar, dt=dt)
    # the coexistence curve of the main text's Fig. 2: delta = 2/3 (time step by the rule at
    # the liquid density for that delta) and delta = 1/3 advected at U = 5 U_ch with
    # U_ch = sqrt(p_cr / rho_cr) (time step also capped at 0.5 / (1 + U))
    u_ch = math.sqrt(pc / rc)
    fig2 = {"U_ch": u_ch, "U": 5.0 * u_ch, "dt_delta_2_3": {}, "dt_advected": {}}
    for k in range(70, 96):
        key = "%.2f" % (k / 100.0)
        rl = coex[key]["rho_l"]
        fig2["dt_delta_2_3"][key] = dt_rule(rl, k / 100.0 * Tc, 2.0 / 3.0)
        fig2["dt_advected"][key] = min(coex[key]["dt"], 0.5 / (1.0 + 5.0 * u_ch))
    data = {
        "note": "written by oracle/write_workloads.py from oracle/thermo.py (vdW a=2/49, b=2/21, R=1, delta=1/3)",
        "critical": {"rho": rc, "T": Tc, "p": pc},
        "delta": DELTA,
        "coexistence": coex,
        "shock": shocks,
        "supercritical_1.10": {"dt": dt_rule(sup_rho, 1.1 * Tc)},
        "figure2": fig2,
        "dieterici": dieterici,
        "nonclassical": nonclassical,
        "simplified": simplified,
        # sound-pulse experiments: the time step of a uniform saturated vapour or liquid
        # (each by the rule at its own state), and of the critical state
        "sound": dict({"%.2f" % (k / 100.0): {
            "dt_v": dt_rule(coex["%.2f" % (k / 100.0)]["rho_v"], k / 100.0 * Tc),
            "dt_l": coex["%.2f" % (k / 100.0)]["dt"]} for k in range(70, 96)},
            critical={"dt": dt_rule(rc, Tc)}),
    }
    with open(OUT, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
        fh.write("\n")


if __name__ == "__main__":
    main()
