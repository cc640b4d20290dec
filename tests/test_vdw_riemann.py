"""The exact van der Waals Riemann solver (tests/vdw_riemann.py) and the oracle's shock
tubes against it: the SM's case I (delta = 0.329, classical: a fan and a shock), the
anomalous tube of the main text's Fig. 4 (delta = 0.0125, Gamma < 0: a rarefaction shock
and a compression fan) and the SM's case II (delta = 0.0125, Gamma changes sign along both
waves: a fan ended by a shock that is sonic ahead, and a shock sonic behind followed by a
compression fan).

The solver is pinned by what it does not compute itself: the fundamental derivative of
its isentropes against the SM's table, lab-frame Rankine-Hugoniot flux balances of every
shock, the self-similar relations inside every fan, and an independent first-order
finite-volume (Rusanov) solution of the same Euler equations that converges to it under
refinement."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import thermo
from paper_2002_09217_gb300 import inputs

import vdw_riemann as vr
from parity_util import params_of

HERE = os.path.dirname(os.path.abspath(__file__))
TAB = json.load(open(os.path.join(HERE, "..", "paper_2002_09217_gb300", "workloads.json")))["nonclassical"]


def problem(name):
    c = TAB["cases"][name]
    L, R = c["left"], c["right"]
    left = (L["rho"], 0.0, thermo.pressure(L["rho"], L["T"]))
    right = (R["rho"], 0.0, thermo.pressure(R["rho"], R["T"]))
    return c, left, right


@pytest.fixture(scope="module")
def solved():
    out = {}
    for name in ("I", "fig4", "II"):
        c, left, right = problem(name)
        out[name] = (c, left, right, vr.Riemann(c["delta"], left, right))
    return out


def test_gamma_of_the_isentropes_matches_the_sm_table():
    """Gamma = -v p_s''/(2 p_s') of the solver's explicit isentropes against the printed
    values (SM, shock-tube table), kept in tests/golden/shock_tube_gamma.txt."""
    want = {}
    for line in open(os.path.join(HERE, "golden", "shock_tube_gamma.txt")):
        parts = line.split()
        if len(parts) == 6 and not line.startswith("#"):
            want[(parts[0], parts[1])] = float(parts[5])
    assert len(want) == 4
    for name in ("I", "II"):
        c, left, right = problem(name)
        g = vr.Gas(c["delta"])
        assert g.gamma(1.0 / left[0], left[2]) == pytest.approx(want[(name, "L")], abs=6e-4)
        assert g.gamma(1.0 / right[0], right[2]) == pytest.approx(want[(name, "R")], abs=6e-4)
    c, left, right = problem("fig4")
    g = vr.Gas(c["delta"])
    assert g.gamma(1.0 / left[0], left[2]) < 0 and g.gamma(1.0 / right[0], right[2]) < 0


def test_wave_structures(solved):
    d = solved["I"][3].describe()
    assert d["wave1"] == ["fan"] and d["wave3"] == ["shock"]
    d = solved["fig4"][3].describe()
    # the left-moving wave expands the fluid through a shock, the right-moving one
    # compresses it through a fan
    assert d["wave1"] == ["shock"] and d["wave3"] == ["fan"]
    d = solved["II"][3].describe()
    assert d["wave1"] == ["fan", "shock"] and d["wave3"] == ["shock", "fan"]
    for name in ("I", "fig4", "II"):
        rp = solved[name][3]
        assert rp.mismatch < 1e-12
        assert solved[name][2][2] < rp.ps < solved[name][1][2]


def _conserved(gas, rho, u, p):
    v = 1.0 / rho
    E = gas.e(v, p) + 0.5 * u * u
    return np.array([rho, rho * u, rho * E]), np.array([rho * u, rho * u * u + p, u * (rho * E + p)])


def test_shocks_balance_the_lab_frame_fluxes(solved):
    """F(U_b) - F(U_a) = sigma (U_b - U_a) for mass, momentum and total energy."""
    n = 0
    for name in ("I", "fig4", "II"):
        rp = solved[name][3]
        for fam, waves in ((-1, rp.w1), (+1, rp.w3)):
            for w in waves:
                if w[0] != "shock":
                    continue
                (va, pa, ua), (vb, pb, ub), m = w[1], w[2], w[3]
                sigma = ua + fam * m * va
                Ua, Fa = _conserved(rp.g, 1.0 / va, ua, pa)
                Ub, Fb = _conserved(rp.g, 1.0 / vb, ub, pb)
                np.testing.assert_allclose(Fb - Fa, sigma * (Ub - Ua), rtol=1e-10, atol=1e-13)
                n += 1
    assert n == 4


def test_fans_are_self_similar_and_isentropic(solved):
    """Inside a fan of family k at x/t = xi: u + s c = xi, and T (v - b)^delta is that of the
    fan's base state."""
    for name in ("I", "fig4", "II"):
        c, left, right, rp = solved[name]
        g = rp.g
        for piece in rp.seg:
            if piece[0] != "fan":
                continue
            fam, base, va, vb, xa, xb = piece[1:]
            ent0 = g.T(base[0], base[1]) * (base[0] - g.b) ** g.d
            for xi in np.linspace(xa, xb, 7)[1:-1]:
                rho, u, p = rp.state_at(xi)
                v = 1.0 / rho
                assert u + fam.s * g.c(v, p) == pytest.approx(xi, abs=1e-10)
                assert g.T(v, p) * (v - g.b) ** g.d == pytest.approx(ent0, rel=1e-10)


def test_composite_waves_are_sonic_where_their_pieces_meet(solved):
    """Case II: the left wave's shock moves at the sound speed of the fan state it starts
    from (m = C ahead) and leaves a subsonic state; the right wave's shock leaves a state
    that is exactly sonic (m = C behind), from which the compression fan starts."""
    rp = solved["II"][3]
    g = rp.g
    fan, shock = rp.w1
    (va, pa, _), (vb, pb, _), m = shock[1], shock[2], shock[3]
    base = fan[1]
    assert m == pytest.approx(g.C(va, base[0], base[1]), rel=1e-9)
    assert m <= g.C(vb, vb, pb) * (1 + 1e-9)
    shock, fan = rp.w3
    (va, pa, _), (vb, pb, _), m = shock[1], shock[2], shock[3]
    assert m == pytest.approx(g.C(vb, vb, pb), rel=1e-9)
    assert fan[1][0] == vb


@pytest.mark.parametrize("name,bar", [("I", 3e-3), ("fig4", 6e-3), ("II", 6e-3)])
def test_exact_solution_is_the_limit_of_a_finite_volume_solution(solved, name, bar):
    c, left, right, rp = solved[name]
    t = c["t_star"] / TAB["U_ch"]
    l1 = []
    for n in (2000, 4000):
        x, rho, _, _ = vr.rusanov_tube(c["delta"], left, right, n, t)
        re, _, _ = rp.profile(x, t, 0.5)
        l1.append(np.abs(rho - re).mean() / np.abs(re).mean())
    assert l1[1] < bar and l1[1] < 0.8 * l1[0], l1


@pytest.mark.parametrize("name,bar", [("I", 3.5e-3), ("fig4", 1.1e-2), ("II", 1.2e-2)])
def test_oracle_tubes_converge_to_the_exact_solution(solved, name, bar):
    """The oracle's shock tubes at t* on 200 and 400 nodes: relative L1(rho) against the
    exact solution below the bar and falling with refinement (measured: case I 4.6e-3,
    2.7e-3, 1.5e-3 at 200, 400, 800 nodes; Fig. 4 1.4e-2, 8.7e-3, 5.6e-3; case II 1.5e-2,
    9.5e-3, 6.7e-3)."""
    rp = solved[name][3]
    l1 = []
    for nx in (200, 400):
        w = inputs.nonclassical_tube(name, nx=nx)
        P = params_of(w)
        st = oracle.step(P, oracle.init_state(P, *w.fields()), w.steps)
        rho = oracle.moments(P, st)["rho"][0]
        re, _, _ = rp.profile(np.arange(nx) + 0.5, w.steps * w.dt, nx / 2)
        l1.append(float(np.abs(rho - re).mean() / np.abs(re).mean()))
    assert l1[1] < bar and l1[1] < 0.75 * l1[0], l1
