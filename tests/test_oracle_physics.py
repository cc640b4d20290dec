"""Physics pins of the oracle: limits and benchmarks whose answers are fixed
independently of the scheme.

- ideal-gas limit (a = b = 0): Sod shock tube against the exact Riemann solution,
  with the error falling under refinement;
- Galilean boost: a run with every velocity raised by U (U*dt an integer number of
  nodes) equals the unboosted run shifted by U*dt per step, up to an interpolation error
  of the energy population that falls at high order under refinement;
- flat liquid-vapour interface: bulk densities against Maxwell's equal-area rule
  (main text, Fig. 2), for delta = 1/3 and 2/3;
- speed of sound (main text, Fig. 1): a pressure pulse in saturated vapour and liquid
  travels at the closed-form isentropic speed; at the critical point the measured speed
  converges to sqrt(2 p_cr v_cr) as the pulse widens;
- lagged interface / heat-flux terms against 1-D finite differences written here;
- thermodynamics: critical point, equal-area rule by quadrature, Rankine-Hugoniot
  closed form against a direct root solve;
- the Dieterici EoS (SM "Coexistence curve"): its critical point, the SM's reduced form,
  Maxwell densities that obey corresponding states and equal chemical potentials, and the
  oracle's isothermal flat interface on those densities;
- isothermal runs carry sound at the isothermal speed sqrt((dp/drho)_T) (SM figure);
- non-classical gas dynamics (main text, Fig. 4; SM "Shock tube"): the fundamental
  derivative against the SM's printed table and against finite differences along an
  isentrope; the anomalous tube's rarefaction keeps its steepness (a rarefaction shock)
  while the classical case's rarefaction spreads.
"""
import dataclasses
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle
from oracle import thermo

from exact_riemann import solve as riemann


def _sod(nx):
    w = 2.0 * nx / 400.0
    tend = 60.0 * nx / 400.0
    P = oracle.Params(nx=nx, ny=1, bc_x=1, a=0.0, b=0.0, delta=0.4, kappa=0.0, tau=1.0,
                      dt=0.5, p_floor=1e-6)
    x = np.arange(nx) + 0.5
    sw = 0.5 * (1.0 - np.tanh((x - nx / 2) / w))
    rho = (0.125 + 0.875 * sw)[None, :]
    p = (0.01 + 0.09 * sw)[None, :]
    st = oracle.init_state(P, rho, 0 * rho, 0 * rho, p / rho)
    st = oracle.step(P, st, int(round(tend / P.dt)))
    m = oracle.moments(P, st)
    ex = riemann(1.0, 0.0, 0.1, 0.125, 0.0, 0.01, 1.4, x, tend, nx / 2)
    l1 = lambda a, b: np.abs(a - b).sum() / np.abs(b).sum()
    return l1(m["rho"][0], ex[0]), l1(m["p"][0], ex[2])


def test_ideal_gas_sod_matches_exact_riemann_and_converges():
    """a = b = 0, delta = 0.4 (gamma = 1.4): the model is an ideal-gas kinetic
    scheme; density and pressure within 1.5 % (L1) of the exact solution at 400
    nodes, and closer at 800."""
    r400, p400 = _sod(400)
    r200, _ = _sod(200)
    assert r400 < 0.015 and p400 < 0.015
    assert r400 < r200


@pytest.mark.slow
def _boost_gap(nx, steps, U=2.0):
    """Largest difference per field between a run boosted by U along x and the
    unboosted run rolled by U*dt*steps nodes (ideal gas, periodic sine wave)."""
    P = oracle.Params(nx=nx, ny=4, a=0.0, b=0.0, delta=0.4, kappa=0.0, tau=1.0, dt=0.5,
                      p_floor=1e-6)
    X = np.arange(nx)[None, :] * np.ones((4, 1))
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * X / nx)
    T = np.full_like(rho, 0.12)
    shift = int(round(U * P.dt * steps))
    a = oracle.moments(P, oracle.step(P, oracle.init_state(P, rho, 0 * rho, 0 * rho, T), steps))
    b = oracle.moments(P, oracle.step(P, oracle.init_state(P, rho, 0 * rho + U, 0 * rho, T), steps))
    return {k: float(np.abs(np.roll(a[k], shift, axis=1) - (b[k] - (U if k == "ux" else 0.0))).max())
            for k in a}


def test_galilean_boost_is_a_shift():
    """Departure points, gauge differences and equilibria see only v - u, so the density
    and velocity after one step are exactly the shifted unboosted ones; the energy
    population's transfer map preserves moments only to second order per axis, so T
    differs by an interpolation error, which must shrink under refinement at the
    interpolation's order (a dropped or mis-signed u anywhere gives O(1) gaps)."""
    one = _boost_gap(24, 1)
    assert one["rho"] < 1e-13 and one["ux"] < 1e-13 and one["uy"] < 1e-13, one
    assert one["T"] < 1e-9, one
    coarse, fine = _boost_gap(24, 3), _boost_gap(48, 3)
    for k in ("rho", "ux", "T", "p"):
        assert fine[k] < coarse[k] / 16.0, (k, coarse, fine)
    assert coarse["T"] < 1e-7 and coarse["uy"] < 1e-13, coarse


def _oracle_pulse_speed(w, travel=0.3):
    """Speed of the right-going pressure pulse of an oracle run: slope of its centroid
    between the times it has travelled ~travel/3 and ~travel of the box."""
    P = oracle.Params(nx=w.nx, ny=w.ny, dt=w.dt, tau=w.tau, kappa=w.kappa, delta=w.delta,
                      p_floor=w.p_floor)
    st = oracle.init_state(P, *w.fields())
    x0 = w.nx / 4.0
    c_guess = thermo.sound_speed(w.rho[0, w.nx // 2], w.T[0, 0], w.delta)
    n2 = int(round(travel * w.nx / c_guess / w.dt))
    n1 = n2 // 3
    xs = np.arange(w.nx)
    sel = (xs >= x0) & (xs < x0 + w.nx / 2)
    cents = []
    done = 0
    for n in (n1, n2):
        st = oracle.step(P, st, n - done)
        done = n
        p = oracle.moments(P, st)["p"].mean(axis=0)
        d = np.clip(p[sel] - p[int(x0 + w.nx / 2) % w.nx], 0.0, None)
        cents.append((xs[sel] * d).sum() / d.sum())
    return (cents[1] - cents[0]) / ((n2 - n1) * w.dt), c_guess


@pytest.mark.parametrize("phase", ["vapour", "liquid"])
def test_sound_pulse_travels_at_the_isentropic_speed(phase):
    from paper_2002_09217_gb300 import inputs
    w = inputs.sound_pulse(0.9, phase, nx=400, width=6.0)
    c, c_th = _oracle_pulse_speed(w)
    # the closed form at the tabulated state (not the measurement's own guess)
    rv, rl = thermo.maxwell(0.9)
    want = thermo.sound_speed(rv if phase == "vapour" else rl, 0.9 * thermo.critical()[1], 1.0 / 3.0)
    assert c == pytest.approx(want, rel=1e-3)
    # the isothermal speed is clearly lower: the pulse is adiabatic, as it must be
    rho0 = rv if phase == "vapour" else rl
    T0 = 0.9 * thermo.critical()[1]
    c_T = math.sqrt(T0 / (1 - thermo.B_VDW * rho0) ** 2 - 2 * thermo.A_VDW * rho0)
    assert c > c_T * 1.05


def test_fp32_population_storage_slows_a_weak_pulse():
    """Why the mixed form's pulse is slower: rounding only the stored populations to FP32
    after every step (all arithmetic FP64) already slows a 1e-3 pulse by about a
    percent to a few percent, the more the smaller dt (a smaller per-step change is fewer
    ulps of the populations); rounding the stored gauge alone changes nothing."""
    from paper_2002_09217_gb300 import inputs
    w = inputs.sound_pulse(0.85, "vapour", nx=256, width=6.0)
    want = thermo.sound_speed(w.rho[0, w.nx // 2], w.T[0, 0], w.delta)

    def run(planes, dt):
        P = oracle.Params(nx=w.nx, ny=1, dt=dt, tau=w.tau, kappa=0.0, delta=w.delta, p_floor=w.p_floor)
        st = oracle.init_state(P, *w.fields())
        x0 = w.nx / 4.0
        xs = np.arange(w.nx)
        sel = (xs >= x0) & (xs < x0 + w.nx / 2)
        cents, done = [], 0
        n2 = int(round(0.3 * w.nx / want / dt))
        for n in (n2 // 3, n2):
            for _ in range(n - done):
                st = oracle.step(P, st, 1)
                st[planes] = st[planes].astype(np.float32).astype(np.float64)
            done = n
            p = oracle.moments(P, st)["p"][0]
            d = np.clip(p[sel] - p[int(x0 + w.nx / 2)], 0.0, None)
            cents.append((xs[sel] * d).sum() / d.sum())
        return (cents[1] - cents[0]) / ((n2 - n2 // 3) * dt) / want - 1.0

    pops, gauge = slice(0, 18), slice(18, 21)
    assert abs(run(gauge, 0.125)) < 1e-3
    e_quarter, e_eighth = run(pops, 0.25), run(pops, 0.125)
    assert -0.05 < e_quarter < -0.005, e_quarter
    assert e_eighth < e_quarter, (e_quarter, e_eighth)


def test_sound_speed_at_the_critical_point_converges_with_pulse_width():
    """(dp/drho)_T = 0 at the critical point, yet the adiabatic speed is finite,
    sqrt(2 p_cr v_cr); a finite pulse is slowed by dissipation, less so when wider."""
    from paper_2002_09217_gb300 import inputs
    rc, Tc, pc = thermo.critical()
    want = math.sqrt(2.0 * pc / rc)
    errs = []
    for nx, width in ((400, 6.0), (800, 12.0)):
        c, _ = _oracle_pulse_speed(inputs.sound_pulse(phase="critical", nx=nx, width=width))
        errs.append(abs(c / want - 1.0))
    assert errs[1] < 0.05 and errs[1] < errs[0] / 2.5, errs


def test_flat_interface_coexistence_matches_maxwell():
    """Slab of liquid in vapour at T = 0.9 T_cr: after relaxing, the bulk
    densities sit on Maxwell's equal-area values within 1 % (main text, Fig. 2)."""
    Tr = 0.9
    rc, Tc, pc = thermo.critical()
    rv, rl = thermo.maxwell(Tr)
    nx = 128
    P = oracle.Params(nx=nx, ny=1, kappa=0.02, tau=1.0, dt=0.5)
    x = np.arange(nx) + 0.5
    rho = (rv + (rl - rv) * 0.5 * (np.tanh((x - 32) / 4) - np.tanh((x - 96) / 4)))[None, :]
    st = oracle.init_state(P, rho, 0 * rho, 0 * rho, np.full_like(rho, Tr * Tc))
    st = oracle.step(P, st, 3000)
    acc_v = acc_l = 0.0
    n = 0
    for _ in range(10):
        st = oracle.step(P, st, 100)
        r = oracle.moments(P, st)["rho"][0]
        acc_v += r[:8].mean() + r[-8:].mean()
        acc_l += r[56:72].mean()
        n += 1
    assert acc_v / (2 * n) == pytest.approx(rv, rel=0.01)
    assert acc_l / n == pytest.approx(rl, rel=0.01)


def test_coexistence_does_not_depend_on_delta():
    """Fig. 2: the saturated densities are those of Maxwell's rule also for C_v = 3R/2
    (delta = 2/3), with its own (smaller) time step."""
    from paper_2002_09217_gb300 import experiments, inputs
    w = inputs.coexistence_slab(0.9, 2.0 / 3.0, nx=128, steps=4000)
    P = oracle.Params(nx=w.nx, ny=w.ny, dt=w.dt, tau=w.tau, kappa=w.kappa, delta=w.delta,
                      p_floor=w.p_floor)
    st = oracle.step(P, oracle.init_state(P, *w.fields()), 3000)
    rv_acc = rl_acc = 0.0
    for _ in range(5):
        st = oracle.step(P, st, 200)
        v, l = experiments.bulk_densities(oracle.moments(P, st)["rho"])
        rv_acc += v / 5
        rl_acc += l / 5
    rv, rl = thermo.maxwell(0.9)
    assert rv_acc == pytest.approx(rv, rel=0.01)
    assert rl_acc == pytest.approx(rl, rel=0.01)


def test_nonlocal_terms_match_one_dimensional_differences():
    """For fields varying in x only, the D2Q9 stencils reduce to the central
    differences d = (phi[x+1]-phi[x-1])/2, lap = phi[x+1]+phi[x-1]-2 phi[x]."""
    nx = 24
    P = oracle.Params(nx=nx, ny=3, kappa=0.03, tau=0.9, dt=0.6)
    x = np.arange(nx)
    rho = 3.5 + 1.2 * np.sin(2 * np.pi * x / nx) + 0.3 * np.cos(6 * np.pi * x / nx)
    T = 0.12 + 0.01 * np.sin(4 * np.pi * x / nx)
    nl = oracle.nonlocal_fields(P, np.tile(rho, (3, 1)), np.tile(T, (3, 1)))
    d = lambda f: (np.roll(f, -1) - np.roll(f, 1)) / 2.0
    lap = lambda f: np.roll(f, -1) + np.roll(f, 1) - 2.0 * f
    dr = d(rho)
    Kxx = -P.kappa * (rho * lap(rho) + 0.5 * dr * dr) + P.kappa * dr * dr
    np.testing.assert_allclose(nl[0, 1], -d(Kxx), rtol=1e-11, atol=1e-14)
    np.testing.assert_allclose(nl[1, 1], 0.0, atol=1e-14)
    np.testing.assert_allclose(nl[2, 1], 0.5 * P.kappa * dr * dr, rtol=1e-12, atol=1e-16)
    p = thermo.pressure(rho, T)
    h = (P.R / P.delta) * T - P.a * rho + p / rho
    mu = (P.tau - 0.5) * np.maximum(p, P.p_floor) * P.dt
    k = mu * (P.R / P.delta + P.R)
    q = -mu * d(h) + k * d(T)
    np.testing.assert_allclose(nl[3, 1], 2.0 * d(q), rtol=1e-10, atol=1e-14)


def test_heat_flux_source_vanishes_for_ideal_gas_default_conductivity():
    """With k = mu (C_v + R) and a = b = 0, h = (C_v + R) T so M_0 = 0."""
    P = oracle.Params(nx=10, ny=7, a=0.0, b=0.0, delta=0.4, tau=0.9)
    r = np.random.default_rng(3)
    nl = oracle.nonlocal_fields(P, r.uniform(0.5, 1.5, (7, 10)), r.uniform(0.1, 0.2, (7, 10)))
    assert np.abs(nl[3]).max() < 1e-15


# -------------------------------------------------------------- thermo
def test_critical_point_constants():
    rc, Tc, pc = thermo.critical()
    assert rc == pytest.approx(3.5)
    assert Tc == pytest.approx(8.0 / 63.0)
    assert pc == pytest.approx(1.0 / 6.0)
    # inflection of the critical isotherm: dp/drho = d2p/drho2 = 0
    h = 1e-4
    p = lambda r: thermo.pressure(r, Tc)
    assert (p(rc + h) - p(rc - h)) / (2 * h) == pytest.approx(0.0, abs=1e-7)
    assert (p(rc + h) - 2 * p(rc) + p(rc - h)) / h ** 2 == pytest.approx(0.0, abs=1e-4)


@pytest.mark.parametrize("Tr", [0.7, 0.8, 0.85, 0.9, 0.95])
def test_maxwell_equal_area_by_quadrature(Tr):
    rc, Tc, pc = thermo.critical()
    rv, rl = thermo.maxwell(Tr)
    T = Tr * Tc
    ps = thermo.pressure(rv, T)
    assert thermo.pressure(rl, T) == pytest.approx(ps, rel=1e-10)
    area, _ = integrate.quad(lambda v: thermo.pressure(1.0 / v, T) - ps, 1.0 / rl, 1.0 / rv,
                             epsabs=1e-14, epsrel=1e-13, limit=200)
    assert abs(area) < 1e-10


@pytest.mark.parametrize("Tr,Ma", [(0.8, 1.5), (0.9, 1.47), (0.7, 3.0), (0.95, 1.2)])
def test_rankine_hugoniot_closed_form_matches_root_solve(Tr, Ma):
    rc, Tc, pc = thermo.critical()
    rv, _ = thermo.maxwell(Tr)
    r1, u1, p1, T1 = thermo.post_shock_for_mach(rv, Tr * Tc, Ma, 1.0 / 3.0)
    M0, u, p = thermo.rh_root_solve(rv, thermo.pressure(rv, Tr * Tc), r1, 1.0 / 3.0)
    assert M0 == pytest.approx(Ma, rel=1e-10)
    assert u == pytest.approx(u1, rel=1e-10)
    assert p == pytest.approx(p1, rel=1e-10)


def test_sound_speed_at_critical_point():
    """The isentropic speed at the critical point is sqrt(2 p_cr v_cr) for delta =
    1/3... independent of delta it equals sqrt(R T_cr (1+delta)/(1-b rho_cr)^2 - 2 a rho_cr)."""
    rc, Tc, pc = thermo.critical()
    for delta in (1.0 / 3.0, 2.0 / 3.0):
        c = thermo.sound_speed(rc, Tc, delta)
        want = math.sqrt(Tc * (1 + delta) / (1 - thermo.B_VDW * rc) ** 2 - 2 * thermo.A_VDW * rc)
        assert c == pytest.approx(want, rel=1e-14)
    # at the critical point (dp/drho)_T = 0, so c^2 = (T/(rho^2 C_v)) (dp/dT)^2
    delta = 1.0 / 3.0
    dpdT = rc / (1 - thermo.B_VDW * rc)
    assert thermo.sound_speed(rc, Tc, delta) ** 2 == pytest.approx(Tc * dpdT ** 2 * delta / rc ** 2, rel=1e-12)


# ------------------------------------------------------------ Dieterici, isothermal
def test_dieterici_critical_point_and_reduced_form():
    rc, Tc, pc = thermo.dieterici_critical()
    h = 1e-4 * rc
    p = lambda r: thermo.dieterici_pressure(r, Tc)
    assert p(rc) == pytest.approx(pc, rel=1e-14)
    assert abs((p(rc + h) - p(rc - h)) / (2 * h)) < 1e-7 * pc / rc
    assert abs((p(rc + h) - 2 * p(rc) + p(rc - h)) / h ** 2) < 1e-5 * pc / rc ** 2
    rng = np.random.default_rng(5)
    for _ in range(20):
        rr, Tr = rng.uniform(0.1, 1.9), rng.uniform(0.6, 1.4)
        reduced = rr * Tr * math.e ** 2 / (2.0 - rr) * math.exp(-2.0 * rr / Tr)
        assert thermo.dieterici_pressure(rr * rc, Tr * Tc) / pc == pytest.approx(reduced, rel=1e-13)


@pytest.mark.parametrize("Tr", [0.7, 0.85, 0.95])
def test_dieterici_maxwell_equal_chemical_potential_and_corresponding_states(Tr):
    rv, rl = thermo.dieterici_maxwell(Tr)
    rc, Tc, pc = thermo.dieterici_critical()
    T = Tr * Tc
    assert thermo.dieterici_pressure(rv, T) == pytest.approx(thermo.dieterici_pressure(rl, T), rel=1e-12)
    # mu(rho_l) - mu(rho_v) = integral of (dp/drho)_T / rho, by Simpson's rule on the
    # analytic derivative (a different integrand from the equal-area solve)
    r = np.linspace(rv, rl, 20001)
    f = thermo.dieterici_dp_drho_T(r, T) / r
    dmu = integrate.simpson(f, x=r)
    assert abs(dmu) < 1e-9 * thermo.dieterici_pressure(rv, T) / rv
    # other constants, same reduced coexistence
    a2, b2 = 0.2, 0.05
    rv2, rl2 = thermo.dieterici_maxwell(Tr, a=a2, b=b2)
    rc2 = thermo.dieterici_critical(a2, b2)[0]
    assert rv2 / rc2 == pytest.approx(rv / rc, rel=1e-9)
    assert rl2 / rc2 == pytest.approx(rl / rc, rel=1e-9)


@pytest.mark.parametrize("Tr", [0.75, 0.9])
def test_isothermal_dieterici_flat_interface_on_maxwell(Tr):
    from paper_2002_09217_gb300 import experiments, inputs
    w = inputs.dieterici_slab(Tr, nx=128, steps=3000)
    P = oracle.Params(nx=w.nx, ny=w.ny, dt=w.dt, tau=w.tau, kappa=w.kappa, a=w.a, b=w.b,
                      p_floor=w.p_floor, eos="dieterici", isothermal=True, T_iso=w.T[0, 0])
    st = oracle.step(P, oracle.init_state(P, *w.fields()), w.steps)
    m = oracle.moments(P, st)
    v, l = experiments.bulk_densities(m["rho"])
    rv, rl = thermo.dieterici_maxwell(Tr)
    assert v == pytest.approx(rv, rel=0.01) and l == pytest.approx(rl, rel=0.01)
    np.testing.assert_allclose(m["T"], w.T[0, 0], rtol=1e-15)   # held


def test_isothermal_pulse_travels_at_the_isothermal_speed():
    from paper_2002_09217_gb300 import inputs
    w = inputs.sound_pulse(0.9, "vapour", nx=400, width=6.0, isothermal=True)
    P = oracle.Params(nx=w.nx, ny=w.ny, dt=w.dt, tau=w.tau, kappa=0.0, delta=w.delta,
                      p_floor=w.p_floor, isothermal=True, T_iso=w.T[0, 0])
    rho0, T0 = w.rho[0, w.nx // 2], w.T[0, 0]
    cT = math.sqrt(thermo.dp_drho_T(rho0, T0))
    st = oracle.init_state(P, *w.fields())
    x0 = w.nx / 4.0
    xs = np.arange(w.nx)
    sel = (xs >= x0) & (xs < x0 + w.nx / 2)
    n2 = int(round(0.3 * w.nx / cT / w.dt))
    cents, done = [], 0
    for n in (n2 // 3, n2):
        st = oracle.step(P, st, n - done)
        done = n
        p = oracle.moments(P, st)["p"][0]
        d = np.clip(p[sel] - p[int(x0 + w.nx / 2)], 0.0, None)
        cents.append((xs[sel] * d).sum() / d.sum())
    c = (cents[1] - cents[0]) / ((n2 - n2 // 3) * w.dt)
    assert c == pytest.approx(cT, rel=1e-3)
    assert c < 0.7 * thermo.sound_speed(rho0, T0, w.delta)


# ------------------------------------------------- current-time non-local terms
def test_current_time_nonlocal_terms_differ_from_lagged_at_second_order():
    """One step of the two-pass (current-time) variant differs from the lagged step by
    dt x (the force's change over dt) ~ dt^2 in the velocity, so halving dt divides the
    difference by ~4; the two coincide where the non-local terms vanish."""
    from paper_2002_09217_gb300 import inputs
    w = inputs.slab(nx=64, ny=1, Tr=0.9, amp=0.0, steps=1)
    base = oracle.Params(nx=w.nx, ny=1, tau=1.0, kappa=0.02, p_floor=w.p_floor)
    # a relaxed interface moving slowly: lagged and current terms differ by its motion
    st0 = oracle.init_state(dataclasses.replace(base, dt=0.25), w.rho, 0 * w.rho + 0.05, 0 * w.rho, w.T)
    st0 = oracle.step(dataclasses.replace(base, dt=0.25), st0, 40)
    gaps = []
    for dt in (0.2, 0.1):
        lag = oracle.moments(dataclasses.replace(base, dt=dt), oracle.step(dataclasses.replace(base, dt=dt), st0, 1))
        cur = oracle.moments(dataclasses.replace(base, dt=dt, nonlocal_="current"),
                             oracle.step(dataclasses.replace(base, dt=dt, nonlocal_="current"), st0, 1))
        gaps.append(np.abs(cur["ux"] - lag["ux"]).max())
    assert gaps[0] > 0.0
    assert 3.0 < gaps[0] / gaps[1] < 5.5, gaps
    # no interface, no heat flux: nothing to lag
    ideal = oracle.Params(nx=16, ny=1, a=0.0, b=0.0, delta=0.4, tau=1.0, dt=0.5, p_floor=1e-6)
    x = np.arange(16)[None, :]
    st = oracle.init_state(ideal, 1.0 + 0.1 * np.sin(2 * np.pi * x / 16), 0 * x + 0.0, 0 * x + 0.0,
                           np.full((1, 16), 0.1))
    a1 = oracle.step(ideal, st, 3)
    a2 = oracle.step(dataclasses.replace(ideal, nonlocal_="current"), st, 3)
    np.testing.assert_array_equal(a1, a2)


def test_current_time_variant_keeps_coexistence():
    from paper_2002_09217_gb300 import experiments, inputs
    w = inputs.coexistence_slab(0.9, nx=128, steps=3000)
    P = oracle.Params(nx=w.nx, ny=1, dt=w.dt, tau=w.tau, kappa=w.kappa, p_floor=w.p_floor,
                      nonlocal_="current")
    st = oracle.step(P, oracle.init_state(P, *w.fields()), w.steps)
    v, l = experiments.bulk_densities(oracle.moments(P, st)["rho"])
    rv, rl = thermo.maxwell(0.9)
    assert v == pytest.approx(rv, rel=0.01) and l == pytest.approx(rl, rel=0.01)


# ------------------------------------------------------------ non-classical dynamics
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "shock_tube_gamma.txt")


def test_fundamental_derivative_matches_the_printed_table():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 4
    rc, Tc, pc = thermo.critical()
    for case, side, p, r, d, want in rows:
        p, r, d, want = float(p), float(r), float(d), float(want)
        # reduced van der Waals constants (a = 3, b = 1/3) and the dimensional ones agree
        g_red = thermo.fundamental_derivative(p, r, d, a=3.0, b=1.0 / 3.0)
        g_dim = thermo.fundamental_derivative(p * pc, r * rc, d)
        assert g_red == pytest.approx(want, abs=6e-4), (case, side)
        assert g_dim == pytest.approx(g_red, rel=1e-12)


@pytest.mark.parametrize("p,r,d", [(1.09, 0.879, 0.0125), (0.885, 0.562, 0.0125), (1.6077, 1.01, 0.329)])
def test_fundamental_derivative_from_an_isentrope(p, r, d):
    """Gamma = (v^3 / 2c^2) p''(v) along the isentrope T (v - b)^delta = const of the vdW
    fluid with constant C_v, by finite differences: the same number as the closed form;
    the anomalous states of Fig. 4 have Gamma < 0."""
    rc, Tc, pc = thermo.critical()
    a, b, R = thermo.A_VDW, thermo.B_VDW, thermo.R_GAS
    v0 = 1.0 / (r * rc)
    K = thermo.temperature(r * rc, p * pc) * (v0 - b) ** d
    ps = lambda v: R * K * (v - b) ** (-d) / (v - b) - a / (v * v)
    h = 1e-4 * v0
    d1 = (ps(v0 + h) - ps(v0 - h)) / (2 * h)
    d2 = (ps(v0 + h) - 2 * ps(v0) + ps(v0 - h)) / (h * h)
    gamma = v0 ** 3 * d2 / (2.0 * (-v0 * v0 * d1))
    assert gamma == pytest.approx(thermo.fundamental_derivative(p * pc, r * rc, d), rel=1e-5, abs=1e-6)
    if d < 0.05 and p < 1.1:
        assert gamma < 0.0


def _oracle_steepness(case, nx=400):
    from paper_2002_09217_gb300 import inputs
    w = inputs.nonclassical_tube(case, nx=nx)
    P = oracle.Params(nx=w.nx, ny=1, bc_x=1, delta=w.delta, tau=w.tau, dt=w.dt, kappa=0.0,
                      p_floor=w.p_floor)
    st = oracle.init_state(P, *w.fields())
    out, done = [], 0
    for n in (w.steps // 2, w.steps):
        st = oracle.step(P, st, n - done)
        done = n
        r = oracle.moments(P, st)["rho"][0]
        g = np.abs(np.diff(r))
        il = int(np.argmax(g[: nx // 2]))
        out.append((g[il], il, g[nx // 2:].max(), r[max(0, il - 10)], r[il + 11]))
    return out


def test_anomalous_tube_has_a_rarefaction_shock():
    """Fig. 4 (delta = 0.0125, Gamma < 0 on both sides): the left-moving wave expands the
    fluid yet stays as steep from t*/2 to t* (a shock, not a fan)."""
    (g1, x1, _, _, _), (g2, x2, _, outer, inner) = _oracle_steepness("fig4")
    assert x2 < x1                       # it moves left
    assert outer > inner                 # the fluid behind it is less dense: an expansion
    assert g2 > 0.75 * g1, (g1, g2)


def test_classical_tube_has_a_rarefaction_fan():
    """Case I (delta = 0.329 > delta_BZT): the rarefaction spreads (its peak gradient
    about halves from t*/2 to t*) while the compression shock keeps its steepness."""
    (g1, x1, s1, _, _), (g2, x2, s2, _, _) = _oracle_steepness("I")
    assert x2 < x1
    assert g2 < 0.65 * g1, (g1, g2)
    assert s2 > 0.85 * s1, (s1, s2)


# -------------------------------------------------- simplified near-critical EoS
def test_double_well_coexistence_and_sound_speed_closed_forms():
    """Equal pressure p0 and equal chemical potential at rho_v, rho_l (Simpson on
    (dp/drho)/rho), and sqrt(dp/drho) = sqrt(2 beta rho) (rho_l - rho_v) there (SM)."""
    sp = thermo.SIMP
    rv, rl = sp["rho_v"], sp["rho_l"]
    assert thermo.simplified_pressure(rv) == pytest.approx(sp["p0"], rel=1e-15)
    assert thermo.simplified_pressure(rl) == pytest.approx(sp["p0"], rel=1e-15)
    r = np.linspace(rv, rl, 20001)
    h = 1e-6
    dpdr = (thermo.simplified_pressure(r + h) - thermo.simplified_pressure(r - h)) / (2 * h)
    assert abs(integrate.simpson(dpdr / r, x=r)) < 1e-9
    for rho in (rv, rl):
        want = math.sqrt(2 * sp["beta"] * rho) * (rl - rv)
        assert thermo.simplified_sound_speed(rho) == pytest.approx(want, rel=1e-14)


@pytest.mark.parametrize("phase", ["liquid", "vapour"])
def test_double_well_pulse_speed(phase):
    """Isothermal pulses in the saturated phases of the simplified EoS travel at the
    closed-form speed (SM figure of the speed of sound with this EoS)."""
    from paper_2002_09217_gb300 import inputs
    w = inputs.simplified_eos("pulse", phase, nx=400, pulse_width=6.0)
    P = oracle.Params(nx=w.nx, ny=1, dt=w.dt, tau=w.tau, kappa=0.0, p_floor=w.p_floor,
                      eos="simplified", isothermal=True, T_iso=w.T[0, 0], eos_params=w.eos_params)
    rho0 = w.rho[0, w.nx // 2]
    c_th = thermo.simplified_sound_speed(rho0)
    st = oracle.init_state(P, *w.fields())
    x0 = w.nx / 4.0
    xs = np.arange(w.nx)
    sel = (xs >= x0) & (xs < x0 + w.nx / 2)
    n2 = int(round(0.3 * w.nx / c_th / w.dt))
    cents, done = [], 0
    for n in (n2 // 3, n2):
        st = oracle.step(P, st, n - done)
        done = n
        p = oracle.moments(P, st)["p"][0]
        d = np.clip(p[sel] - p[int(x0 + w.nx / 2)], 0.0, None)
        cents.append((xs[sel] * d).sum() / d.sum())
    c = (cents[1] - cents[0]) / ((n2 - n2 // 3) * w.dt)
    assert c == pytest.approx(c_th, rel=1e-3)
