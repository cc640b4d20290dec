"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed-form
Maxwell-Boltzmann moments, a separately written Lagrange form of the transfer
matrix, numpy's linear solver, exact polynomial reproduction, exact copies for
integer shifts, conservation identities computed here from the moments, and
uniform states that must stay put.
"""
import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(20020921)
W = oracle.weights()
CX = np.array([i % 3 - 1 for i in range(9)], dtype=float)
CY = np.array([i // 3 - 1 for i in range(9)], dtype=float)
MOMS = [(0, 0), (1, 0), (0, 1), (1, 1), (2, 0), (0, 2), (2, 1), (1, 2), (2, 2)]
T_L = 1.0 / 3.0


def rand_gauge():
    return np.array([RNG.uniform(0.05, 0.8), RNG.uniform(-1.0, 1.0), RNG.uniform(-1.0, 1.0)])


def moments_here(lam, f):
    vx, vy = oracle.velocities(lam)
    return np.array([np.sum(f * vx ** m * vy ** n) for m, n in MOMS])


def lagrange_map_1d(s_src, u_src, s_dst, u_dst, k):
    """l_k evaluated at the three source velocities: Lagrange basis on the target
    velocities {u_dst - s_dst, u_dst, u_dst + s_dst} (index k = c + 1)."""
    nodes = [u_dst - s_dst, u_dst, u_dst + s_dst]
    out = []
    for a in range(3):
        v = s_src * (a - 1) + u_src
        num = 1.0
        den = 1.0
        for j in range(3):
            if j != k:
                num *= v - nodes[j]
                den *= nodes[k] - nodes[j]
        out.append(num / den)
    return np.array(out)


# ---------------------------------------------------------------- lattice
def test_weights_and_lattice_temperature():
    assert W.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.sum(W * CX * CX) == pytest.approx(T_L, abs=1e-15)
    assert np.sum(W * CX * CY) == pytest.approx(0.0, abs=1e-15)
    assert W[4] == pytest.approx(4.0 / 9.0)


@pytest.mark.parametrize("trial", range(5))
def test_equilibrium_moments_are_maxwell_boltzmann(trial):
    """rho W_i in gauge (theta, u) has the nine Maxwell-Boltzmann moments with
    temperature theta*T_L exactly (SM "Equilibrium")."""
    lam = rand_gauge()
    rho = RNG.uniform(0.2, 7.0)
    M = oracle.moment_matrix(lam)
    got = M @ (rho * W)
    th, ux, uy = lam
    sx, sy = ux * ux + th * T_L, uy * uy + th * T_L
    want = rho * np.array([1, ux, uy, ux * uy, sx, sy, sx * uy, ux * sy, sx * sy])
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------- transfer matrix
@pytest.mark.parametrize("trial", range(8))
def test_gauge_matrix_equals_separable_lagrange_map(trial):
    src, dst = rand_gauge(), rand_gauge()
    G = oracle.gauge_matrix(src, dst)
    ss, sd = np.sqrt(src[0]), np.sqrt(dst[0])
    want = np.zeros((9, 9))
    for i in range(9):
        kx, ky = i % 3, i // 3
        gx = lagrange_map_1d(ss, src[1], sd, dst[1], kx)
        gy = lagrange_map_1d(ss, src[2], sd, dst[2], ky)
        for j in range(9):
            want[i, j] = gx[j % 3] * gy[j // 3]
    np.testing.assert_allclose(G, want, rtol=1e-10, atol=1e-11)


@pytest.mark.parametrize("trial", range(5))
def test_gauge_matrix_equals_library_solve(trial):
    src, dst = rand_gauge(), rand_gauge()
    G = oracle.gauge_matrix(src, dst)
    want = np.linalg.solve(oracle.moment_matrix(dst), oracle.moment_matrix(src))
    np.testing.assert_allclose(G, want, rtol=1e-10, atol=1e-11)


@pytest.mark.parametrize("trial", range(5))
def test_gauge_preserves_nine_moments_identity_and_composition(trial):
    a, b, c = rand_gauge(), rand_gauge(), rand_gauge()
    f = RNG.uniform(0.0, 1.0, 9)
    fb = oracle.gauge_matrix(a, b) @ f
    np.testing.assert_allclose(moments_here(b, fb), moments_here(a, f), rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(oracle.gauge_matrix(a, a), np.eye(9), atol=1e-12)
    comp = oracle.gauge_matrix(b, c) @ oracle.gauge_matrix(a, b)
    np.testing.assert_allclose(comp, oracle.gauge_matrix(a, c), rtol=1e-9, atol=1e-10)


def test_printed_explicit_form_is_the_negated_map():
    """The dot-product form printed with the transfer matrix, taken literally
    (A = (u'-u)/sqrt3 - i sqrt(p/rho), B, w as printed, p/rho = theta T_L),
    equals minus the moment-matching map; the definition G = M'^-1 M is used."""
    src, dst = np.array([0.3, 0.1, -0.2]), np.array([0.45, -0.05, 0.15])
    p_rho, pp_rho = src[0] * T_L, dst[0] * T_L

    def g1(axis, i, j):
        A = (dst[axis] - src[axis]) / np.sqrt(3.0) - i * np.sqrt(p_rho)
        B = pp_rho if j == 0 else j * np.sqrt(pp_rho) * A
        return A * A - B

    def w(i):
        return 1.0 / pp_rho if i == 0 else -1.0 / (2.0 * pp_rho)

    lit = np.zeros((9, 9))
    for out in range(9):
        k, l = out % 3 - 1, out // 3 - 1
        for inn in range(9):
            i, j = inn % 3 - 1, inn // 3 - 1
            lit[out, inn] = w(k) * w(l) * g1(1, i, k) * g1(2, j, l)
    G = oracle.gauge_matrix(src, dst)
    # the printed form is separable with both factors negated -> overall sign +,
    # so compare the 1-D factors: each printed factor is -l_k
    gx_lit = np.array([[w(k) * g1(1, i, k) for i in (-1, 0, 1)] for k in (-1, 0, 1)])
    gx = np.array([lagrange_map_1d(np.sqrt(src[0]), src[1], np.sqrt(dst[0]), dst[1], k)
                   for k in range(3)])
    np.testing.assert_allclose(gx_lit, -gx, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(lit, G, rtol=1e-10, atol=1e-12)


# --------------------------------------------------------------- Lagrange
def test_lagrange_reproduces_cubics_and_nodes():
    for xi in RNG.uniform(1.0, 2.0, 20):
        a = oracle.lagrange4(xi)
        assert a.sum() == pytest.approx(1.0, abs=1e-14)
        for deg in range(4):
            assert np.dot(a, np.arange(4.0) ** deg) == pytest.approx(xi ** deg, rel=1e-13, abs=1e-13)
    for k in range(4):
        np.testing.assert_allclose(oracle.lagrange4(float(k)), np.eye(4)[k], atol=0)


# -------------------------------------------------------------- streaming
def _random_state(P, lam=None):
    N = P.nx * P.ny
    st = np.zeros((oracle.NPLANES, P.ny, P.nx))
    st[0:9] = RNG.uniform(0.1, 1.0, (9, P.ny, P.nx))
    st[9:18] = RNG.uniform(0.1, 1.0, (9, P.ny, P.nx))
    if lam is None:
        st[18] = RNG.uniform(0.1, 0.4, (P.ny, P.nx))
        st[19] = RNG.uniform(-0.2, 0.2, (P.ny, P.nx))
        st[20] = RNG.uniform(-0.2, 0.2, (P.ny, P.nx))
    else:
        st[18], st[19], st[20] = lam
    st[21] = RNG.uniform(1.0, 2.0, (P.ny, P.nx))
    st[22] = 0.13
    return st


def test_integer_shift_streaming_is_an_exact_copy():
    """Uniform gauge theta = 1, u = (1, 0): every departure point is a node, so
    f~_i(x) = f_i(x - c_i - (1,0)) exactly (Eqs. f/g streaming)."""
    P = oracle.Params(nx=7, ny=5)
    st = _random_state(P, lam=(1.0, 1.0, 0.0))
    for X, Y in [(0, 0), (3, 2), (6, 4)]:
        ft, gt = oracle.stream_node(P, st, X, Y, (1.0, 1.0, 0.0))
        for i in range(9):
            xs = (X - int(CX[i]) - 1) % P.nx
            ys = (Y - int(CY[i])) % P.ny
            assert ft[i] == pytest.approx(st[i, ys, xs], rel=1e-13, abs=1e-13)
            assert gt[i] == pytest.approx(st[9 + i, ys, xs], rel=1e-13, abs=1e-13)


def test_uniform_gauge_streaming_conserves_each_direction_sum():
    """All nodes in one gauge, periodic: the Lagrange weights sum to one and the
    stencil is shift invariant, so sum_x f~_i = sum_x f_i for every i."""
    P = oracle.Params(nx=9, ny=8)
    lam = (0.37, 0.23, -0.41)
    st = _random_state(P, lam=lam)
    tot_f = np.zeros(9)
    tot_g = np.zeros(9)
    for Y in range(P.ny):
        for X in range(P.nx):
            ft, gt = oracle.stream_node(P, st, X, Y, lam)
            tot_f += ft
            tot_g += gt
    np.testing.assert_allclose(tot_f, st[0:9].sum(axis=(1, 2)), rtol=1e-12)
    np.testing.assert_allclose(tot_g, st[9:18].sum(axis=(1, 2)), rtol=1e-12)


def test_streaming_of_smooth_field_is_fourth_order_accurate():
    """A cubic-in-x population field (all nodes in one gauge, zero-gradient far
    away) is reconstructed exactly at interior departure points."""
    P = oracle.Params(nx=16, ny=6, bc_x=1, bc_y=0)
    lam = (0.29, 0.17, 0.0)
    st = _random_state(P, lam=lam)
    x = np.arange(P.nx, dtype=float)
    poly = lambda xx: 0.5 + 0.1 * xx - 0.01 * xx ** 2 + 0.0004 * xx ** 3
    for i in range(18):
        st[i] = poly(x)[None, :] * (1.0 + 0.1 * (i % 9))
    vx, _ = oracle.velocities(lam)
    ft, _ = oracle.stream_node(P, st, 8, 3, lam)
    for i in range(9):
        assert ft[i] == pytest.approx(poly(8 - vx[i]) * (1.0 + 0.1 * i), rel=1e-12)


# -------------------------------------------------------------- collision
def _collision_case(with_force=True):
    P = oracle.Params(nx=4, ny=4, tau=0.9, dt=0.7)
    lam = np.array([0.21, 0.13, -0.07])
    rho = 3.1
    f = rho * W * (1.0 + 0.05 * RNG.uniform(-1, 1, 9))
    g = f * 0.4 * (1.0 + 0.05 * RNG.uniform(-1, 1, 9))
    F = (0.011, -0.006) if with_force else (0.0, 0.0)
    rEl = 0.002 if with_force else 0.0
    mac = oracle.macro(P, lam, f, g, F[0], F[1], rEl)
    return P, lam, f, g, F, rEl, mac


def test_macro_fields_follow_the_moment_definitions():
    P, lam, f, g, F, rEl, mac = _collision_case()
    vx, vy = oracle.velocities(lam)
    rho = f.sum()
    ux, uy = (f * vx).sum() / rho, (f * vy).sum() / rho
    assert mac["rho"] == pytest.approx(rho, rel=1e-14)
    assert mac["ux"] == pytest.approx(ux, rel=1e-13)
    uhx = ux + F[0] * P.dt / (2 * rho)
    assert mac["uhx"] == pytest.approx(uhx, rel=1e-13)
    E = g.sum() / (2 * rho)
    e = E - 0.5 * (mac["uhx"] ** 2 + mac["uhy"] ** 2) - rEl / rho
    T = (e + P.a * rho) * P.delta / P.R
    assert mac["T"] == pytest.approx(T, rel=1e-12)
    p = rho * P.R * T / (1 - P.b * rho) - P.a * rho ** 2
    assert mac["p"] == pytest.approx(p, rel=1e-12)
    assert mac["theta"] == pytest.approx(max(p, P.p_floor) / (rho * T_L), rel=1e-12)


def test_collision_conserves_mass_momentum_and_energy_budget():
    """sum f* = rho, sum f* v = rho u + F dt, sum g* = sum g~ + dt (M_0 + 2 uhat.F)
    (Eqs. f/g collision with S_i, gtilde and phi; force-work reading)."""
    P, lam, f, g, F, rEl, mac = _collision_case()
    M0 = 0.0037
    fo, go = oracle.collide(P, lam, f, g, mac, F[0], F[1], M0)
    vx, vy = oracle.velocities(lam)
    rho = f.sum()
    assert fo.sum() == pytest.approx(rho, rel=1e-13)
    assert (fo * vx).sum() == pytest.approx((f * vx).sum() + F[0] * P.dt, rel=1e-12, abs=1e-14)
    assert (fo * vy).sum() == pytest.approx((f * vy).sum() + F[1] * P.dt, rel=1e-12, abs=1e-14)
    work = 2.0 * (mac["uhx"] * F[0] + mac["uhy"] * F[1])
    assert go.sum() == pytest.approx(g.sum() + P.dt * (M0 + work), rel=1e-12)


def test_heat_flux_correction_has_only_a_zeroth_moment():
    """gtilde sums to M_0 and carries no momentum-like first moment (Eq. gtilde)."""
    P, lam, f, g, F, rEl, mac = _collision_case(with_force=False)
    _, g0 = oracle.collide(P, lam, f, g, mac, 0.0, 0.0, 0.0)
    _, g1 = oracle.collide(P, lam, f, g, mac, 0.0, 0.0, 0.05)
    d = (g1 - g0) / P.dt
    vx, vy = oracle.velocities(lam)
    assert d.sum() == pytest.approx(0.05, rel=1e-12)
    assert abs((d * vx).sum()) < 1e-14 and abs((d * vy).sum()) < 1e-14


def test_unforced_equilibria_have_the_target_moments():
    """With omega = 1 and no force, f* = f^eq and g* = g^eq: their moments are
    rho, rho u, and 2 rho E, 2 rho u H with H = E + P/rho (Eq. geq, SM heat flux)."""
    P, lam, f, g, F, rEl, mac = _collision_case(with_force=False)
    P.tau = 1.0
    fo, go = oracle.collide(P, lam, f, g, mac, 0.0, 0.0, 0.0)
    vx, vy = oracle.velocities(lam)
    rho, ux, uy, E = mac["rho"], mac["ux"], mac["uy"], mac["E"]
    H = E + mac["P"] / rho
    assert go.sum() == pytest.approx(2 * rho * E, rel=1e-12)
    assert (go * vx).sum() == pytest.approx(2 * rho * ux * H, rel=1e-11)
    assert (go * vy).sum() == pytest.approx(2 * rho * uy * H, rel=1e-11)
    # pressure tensor of f^eq: rho u u + P I (equilibrium moments of the co-moving frame)
    assert (fo * vx * vx).sum() == pytest.approx(rho * ux * ux + mac["P"], rel=1e-11)
    assert (fo * vx * vy).sum() == pytest.approx(rho * ux * uy, rel=1e-10, abs=1e-14)


def test_forced_g_equilibrium_carries_uhat_H_flux():
    """With the force, the forced g^eq has sum = 2 rho E and first moment
    2 rho uhat H (SM, heat flux with force), checked with omega = 1 after removing
    the separately defined phi source."""
    P, lam, f, g, F, rEl, mac = _collision_case(with_force=True)
    P.tau = 1.0
    _, go = oracle.collide(P, lam, f, g, mac, F[0], F[1], 0.0)
    vx, vy = oracle.velocities(lam)
    rho, E = mac["rho"], mac["E"]
    H = E + mac["P"] / rho
    work = 2.0 * (mac["uhx"] * F[0] + mac["uhy"] * F[1])
    # phi_i = 2 W_i uhat.F in the co-moving frame: zeroth moment = work,
    # first moment = work * u
    geq_sum = go.sum() - P.dt * work
    geq_vx = (go * vx).sum() - P.dt * work * mac["ux"]
    assert geq_sum == pytest.approx(2 * rho * E, rel=1e-12)
    assert geq_vx == pytest.approx(2 * rho * mac["uhx"] * H, rel=1e-10)


@pytest.mark.parametrize("lattice", ["d2q9", "d2q16"])
@pytest.mark.parametrize("force", [(0.09, -0.05), (-0.02, 0.13), (0.0, 0.0)])
def test_forced_g_equilibrium_second_moment_is_the_paper_R(lattice, force):
    """Second moment of the forced g equilibrium (SM, Chapman-Enskog with force, the
    modified equilibrium moments): R_ab = sum g^eq v_a v_b
    = 2 rho uhat_a uhat_b (H + P/rho) + 2 P H delta_ab, with H = E + P/rho and E the
    total energy per mass (reading R8).  The force tensor I = uhat F + F uhat +
    dt F F E/(2P) inside M and N cancels from the zeroth and first moments but not from
    this one: a wrong factor, a dropped F F term or a missing off-diagonal entry of I
    changes R.  The force is strong enough for the dt^2 F F part to count (about 0.5 %
    of R_xx).  Checked with omega = 1, M_0 = 0 and the phi source (2 W_i uhat.F in the
    co-moving frame, second moment work (P/rho delta + u u)) removed."""
    rng = np.random.default_rng(5150)
    W_l = oracle.weights(lattice)
    Q = len(W_l)
    P = oracle.Params(nx=4, ny=4, tau=1.0, dt=0.7, lattice=lattice)
    lam = np.array([0.21 if lattice == "d2q9" else 0.07, 0.13, -0.07])
    rho = 3.1
    f = rho * W_l * (1.0 + 0.05 * rng.uniform(-1, 1, Q))
    g = f * 0.4 * (1.0 + 0.05 * rng.uniform(-1, 1, Q))
    mac = oracle.macro(P, lam, f, g, force[0], force[1], 0.002)
    assert mac["p"] > P.p_floor   # the case uses the van der Waals pressure itself
    _, go = oracle.collide(P, lam, f, g, mac, force[0], force[1], 0.0)
    vx, vy = oracle.velocities(lam, lattice)
    rho_, E, Pg = mac["rho"], mac["E"], mac["P"]
    uh = np.array([mac["uhx"], mac["uhy"]])
    u = np.array([mac["ux"], mac["uy"]])
    H = E + Pg / rho_
    work = 2.0 * (uh[0] * force[0] + uh[1] * force[1])
    v = (vx, vy)
    for a in range(2):
        for b in range(2):
            phi_ab = work * ((Pg / rho_) * (a == b) + u[a] * u[b])
            R_ab = (go * v[a] * v[b]).sum() - P.dt * phi_ab
            want = 2 * rho_ * uh[a] * uh[b] * (H + Pg / rho_) + 2 * Pg * H * (a == b)
            assert R_ab == pytest.approx(want, rel=1e-11, abs=1e-14), (a, b)


# ------------------------------------------------------------- whole step
@pytest.mark.parametrize("u", [(0.0, 0.0), (0.37, -0.21), (-1.3, 0.8)])
def test_uniform_state_is_stationary_for_any_velocity(u):
    P = oracle.Params(nx=6, ny=5, dt=0.5, tau=1.0)
    rho = np.full((5, 6), 2.3)
    st = oracle.init_state(P, rho, np.full_like(rho, u[0]), np.full_like(rho, u[1]),
                           np.full_like(rho, 0.14))
    out = oracle.step(P, st, 3)
    m = oracle.moments(P, out)
    np.testing.assert_allclose(m["rho"], 2.3, rtol=1e-13)
    np.testing.assert_allclose(m["ux"], u[0], atol=1e-13)
    np.testing.assert_allclose(m["uy"], u[1], atol=1e-13)
    np.testing.assert_allclose(m["T"], 0.14, rtol=1e-12)


def test_periodic_step_conserves_mass_to_round_off_in_a_uniform_gauge_flow():
    """Density perturbation on a uniformly moving, isothermal-gauge background:
    total mass drifts only through interpolation between unequal gauges, which is
    second order in the perturbation."""
    P = oracle.Params(nx=16, ny=8, dt=0.5, tau=1.0)
    x = np.arange(16)[None, :] * np.ones((8, 1))
    rho = 2.0 * (1.0 + 1e-4 * np.sin(2 * np.pi * x / 16))
    st = oracle.init_state(P, rho, np.full_like(rho, 0.2), np.zeros_like(rho), np.full_like(rho, 0.14))
    out = oracle.step(P, st, 4)
    m0 = oracle.moments(P, st)["rho"].sum()
    m1 = oracle.moments(P, out)["rho"].sum()
    assert abs(m1 / m0 - 1.0) < 1e-9


def test_step_nodes_matches_full_step():
    P = oracle.Params(nx=12, ny=6, dt=0.5, tau=1.0, kappa=0.02)
    x = np.arange(12)[None, :] * np.ones((6, 1))
    rho = 3.0 + 1.5 * np.tanh((x - 6) / 2.0)
    st = oracle.init_state(P, rho, 0.05 * np.ones_like(rho), np.zeros_like(rho), np.full_like(rho, 0.12))
    full = oracle.step(P, st, 1)
    nodes = np.array([0, 5, 17, 40, 71])
    part = oracle.step_nodes(P, st, nodes)
    flat = full.reshape(oracle.NPLANES, -1)
    np.testing.assert_array_equal(part, flat[:, nodes].T)
