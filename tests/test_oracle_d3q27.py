"""Pins of the 3-D (D3Q27) oracle.

The model is written for D dimensions; on D3Q27 = C1^3 (C1 = {-1, 0, 1}, W = 1/6, 2/3,
1/6 per axis, T_L = 1/3) it is checked against what fixes it independently:

- on a grid one node thick in z (or in y) the z- (y-) marginals of the populations obey
  exactly the D2Q9 scheme (partition of unity of the per-axis transfer map and of the
  reconstruction, Sigma_z W_z = 1, and D/2 = 3/2 against 1 in the heat-flux correction,
  cancelled by the extra theta T_L of v^2): the 3-D oracle must reproduce the pinned D2Q9
  oracle there, with the Korteweg force and heat flux active;
- exchanging axes of the input exchanges them in the result (a swapped index or a
  dropped z term breaks it);
- rho W_i carries the 27 Maxwell-Boltzmann moments M_lmn, l, m, n <= 2, of temperature
  theta T_L; the transfer matrix equals the product of three 3-node Lagrange maps and
  numpy's solve, and preserves the 27 moments;
- uniform states at any velocity are stationary; a single-node step equals the full step;
- a shear wave along z decays at the kinematic viscosity (tau - 1/2)(p/rho) dt of the
  main text (the 3-D collision and the z streaming together).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import core3d as o3

RNG = np.random.default_rng(327)
T_L = 1.0 / 3.0


def smooth_fields(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    rho = 1.6 + 0.35 * np.sin(2 * np.pi * x / nx + 0.3) * np.cos(2 * np.pi * y / ny) * np.cos(2 * np.pi * z / nz + 0.1)
    ux = 0.04 * np.cos(2 * np.pi * y / ny) * np.sin(2 * np.pi * z / nz)
    uy = 0.03 * np.sin(2 * np.pi * x / nx) + 0.01 * np.cos(2 * np.pi * z / nz)
    uz = 0.02 * np.cos(2 * np.pi * x / nx) * np.sin(2 * np.pi * y / ny)
    T = 0.28 + 0.01 * np.cos(2 * np.pi * (x / nx + y / ny))
    return rho, ux, uy, uz, T


def test_one_plane_in_z_reduces_to_d2q9():
    nx, ny = 10, 6
    rho, ux, uy, _, T = smooth_fields(nx, ny, 1)
    P2 = oracle.Params(nx=nx, ny=ny, kappa=0.02, tau=0.9, dt=0.5)
    P3 = o3.Params3(nx=nx, ny=ny, nz=1, kappa=0.02, tau=0.9, dt=0.5)
    m2 = oracle.moments(P2, oracle.step(P2, oracle.init_state(P2, rho[0], ux[0], uy[0], T[0]), 5))
    m3 = o3.moments(P3, o3.step(P3, o3.init_state(P3, rho, ux, uy, 0 * rho, T), 5))
    for k in ("rho", "ux", "uy", "T", "p"):
        err = np.abs(m3[k][0] - m2[k]).max() / max(np.abs(m2[k]).max(), 0.1)
        assert err < 1e-12, (k, err)
    assert np.abs(m3["uz"]).max() < 1e-13


def test_one_plane_in_y_reduces_to_d2q9_in_the_xz_plane():
    """The z axis itself: D3Q27 on (nx, 1, nz) equals D2Q9 on (nx, nz) with (u_x, u_z) in
    the role of (u_x, u_y), zero-gradient ends in z."""
    nx, nz = 9, 7
    rho, ux, _, uz, T = smooth_fields(nx, 1, nz)
    P2 = oracle.Params(nx=nx, ny=nz, bc_y=1, kappa=0.02, tau=0.9, dt=0.5)
    P3 = o3.Params3(nx=nx, ny=1, nz=nz, bc_z=1, kappa=0.02, tau=0.9, dt=0.5)
    f2 = [a[:, 0, :] for a in (rho, ux, uz, T)]
    m2 = oracle.moments(P2, oracle.step(P2, oracle.init_state(P2, *f2), 4))
    m3 = o3.moments(P3, o3.step(P3, o3.init_state(P3, rho, ux, 0 * rho, uz, T), 4))
    pairs = {"rho": "rho", "ux": "ux", "uz": "uy", "T": "T", "p": "p"}
    for k3, k2 in pairs.items():
        err = np.abs(m3[k3][:, 0, :] - m2[k2]).max() / max(np.abs(m2[k2]).max(), 0.1)
        assert err < 1e-12, (k3, err)
    assert np.abs(m3["uy"]).max() < 1e-13


def test_exchanging_axes_exchanges_the_result():
    nx, ny, nz = 5, 4, 3
    rho, ux, uy, uz, T = smooth_fields(nx, ny, nz)
    P = o3.Params3(nx=nx, ny=ny, nz=nz, kappa=0.02, tau=0.9, dt=0.5)
    a = o3.moments(P, o3.step(P, o3.init_state(P, rho, ux, uy, uz, T), 2))
    # x <-> z: arrays (z, y, x) -> (x, y, z), velocities u_x <-> u_z
    tr = lambda v: np.ascontiguousarray(np.transpose(v, (2, 1, 0)))
    Q = o3.Params3(nx=nz, ny=ny, nz=nx, kappa=0.02, tau=0.9, dt=0.5)
    b = o3.moments(Q, o3.step(Q, o3.init_state(Q, tr(rho), tr(uz), tr(uy), tr(ux), tr(T)), 2))
    swap = {"rho": "rho", "ux": "uz", "uy": "uy", "uz": "ux", "T": "T", "p": "p"}
    for ka, kb in swap.items():
        err = np.abs(tr(a[ka]) - b[kb]).max() / max(np.abs(a[ka]).max(), 0.1)
        assert err < 1e-12, (ka, err)


def rand_gauge():
    return np.array([RNG.uniform(0.05, 0.8), RNG.uniform(-1, 1), RNG.uniform(-1, 1), RNG.uniform(-1, 1)])


def velocities(lam):
    s = math.sqrt(lam[0])
    c = np.array([(i % 3 - 1, (i // 3) % 3 - 1, i // 9 - 1) for i in range(27)], dtype=float)
    return s * c + lam[1:]


def test_equilibrium_has_the_27_maxwell_moments():
    def raw(u, var, m):
        return [1.0, u, u * u + var][m]
    for _ in range(4):
        lam = rand_gauge()
        rho = RNG.uniform(0.2, 5.0)
        got = o3.moment_matrix(lam) @ (rho * o3.weights())
        var = lam[0] * T_L
        want = [rho * raw(lam[1], var, r % 3) * raw(lam[2], var, (r // 3) % 3) * raw(lam[3], var, r // 9)
                for r in range(27)]
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


def test_gauge_matrix_is_a_product_of_three_lagrange_maps():
    def map1(s_src, u_src, s_dst, u_dst):
        nodes = s_dst * np.array([-1.0, 0.0, 1.0]) + u_dst
        G = np.zeros((3, 3))
        for k in range(3):
            for a in range(3):
                v = s_src * (a - 1) + u_src
                G[k, a] = np.prod([(v - nodes[j]) / (nodes[k] - nodes[j]) for j in range(3) if j != k])
        return G
    for _ in range(4):
        src, dst = rand_gauge(), rand_gauge()
        G = o3.gauge_matrix(src, dst)
        ss, sd = math.sqrt(src[0]), math.sqrt(dst[0])
        want = np.kron(map1(ss, src[3], sd, dst[3]), np.kron(map1(ss, src[2], sd, dst[2]), map1(ss, src[1], sd, dst[1])))
        np.testing.assert_allclose(G, want, rtol=1e-9, atol=1e-10)
        lib = np.linalg.solve(o3.moment_matrix(dst), o3.moment_matrix(src))
        np.testing.assert_allclose(G, lib, rtol=1e-9, atol=1e-10)
        f = RNG.uniform(0, 1, 27)
        va, vb = velocities(src), velocities(dst)
        fb = G @ f
        for r in range(27):
            l, m, n = r % 3, (r // 3) % 3, r // 9
            ma = np.sum(f * va[:, 0] ** l * va[:, 1] ** m * va[:, 2] ** n)
            mb = np.sum(fb * vb[:, 0] ** l * vb[:, 1] ** m * vb[:, 2] ** n)
            assert mb == pytest.approx(ma, rel=1e-10, abs=1e-11)


@pytest.mark.parametrize("u", [(0.0, 0.0, 0.0), (0.3, -0.2, 0.45)])
def test_uniform_state_is_stationary(u):
    P = o3.Params3(nx=4, ny=3, nz=3, dt=0.5, tau=1.0)
    shp = (3, 3, 4)
    st = o3.init_state(P, np.full(shp, 2.1), np.full(shp, u[0]), np.full(shp, u[1]), np.full(shp, u[2]),
                       np.full(shp, 0.15))
    m = o3.moments(P, o3.step(P, st, 2))
    np.testing.assert_allclose(m["rho"], 2.1, rtol=1e-13)
    for k, v in zip(("ux", "uy", "uz"), u):
        np.testing.assert_allclose(m[k], v, atol=1e-13)
    np.testing.assert_allclose(m["T"], 0.15, rtol=1e-12)


def test_step_nodes_matches_full_step():
    nx, ny, nz = 5, 4, 3
    P = o3.Params3(nx=nx, ny=ny, nz=nz, kappa=0.02, tau=0.9, dt=0.5)
    st = o3.init_state(P, *smooth_fields(nx, ny, nz))
    full = o3.step(P, st, 1).reshape(o3.NPLANES, -1)
    nodes = np.array([0, 7, 23, 41, 59])
    np.testing.assert_array_equal(o3.step_nodes(P, st, nodes), full[:, nodes].T)


def test_shear_wave_along_z_decays_at_the_kinematic_viscosity():
    """u_x = U sin(k z) on a 1 x 1 x 32 column of an ideal gas: decay rate nu k^2 with
    nu = (tau - 1/2) (p/rho) dt, within 3 % at 32 nodes per wavelength (the D2Q9 figure
    at that resolution is 2.6 %)."""
    nz, U, T0 = 32, 1e-4, 0.12
    P = o3.Params3(nx=1, ny=1, nz=nz, a=0.0, b=0.0, delta=0.4, kappa=0.0, tau=0.9, dt=0.5, p_floor=1e-6)
    z = (np.arange(nz)[:, None, None] * np.ones((1, 1, 1))).astype(float)
    k = 2 * np.pi / nz
    one = np.ones_like(z)
    st = o3.init_state(P, one, U * np.sin(k * z), 0 * z, 0 * z, T0 * one)
    amp = lambda s: 2.0 * np.mean(o3.moments(P, s)["ux"][:, 0, 0] * np.sin(k * z[:, 0, 0]))
    a0 = amp(st)
    steps = 40
    a1 = amp(o3.step(P, st, steps))
    got = -math.log(a1 / a0) / (steps * P.dt)
    want = (P.tau - 0.5) * T0 * P.dt * k * k
    assert got == pytest.approx(want, rel=0.03), (got, want)


def test_galilean_boost_along_z_is_a_shift():
    """A run boosted by U along z (U dt = one node) equals the unboosted run shifted by one
    node after one step: density and velocity to round-off (departure points, gauge
    differences and equilibria see only v - u), T to the interpolation error of the energy
    population (the 3-node maps keep second moments per axis, as on D2Q9)."""
    nz, U = 12, 2.0
    P = o3.Params3(nx=2, ny=2, nz=nz, a=0.0, b=0.0, delta=0.4, kappa=0.0, tau=1.0, dt=0.5, p_floor=1e-6)
    z = np.arange(nz)[:, None, None] * np.ones((1, 2, 2))
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * z / nz)
    T = np.full_like(rho, 0.12)
    a = o3.moments(P, o3.step(P, o3.init_state(P, rho, 0 * rho, 0 * rho, 0 * rho, T), 1))
    b = o3.moments(P, o3.step(P, o3.init_state(P, rho, 0 * rho, 0 * rho, 0 * rho + U, T), 1))
    for k, bar in (("rho", 1e-11), ("ux", 1e-12), ("uy", 1e-12), ("uz", 1e-11), ("T", 1e-8)):
        gap = np.abs(np.roll(a[k], 1, axis=0) - (b[k] - (U if k == "uz" else 0.0))).max()
        assert gap < bar, (k, gap)


@pytest.mark.parametrize("force", [(0.07, -0.04, 0.05), (0.0, 0.11, -0.03)])
def test_forced_g_equilibrium_second_moment_is_the_paper_R_in_3d(force):
    """The forced g equilibrium's second moment in three dimensions (SM, Chapman-Enskog
    with force, the modified equilibrium moments; reading R18 for the 3-D tensors):
    sum g^eq v_a v_b = 2 rho uhat_a uhat_b (H + P/rho) + 2 P H delta_ab for all nine
    (a, b), with omega = 1, M_0 = 0 and the force-work source phi (2 W_i uhat.F in the
    co-moving frame) removed.  Also the zeroth and first moments 2 rho E, 2 rho uhat H."""
    rng = np.random.default_rng(2718)
    w = o3.weights()
    P = o3.Params3(nx=4, ny=4, nz=4, tau=1.0, dt=0.6)
    lam = np.array([0.19, 0.11, -0.06, 0.04])
    rho = 2.9
    f = rho * w * (1.0 + 0.05 * rng.uniform(-1, 1, 27))
    g = f * 0.4 * (1.0 + 0.05 * rng.uniform(-1, 1, 27))
    mac = o3.macro(P, lam, f, g, force, 0.002)
    assert mac["p"] > P.p_floor
    _, go = o3.collide(P, lam, f, g, mac, force, 0.0)
    s = math.sqrt(lam[0])
    c = np.array([[i % 3 - 1, (i // 3) % 3 - 1, i // 9 - 1] for i in range(27)], dtype=float)
    v = s * c + lam[1:][None, :]
    rho_, E, Pg = mac["rho"], mac["E"], mac["P"]
    uh = np.array([mac["uhx"], mac["uhy"], mac["uhz"]])
    u = np.array([mac["ux"], mac["uy"], mac["uz"]])
    H = E + Pg / rho_
    work = 2.0 * float(uh @ np.asarray(force))
    assert go.sum() - P.dt * work == pytest.approx(2 * rho_ * E, rel=1e-12)
    for a in range(3):
        q_a = (go * v[:, a]).sum() - P.dt * work * u[a]
        assert q_a == pytest.approx(2 * rho_ * uh[a] * H, rel=1e-10, abs=1e-14)
        for b in range(3):
            phi_ab = work * ((Pg / rho_) * (a == b) + u[a] * u[b])
            R_ab = (go * v[:, a] * v[:, b]).sum() - P.dt * phi_ab
            want = 2 * rho_ * uh[a] * uh[b] * (H + Pg / rho_) + 2 * Pg * H * (a == b)
            assert R_ab == pytest.approx(want, rel=1e-11, abs=1e-14), (a, b)
