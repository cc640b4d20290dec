"""Exact Riemann solver of the 1-D Euler equations for the van der Waals fluid with a
constant heat capacity C_v = R / delta (the fluid of the main text's Fig. 4 and the SM's
shock-tube table), including non-classical waves where the fundamental derivative Gamma
changes sign.  Test infrastructure: the reference for the shock tubes of the GPU path
and of the oracle.

Thermodynamics in specific volume v = 1/rho:
  p(v, T) = R T/(v - b) - a/v^2,   e(v, p) = (p + a/v^2)(v - b)/delta - a/v,
  isentropes T (v - b)^delta = const, so p_s(v) and its derivatives are explicit;
  the Lagrangian sound speed is C = sqrt(-dp_s/dv) (c = v C) and
  Gamma = -v p_s''/(2 p_s');
  the Hugoniot through a state K, e(v, p) - e_K + (p + p_K)(v - v_K)/2 = 0, is linear in
  p at fixed v, so p_H(v) is explicit.

Waves of family 1 (left, sign s = -1) and 3 (right, s = +1) from a state K:
  fan (isentrope):  u = u_K - s int_{v_K}^{v} C dv';
  shock (Hugoniot): u = u_K - s sign(v - v_K) sqrt(-(p - p_K)(v - v_K)), mass flux
                    m = sqrt(-(p - p_K)/(v - v_K)), speed u_K + s m v_K.
Admissibility (Liu): a shock from the state ahead K to S is admitted when
m^2(K, M) <= m^2(K, S) for every M on the Hugoniot between them (no intermediate shock is
faster; at M -> K this is the Lax bound C_K <= m); a fan when the characteristic speed
increases across it (expansion needs Gamma > 0 along it, compression Gamma < 0).  Where
neither holds over the whole path the wave is composite and is built by marching pieces
from K: a fan ended by a shock that is sonic at the fan's end (m = C there), which either
reaches the target with a subsonic state behind it or is sonic behind as well and is
followed by another fan; or a shock that is sonic behind (its Rayleigh line tangent to the
isentrope of its end state) followed by a fan.  Waves that would need more than eight
pieces are refused.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import quad
from scipy.optimize import brentq

A_VDW, B_VDW, R_GAS = 2.0 / 49.0, 2.0 / 21.0, 1.0


class Gas:
    def __init__(self, delta, a=A_VDW, b=B_VDW, R=R_GAS):
        self.d, self.a, self.b, self.R = float(delta), a, b, R

    # -- state functions ---------------------------------------------------------------
    def p(self, v, T):
        return self.R * T / (v - self.b) - self.a / v ** 2

    def T(self, v, p):
        return (p + self.a / v ** 2) * (v - self.b) / self.R

    def e(self, v, p):
        return (p + self.a / v ** 2) * (v - self.b) / self.d - self.a / v

    # -- isentrope through (vK, pK) ----------------------------------------------------
    def _k(self, vK, pK):
        return self.R * self.T(vK, pK) * (vK - self.b) ** self.d

    def p_s(self, v, vK, pK):
        return self._k(vK, pK) * (v - self.b) ** (-self.d - 1.0) - self.a / v ** 2

    def dp_s(self, v, vK, pK):
        return -(self.d + 1.0) * self._k(vK, pK) * (v - self.b) ** (-self.d - 2.0) + 2.0 * self.a / v ** 3

    def d2p_s(self, v, vK, pK):
        return ((self.d + 1.0) * (self.d + 2.0) * self._k(vK, pK) * (v - self.b) ** (-self.d - 3.0)
                - 6.0 * self.a / v ** 4)

    def C(self, v, vK, pK):
        """Lagrangian sound speed rho c on the isentrope through K."""
        return math.sqrt(-self.dp_s(v, vK, pK))

    def gamma(self, v, p):
        """Fundamental derivative at (v, p) (its isentrope passes through the state)."""
        return -v * self.d2p_s(v, v, p) / (2.0 * self.dp_s(v, v, p))

    def c(self, v, p):
        return v * self.C(v, v, p)

    # -- Hugoniot through (vK, pK) -----------------------------------------------------
    def p_H(self, v, vK, pK):
        eK = self.e(vK, pK)
        num = eK - (self.a / self.d) * (v - self.b) / v ** 2 + self.a / v - 0.5 * pK * (v - vK)
        return num / ((v - self.b) / self.d + 0.5 * (v - vK))


def _v_on(curve, p_target, v0, v_far, tol=1e-14):
    """v between v0 and v_far where curve(v) = p_target (bracketed root)."""
    f = lambda v: curve(v) - p_target
    return brentq(f, min(v0, v_far), max(v0, v_far), xtol=tol, rtol=1e-15, maxiter=500)


class Family:
    """Wave curve of family 1 (s = -1, from the left state) or 3 (s = +1, from the right)."""

    def __init__(self, gas: Gas, s: int, v, p, u):
        self.g, self.s, self.vK, self.pK, self.uK = gas, s, float(v), float(p), float(u)

    # -- pieces ---------------------------------------------------------------------
    def fan_u(self, vB, pB, uB, v):
        g = self.g
        if v == vB:
            return uB
        return uB - self.s * quad(lambda x: g.C(x, vB, pB), vB, v, epsabs=0.0, epsrel=1e-13, limit=200)[0]

    def shock_u(self, vA, pA, uA, vB, pB):
        return uA - self.s * math.copysign(math.sqrt(max(0.0, -(pB - pA) * (vB - vA))), vB - vA)

    @staticmethod
    def m2(vA, pA, vB, pB):
        return -(pB - pA) / (vB - vA)

    def fan_ok(self, vB, pB, v_end, n=200):
        """Characteristic speed increases across a fan from vB to v_end: expansion needs
        Gamma >= 0 along it, compression Gamma <= 0."""
        sgn = 1.0 if v_end > vB else -1.0
        for v in np.linspace(vB, v_end, n)[1:]:
            if sgn * self.g.gamma(v, self.g.p_s(v, vB, pB)) < -1e-12:
                return False
        return True

    def liu_ok(self, vA, pA, vS, n=400):
        g = self.g
        pS = g.p_H(vS, vA, pA)
        mS = self.m2(vA, pA, vS, pS)
        for v in np.linspace(vA, vS, n)[1:-1]:
            if self.m2(vA, pA, v, g.p_H(v, vA, pA)) > mS * (1.0 + 1e-9):
                return False
        return True

    # -- the wave to pressure p* --------------------------------------------------------
    def to(self, ps):
        """(u*, v*, pieces) of the wave from K to pressure ps.  Pieces run from K outward:
        ("fan", base (v, p, u), v_a, v_b) or ("shock", (v, p, u) ahead, (v, p, u) behind, m).
        Built by marching from K: in fan mode (Gamma has the sign that makes this direction
        a fan) along the isentrope; where an inflection lies before ps the fan ends at M and
        a shock sonic at M follows, either to ps (if the state behind it is subsonic) or to
        the point where it is sonic behind as well, after which the march goes on with a
        fan; in shock mode along the Hugoniot, to ps if Liu's condition holds, else to the
        point where the state behind becomes sonic, after which a fan follows."""
        g = self.g
        v, p, u = self.vK, self.pK, self.uK
        if abs(ps - p) <= 1e-15 * abs(p):
            return u, v, []
        expand = ps < p
        pieces = []
        for _ in range(8):
            fan_mode = (g.gamma(v, p) > 0) == expand
            if fan_mode:
                vend = _v_on(lambda x: g.p_s(x, v, p), ps, v, self._limit_s(expand, v))
                v_inf = self._inflection(v, p, vend)
                if v_inf is None:
                    pieces.append(("fan", (v, p, u), v, vend))
                    return self.fan_u(v, p, u, vend), vend, pieces
                done, nxt = self._fan_then_shock(v, p, u, ps, v_inf, expand, pieces)
                if done:
                    return nxt[2], nxt[0], pieces
                v, p, u = nxt
            else:
                vend = _v_on(lambda x: g.p_H(x, v, p), ps, v, self._limit_h(expand, v))
                if self.liu_ok(v, p, vend) and self._subsonic_behind(v, p, vend, ps):
                    ue = self.shock_u(v, p, u, vend, ps)
                    pieces.append(("shock", (v, p, u), (vend, ps, ue), math.sqrt(self.m2(v, p, vend, ps))))
                    return ue, vend, pieces
                vM = self._post_sonic_point(v, p, vend)
                pM = g.p_H(vM, v, p)
                uM = self.shock_u(v, p, u, vM, pM)
                pieces.append(("shock", (v, p, u), (vM, pM, uM), math.sqrt(self.m2(v, p, vM, pM))))
                v, p, u = vM, pM, uM
        raise NotImplementedError("wave with more than eight pieces")

    def _limit_s(self, expand, vB=None):
        """Far end of a search along the isentrope from vB (default K): large v for
        expansions, just above b for compressions."""
        vB = self.vK if vB is None else vB
        return vB * 50.0 if expand else self.g.b + 1e-6 * (vB - self.g.b)

    def _limit_h(self, expand, vB=None):
        """Far end of a search along the Hugoniot through vB: large v for expansions, just
        above its asymptote v = (2b/delta + v_B)/(2/delta + 1) for compressions."""
        g = self.g
        vB = self.vK if vB is None else vB
        if expand:
            return vB * 50.0
        vmin = (2.0 * g.b / g.d + vB) / (2.0 / g.d + 1.0)
        return vmin + 1e-9 * (vB - vmin)

    def _inflection(self, vB, pB, vend, n=400):
        """First v between vB and vend where Gamma on the isentrope of B changes sign."""
        g = self.g
        grid = np.linspace(vB, vend, n)
        gam = [g.gamma(x, g.p_s(x, vB, pB)) for x in grid]
        for i in range(1, n):
            if (gam[i] > 0) != (gam[0] > 0):
                return brentq(lambda x: g.gamma(x, g.p_s(x, vB, pB)), grid[i - 1], grid[i], xtol=1e-15)
        return None

    def _subsonic_behind(self, va, pa, vb, pb):
        """Lax bound behind a shock: m <= C at the state behind it."""
        return self.m2(va, pa, vb, pb) <= self.g.C(vb, vb, pb) ** 2 * (1.0 + 1e-9)

    def _post_sonic_point(self, vA, pA, vend, n=800):
        """First point M on the Hugoniot of A toward vend where m(A, M) = C(M) (the Rayleigh
        line tangent to M's isentrope)."""
        g = self.g

        def gap(x):
            px = g.p_H(x, vA, pA)
            return self.m2(vA, pA, x, px) - g.C(x, x, px) ** 2

        grid = np.linspace(vA, vend, n)[1:]
        vals = [gap(x) for x in grid]
        for i in range(1, len(grid)):
            if (vals[i] > 0) != (vals[0] > 0):
                return brentq(gap, grid[i - 1], grid[i], xtol=1e-15, rtol=1e-15, maxiter=500)
        raise NotImplementedError("no sonic point on the Hugoniot before the target")

    def _sonic_shock_end(self, vM, pM, CM2, expand, n=600):
        """The state S (other than M) on the Hugoniot of M where the Rayleigh line of slope
        -CM2 (a shock sonic at M) meets it again, or None."""
        g = self.g
        far = self._limit_h(expand, vM)
        grid = np.linspace(vM, far, n)[1:]
        f = lambda x: self.m2(vM, pM, x, g.p_H(x, vM, pM)) - CM2
        vals = [f(x) for x in grid]
        for i in range(1, len(grid)):
            if (vals[i] > 0) != (vals[0] > 0):
                return brentq(f, grid[i - 1], grid[i], xtol=1e-15, rtol=1e-15, maxiter=500)
        return None

    def _fan_then_shock(self, vB, pB, uB, ps, v_inf, expand, pieces):
        """Fan from B to M (before the inflection), then a shock sonic at M.  Appends the
        pieces; returns (True, (v, p, u) at ps) if the shock reaches ps with a subsonic state
        behind, else (False, state after a shock that is sonic on both sides)."""
        g = self.g

        def end_at_ps(vM):
            pM = g.p_s(vM, vB, pB)
            vS = _v_on(lambda x: g.p_H(x, vM, pM), ps, vM, self._limit_h(expand, vM))
            return self.m2(vM, pM, vS, ps) - g.C(vM, vB, pB) ** 2, vS

        lo, hi = vB + (v_inf - vB) * 1e-9, v_inf - (v_inf - vB) * 1e-9
        try:
            flo, fhi = end_at_ps(lo)[0], end_at_ps(hi)[0]
        except ValueError:
            flo = fhi = 1.0
        if (flo > 0) != (fhi > 0):
            vM = brentq(lambda x: end_at_ps(x)[0], lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
            pM = g.p_s(vM, vB, pB)
            _, vS = end_at_ps(vM)
            if self._subsonic_behind(vM, pM, vS, ps) and self.liu_ok(vM, pM, vS):
                uM = self.fan_u(vB, pB, uB, vM)
                uS = self.shock_u(vM, pM, uM, vS, ps)
                pieces.append(("fan", (vB, pB, uB), vB, vM))
                pieces.append(("shock", (vM, pM, uM), (vS, ps, uS), math.sqrt(self.m2(vM, pM, vS, ps))))
                return True, (vS, ps, uS)

        # the shock stops where it is sonic behind too: C(S) = C(M) = m
        def double(vM):
            pM = g.p_s(vM, vB, pB)
            CM2 = g.C(vM, vB, pB) ** 2
            vS = self._sonic_shock_end(vM, pM, CM2, expand)
            if vS is None:
                return None
            pS = g.p_H(vS, vM, pM)
            return g.C(vS, vS, pS) ** 2 - CM2, vS, pS

        grid = np.linspace(lo, hi, 200)
        vals = [double(x) for x in grid]
        idx = [i for i in range(1, len(grid)) if vals[i] is not None and vals[i - 1] is not None
               and (vals[i][0] > 0) != (vals[i - 1][0] > 0)]
        if not idx:
            raise NotImplementedError("no double-sonic shock on this isentrope")
        i = idx[0]
        vM = brentq(lambda x: double(x)[0], grid[i - 1], grid[i], xtol=1e-15, rtol=1e-15, maxiter=500)
        pM = g.p_s(vM, vB, pB)
        _, vS, pS = double(vM)
        uM = self.fan_u(vB, pB, uB, vM)
        uS = self.shock_u(vM, pM, uM, vS, pS)
        pieces.append(("fan", (vB, pB, uB), vB, vM))
        pieces.append(("shock", (vM, pM, uM), (vS, pS, uS), math.sqrt(self.m2(vM, pM, vS, pS))))
        return False, (vS, pS, uS)


class Riemann:
    """Exact solution of the Riemann problem between left and right states (rho, u, p)."""

    def __init__(self, delta, left, right, p_bracket=None):
        self.g = g = Gas(delta)
        (rL, uL, pL), (rR, uR, pR) = left, right
        self.L = (1.0 / rL, pL, uL)
        self.R = (1.0 / rR, pR, uR)
        self.f1 = Family(g, -1, 1.0 / rL, pL, uL)
        self.f3 = Family(g, +1, 1.0 / rR, pR, uR)
        # with equal side velocities the star pressure lies between the side pressures
        # (one wave expands, the other compresses)
        if p_bracket is None:
            p_bracket = ((min(pL, pR), max(pL, pR)) if uL == uR else
                         (0.5 * min(pL, pR), 2.0 * max(pL, pR)))
        lo, hi = p_bracket
        gap = lambda p: self.f1.to(p)[0] - self.f3.to(p)[0]
        self.ps = brentq(gap, lo, hi, xtol=1e-14, rtol=1e-15, maxiter=300)
        self.us, self.vL, self.w1 = self.f1.to(self.ps)
        u3, self.vR, self.w3 = self.f3.to(self.ps)
        self.mismatch = abs(u3 - self.us)
        self._segments()

    def describe(self):
        return {"p_star": self.ps, "u_star": self.us, "rho_star_left": 1.0 / self.vL,
                "rho_star_right": 1.0 / self.vR,
                "wave1": [w[0] for w in self.w1], "wave3": [w[0] for w in self.w3]}

    def _segments(self):
        """Pieces of the solution in x/t order: ("const", (v, p, u), xi_end) and
        ("fan", family, base, v_a, v_b, xi_a, xi_b)."""
        g = self.g
        seg = []

        def lam(fam, base, v):
            vB, pB, uB = base
            u = fam.fan_u(vB, pB, uB, v)
            return u + fam.s * v * g.C(v, vB, pB)

        # family 1: from the left state toward the star state
        state = self.L
        for w in self.w1:
            if w[0] == "shock":
                (va, pa, ua), (vb, pb, ub), m = w[1], w[2], w[3]
                seg.append(("const", state, ua - m * va))
                state = (vb, pb, ub)
            else:
                base, va, vb = w[1], w[2], w[3]
                xa, xb = lam(self.f1, base, va), lam(self.f1, base, vb)
                seg.append(("const", state, xa))
                seg.append(("fan", self.f1, base, va, vb, xa, xb))
                state = (vb, g.p_s(vb, base[0], base[1]), self.f1.fan_u(*base, vb))
        seg.append(("const", (self.vL, self.ps, self.us), self.us))
        # family 3: listed from the right state inward, reversed into x/t order
        right = []
        state = self.R
        for w in self.w3:
            if w[0] == "shock":
                (va, pa, ua), (vb, pb, ub), m = w[1], w[2], w[3]
                right.append(("edge", state, ua + m * va))
                state = (vb, pb, ub)
            else:
                base, va, vb = w[1], w[2], w[3]
                xa, xb = lam(self.f3, base, va), lam(self.f3, base, vb)
                right.append(("edge", state, xa))
                right.append(("fan", self.f3, base, vb, va, xb, xa))
                state = (vb, g.p_s(vb, base[0], base[1]), self.f3.fan_u(*base, vb))
        # star-right state up to the innermost 3-wave, then outward
        inner = right[::-1]
        first = inner[0]
        seg.append(("const", (self.vR, self.ps, self.us), first[2] if first[0] == "edge" else first[5]))
        for k, piece in enumerate(inner):
            if piece[0] == "fan":
                seg.append(piece)
            else:
                nxt = inner[k + 1] if k + 1 < len(inner) else None
                end = math.inf if nxt is None else (nxt[2] if nxt[0] == "edge" else nxt[5])
                seg.append(("const", piece[1], end))
        if not inner:
            seg[-1] = ("const", (self.vR, self.ps, self.us), math.inf)
        self.seg = seg

    def state_at(self, xi):
        """(rho, u, p) at x/t = xi."""
        g = self.g
        start = -math.inf
        for piece in self.seg:
            if piece[0] == "const":
                if xi < piece[2] or piece[2] == math.inf:
                    v, p, u = piece[1]
                    return 1.0 / v, u, p
                start = piece[2]
            else:
                fam, base, va, vb, xa, xb = piece[1:]
                if xi < xb:
                    def f(v):
                        u = fam.fan_u(*base, v)
                        return u + fam.s * v * g.C(v, base[0], base[1]) - xi
                    v = brentq(f, min(va, vb), max(va, vb), xtol=1e-15, maxiter=300)
                    return 1.0 / v, fam.fan_u(*base, v), g.p_s(v, base[0], base[1])
                start = xb
        v, p, u = self.R
        return 1.0 / v, u, p

    def profile(self, x, t, x0):
        out = np.array([self.state_at((xx - x0) / t) for xx in np.asarray(x, dtype=float)])
        return out[:, 0], out[:, 1], out[:, 2]


# ---------------------------------------------------------------------------------------
# An independent reference for the exact solver: a first-order finite-volume (Rusanov)
# solution of the same Euler equations in conservative variables (rho, rho u, rho E),
# E = e + u^2/2.  Its numerical viscosity selects the vanishing-viscosity (entropy)
# solution, so a wrongly chosen wave structure in the exact solver shows as an O(1) gap.
def _primitive(gas, U):
    rho = U[0]
    u = U[1] / rho
    e = U[2] / rho - 0.5 * u * u
    v = 1.0 / rho
    # e = (p + a/v^2)(v - b)/delta - a/v  =>  p
    p = (e + gas.a / v) * gas.d / (v - gas.b) - gas.a / v ** 2
    return rho, u, p, v


def rusanov_tube(delta, left, right, ncell, t_end, x_len=1.0, cfl=0.4):
    """Cell averages (x, rho, u, p) at t_end of the Riemann problem on [0, x_len] with the
    diaphragm at the middle (zero-gradient ends)."""
    gas = Gas(delta)
    x = (np.arange(ncell) + 0.5) * x_len / ncell
    dx = x_len / ncell
    rho = np.where(x < 0.5 * x_len, left[0], right[0])
    u = np.where(x < 0.5 * x_len, left[1], right[1])
    p = np.where(x < 0.5 * x_len, left[2], right[2])
    v = 1.0 / rho
    e = gas.e(v, p)
    U = np.array([rho, rho * u, rho * (e + 0.5 * u * u)])
    t = 0.0
    while t < t_end:
        rho, u, p, v = _primitive(gas, U)
        c = v * np.sqrt(np.maximum(-gas.dp_s(v, v, p), 0.0))
        smax = np.max(np.abs(u) + c)
        dt = min(cfl * dx / smax, t_end - t)
        F = np.array([rho * u, rho * u * u + p, u * (U[2] + p)])
        Ug = np.concatenate([U[:, :1], U, U[:, -1:]], axis=1)
        Fg = np.concatenate([F[:, :1], F, F[:, -1:]], axis=1)
        sg = np.concatenate([[abs(u[0]) + c[0]], np.abs(u) + c, [abs(u[-1]) + c[-1]]])
        a = np.maximum(sg[:-1], sg[1:])
        flux = 0.5 * (Fg[:, :-1] + Fg[:, 1:]) - 0.5 * a * (Ug[:, 1:] - Ug[:, :-1])
        U = U - dt / dx * (flux[:, 1:] - flux[:, :-1])
        t += dt
    rho, u, p, _ = _primitive(gas, U)
    return x, rho, u, p
