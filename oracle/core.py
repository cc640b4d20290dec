"""ctypes wrapper around ``pond_oracle.c`` (test infrastructure only; see package doc)."""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pond_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NPLANES = 25
# plane layout of a D2Q9 state array of shape (25, ny, nx): f_0..f_8, g_0..g_8, theta, ux,
# uy, rho, T, uhat_x, uhat_y.  Population index i = 3*jy + jx with c = j - 1.
PL = dict(f=0, g=9, theta=18, ux=19, uy=20, rho=21, T=22, uhx=23, uhy=24)

LATTICES = {"d2q9": 0, "d2q16": 1}


def lattice_q(lattice: str = "d2q9") -> int:
    """Populations of a lattice: 9 (D2Q9) or 16 (D2Q16)."""
    return {"d2q9": 9, "d2q16": 16}[lattice]


def plane_layout(lattice: str = "d2q9") -> dict:
    """Plane indices of a state (2Q + 7 planes): f_0.., g_0.., theta, ux, uy, rho, T, uhat."""
    Q = lattice_q(lattice)
    return dict(f=0, g=Q, theta=2 * Q, ux=2 * Q + 1, uy=2 * Q + 2, rho=2 * Q + 3, T=2 * Q + 4,
                uhx=2 * Q + 5, uhy=2 * Q + 6, n=2 * Q + 7)


def lib_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, OpenMP, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + ".%d.tmp" % os.getpid()
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
                                   "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


class _CParams(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("bc_x", C.c_int32), ("bc_y", C.c_int32),
                ("a", C.c_double), ("b", C.c_double), ("R", C.c_double), ("delta", C.c_double),
                ("kappa", C.c_double), ("tau", C.c_double), ("k_cond", C.c_double),
                ("p_floor", C.c_double), ("tol", C.c_double), ("max_iter", C.c_int32),
                ("eos_kind", C.c_int32), ("dt", C.c_double), ("isothermal", C.c_int32),
                ("pad", C.c_int32), ("T_iso", C.c_double), ("sp_beta", C.c_double),
                ("sp_rho_l", C.c_double), ("sp_rho_v", C.c_double), ("sp_p0", C.c_double),
                ("lattice", C.c_int32), ("pad2", C.c_int32)]


@dataclasses.dataclass
class Params:
    nx: int
    ny: int
    bc_x: int = 0
    bc_y: int = 0
    a: float = 2.0 / 49.0
    b: float = 2.0 / 21.0
    R: float = 1.0
    delta: float = 1.0 / 3.0
    kappa: float = 0.0
    tau: float = 0.8
    k_cond: float = -1.0
    p_floor: float = 1e-3 / 6.0
    tol: float = 1e-12
    max_iter: int = 20
    dt: float = 1.0
    eos: str = "vdw"          # "vdw", or "dieterici" / "simplified" (isothermal only)
    isothermal: bool = False  # hold T at T_iso
    T_iso: float = 0.0
    eos_params: tuple = ()    # (beta, rho_l, rho_v, p0) of the "simplified" double well
    nonlocal_: str = "lagged"  # non-local terms from t - dt ("lagged") or from a first
                               # pass's prediction of t ("current", two passes per step)
    lattice: str = "d2q9"      # velocity set: "d2q9" (the paper's) or "d2q16"

    @property
    def Q(self) -> int:
        return lattice_q(self.lattice)

    @property
    def nplanes(self) -> int:
        return 2 * self.Q + 7

    def c(self) -> _CParams:
        if self.eos not in ("vdw", "dieterici", "simplified"):
            raise ValueError("eos must be vdw, dieterici or simplified")
        if self.eos != "vdw" and not self.isothermal:
            raise ValueError("the %s EoS is used isothermally (no caloric closure)" % self.eos)
        sp = tuple(self.eos_params) if self.eos == "simplified" else (0.0, 0.0, 0.0, 0.0)
        return _CParams(self.nx, self.ny, self.bc_x, self.bc_y, self.a, self.b, self.R,
                        self.delta, self.kappa, self.tau, self.k_cond, self.p_floor, self.tol,
                        self.max_iter, {"vdw": 0, "dieterici": 1, "simplified": 2}[self.eos], self.dt,
                        1 if self.isothermal else 0, 0, self.T_iso, *sp, LATTICES[self.lattice], 0)


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        pp = C.POINTER(_CParams)
        lib.orc_moment_matrix.argtypes = [dp, dp]
        lib.orc_gauge_matrix.argtypes = [dp, dp, dp]
        lib.orc_gauge_matrix.restype = C.c_int
        lib.orc_moment_matrix_q.argtypes = [C.c_int32, dp, dp]
        lib.orc_gauge_matrix_q.argtypes = [C.c_int32, dp, dp, dp]
        lib.orc_gauge_matrix_q.restype = C.c_int
        lib.orc_lagrange4.argtypes = [C.c_double, dp]
        lib.orc_nonlocal.argtypes = [pp, dp, dp, dp]
        lib.orc_init.argtypes = [pp, dp, dp, dp, dp, dp]
        lib.orc_stream_node.argtypes = [pp, dp, C.c_int, C.c_int, dp, dp, dp]
        lib.orc_stream_node.restype = C.c_int
        lib.orc_macro.argtypes = [pp, dp, dp, dp, C.c_double, C.c_double, C.c_double, dp]
        lib.orc_collide.argtypes = [pp, dp, dp, dp, dp, C.c_double, C.c_double, C.c_double,
                                    dp, dp]
        lib.orc_collide.restype = C.c_int
        lib.orc_step.argtypes = [pp, dp, dp, dp]
        lib.orc_step.restype = C.c_int
        lib.orc_step_nl.argtypes = [pp, dp, dp, dp, dp]
        lib.orc_step_nl.restype = C.c_int
        lib.orc_step_nodes.argtypes = [pp, dp, C.POINTER(C.c_int64), C.c_int64, dp, dp]
        lib.orc_step_nodes.restype = C.c_int
        lib.orc_moments.argtypes = [pp, dp, dp, dp, dp, dp, dp]
        lib.orc_num_threads.restype = C.c_int
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _d(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def lattice_1d(lattice: str = "d2q9") -> tuple[np.ndarray, np.ndarray, float]:
    """C1, its weights and T_L: D2Q9 {-1, 0, 1}; D2Q16 the four Gauss-Hermite nodes."""
    if lattice == "d2q16":
        ci, co = np.sqrt(3 - np.sqrt(6)), np.sqrt(3 + np.sqrt(6))
        wi, wo = (3 + np.sqrt(6)) / 12, (3 - np.sqrt(6)) / 12
        return np.array([-co, -ci, ci, co]), np.array([wo, wi, wi, wo]), 1.0
    return np.array([-1.0, 0.0, 1.0]), np.array([1 / 6, 2 / 3, 1 / 6]), 1.0 / 3.0


def weights(lattice: str = "d2q9") -> np.ndarray:
    """Weights W_i = W_jx W_jy (index i = q1*jy + jx)."""
    _, w1, _ = lattice_1d(lattice)
    q1 = len(w1)
    return np.array([w1[i % q1] * w1[i // q1] for i in range(q1 * q1)])


def velocities(lam, lattice: str = "d2q9") -> tuple[np.ndarray, np.ndarray]:
    """Shifted velocities v_i = sqrt(theta) c_i + u of gauge lam = (theta, ux, uy)."""
    th, ux, uy = lam
    c1, _, _ = lattice_1d(lattice)
    q1 = len(c1)
    c = np.array([(c1[i % q1], c1[i // q1]) for i in range(q1 * q1)], dtype=np.float64)
    s = np.sqrt(th)
    return s * c[:, 0] + ux, s * c[:, 1] + uy


def moment_matrix(lam, lattice: str = "d2q9") -> np.ndarray:
    Q = lattice_q(lattice)
    out = np.zeros(Q * Q)
    _load().orc_moment_matrix_q(LATTICES[lattice], _p(_d(lam)), _p(out))
    return out.reshape(Q, Q)


def gauge_matrix(src, dst, lattice: str = "d2q9") -> np.ndarray:
    Q = lattice_q(lattice)
    out = np.zeros(Q * Q)
    rc = _load().orc_gauge_matrix_q(LATTICES[lattice], _p(_d(src)), _p(_d(dst)), _p(out))
    if rc:
        raise ValueError("singular moment matrix")
    return out.reshape(Q, Q)


def lagrange4(xi: float) -> np.ndarray:
    out = np.zeros(4)
    _load().orc_lagrange4(float(xi), _p(out))
    return out


def nonlocal_fields(P: Params, rho, T) -> np.ndarray:
    """Lagged interface/heat-flux fields (4, ny, nx): Fx, Fy, rho E_lambda, M_0."""
    rho = _d(rho); T = _d(T)
    out = np.zeros((4, P.ny, P.nx))
    cp = P.c()
    _load().orc_nonlocal(C.byref(cp), _p(rho), _p(T), _p(out))
    return out


def init_state(P: Params, rho, ux, uy, T) -> np.ndarray:
    out = np.zeros((P.nplanes, P.ny, P.nx))
    cp = P.c()
    _load().orc_init(C.byref(cp), _p(_d(rho)), _p(_d(ux)), _p(_d(uy)), _p(_d(T)), _p(out))
    return out


def stream_node(P: Params, state, X: int, Y: int, lam):
    state = _d(state)
    ft = np.zeros(P.Q); gt = np.zeros(P.Q)
    cp = P.c()
    rc = _load().orc_stream_node(C.byref(cp), _p(state), int(X), int(Y), _p(_d(lam)),
                                 _p(ft), _p(gt))
    if rc:
        raise ValueError("singular moment matrix")
    return ft, gt


def macro(P: Params, lam, ft, gt, Fx=0.0, Fy=0.0, rEl=0.0) -> dict:
    out = np.zeros(11)
    cp = P.c()
    _load().orc_macro(C.byref(cp), _p(_d(lam)), _p(_d(ft)), _p(_d(gt)), float(Fx), float(Fy),
                      float(rEl), _p(out))
    keys = ["rho", "ux", "uy", "uhx", "uhy", "E", "e", "T", "p", "P", "theta"]
    return dict(zip(keys, out.tolist())) | {"_raw": out}


def collide(P: Params, lam, ft, gt, mac, Fx=0.0, Fy=0.0, M0=0.0):
    fo = np.zeros(P.Q); go = np.zeros(P.Q)
    raw = mac["_raw"] if isinstance(mac, dict) else _d(mac)
    cp = P.c()
    rc = _load().orc_collide(C.byref(cp), _p(_d(lam)), _p(_d(ft)), _p(_d(gt)), _p(_d(raw)),
                             float(Fx), float(Fy), float(M0), _p(fo), _p(go))
    if rc:
        raise ValueError("singular moment matrix")
    return fo, go


def step(P: Params, state, n: int = 1, stats=None) -> np.ndarray:
    """Advance the full grid by n time steps; returns the new state (2Q + 7, ny, nx)."""
    cur = _d(state).copy()
    nxt = np.empty_like(cur)
    st = np.zeros(4)
    cp = P.c()
    lib = _load()
    if P.nonlocal_ not in ("lagged", "current"):
        raise ValueError("nonlocal_ must be lagged or current")
    pred = np.empty_like(cur) if P.nonlocal_ == "current" else None
    for _ in range(n):
        if pred is None:
            rc = lib.orc_step(C.byref(cp), _p(cur), _p(nxt), _p(st))
        else:
            # pass 1: the lagged step predicts rho, T at t; pass 2 redoes the step from the
            # same state with the non-local terms of that prediction
            rc = lib.orc_step(C.byref(cp), _p(cur), _p(pred), None)
            rc = rc or lib.orc_step_nl(C.byref(cp), _p(cur), _p(pred), _p(nxt), _p(st))
        if rc:
            raise FloatingPointError("oracle step failed (singular moment matrix)")
        cur, nxt = nxt, cur
    if stats is not None:
        stats["streams"] = stats.get("streams", 0.0) + st[0]
        stats["nonconv"] = stats.get("nonconv", 0.0) + st[1]
        stats["clamped"] = stats.get("clamped", 0.0) + st[2]
    return cur


def step_nodes(P: Params, state, nodes, stats=None) -> np.ndarray:
    """One step evaluated at the given flat node indices only; returns (len, 2Q + 7)."""
    state = _d(state)
    nodes = np.ascontiguousarray(np.asarray(nodes, dtype=np.int64))
    out = np.zeros((len(nodes), P.nplanes))
    st = np.zeros(4)
    cp = P.c()
    rc = _load().orc_step_nodes(C.byref(cp), _p(state), nodes.ctypes.data_as(C.POINTER(C.c_int64)),
                                len(nodes), _p(out), _p(st))
    if rc:
        raise FloatingPointError("oracle step failed (singular moment matrix)")
    if stats is not None:
        stats["streams"] = stats.get("streams", 0.0) + st[0]
        stats["nonconv"] = stats.get("nonconv", 0.0) + st[1]
        stats["clamped"] = stats.get("clamped", 0.0) + st[2]
    return out


def moments(P: Params, state) -> dict:
    state = _d(state)
    outs = [np.zeros((P.ny, P.nx)) for _ in range(5)]
    cp = P.c()
    _load().orc_moments(C.byref(cp), _p(state), *[_p(o) for o in outs])
    return dict(zip(["rho", "ux", "uy", "T", "p"], outs))


def num_threads() -> int:
    return int(_load().orc_num_threads())
