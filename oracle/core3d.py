"""ctypes wrapper around ``pond_oracle3d.c``, the 3-D (D3Q27) oracle (test
infrastructure only; see package doc)."""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pond_oracle3d.c")
_LIB = os.path.join(_HERE, "liboracle3d.so")
_lock = threading.Lock()
_lib = None

Q = 27
NPLANES = 2 * Q + 9
# planes of a state (63, nz, ny, nx): f_0..f_26, g_0..g_26, theta, ux, uy, uz, rho, T,
# uhat_x, uhat_y, uhat_z; population i = 9*jz + 3*jy + jx with c = j - 1
PL = dict(f=0, g=27, theta=54, ux=55, uy=56, uz=57, rho=58, T=59, uhx=60, uhy=61, uhz=62)


def build(force: bool = False) -> str:
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + ".%d.tmp" % os.getpid()
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
                                   "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


class _CParams(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("bc_x", C.c_int32), ("bc_y", C.c_int32), ("bc_z", C.c_int32),
                ("a", C.c_double), ("b", C.c_double), ("R", C.c_double), ("delta", C.c_double),
                ("kappa", C.c_double), ("tau", C.c_double), ("k_cond", C.c_double),
                ("p_floor", C.c_double), ("tol", C.c_double), ("max_iter", C.c_int32),
                ("pad", C.c_int32), ("dt", C.c_double)]


@dataclasses.dataclass
class Params3:
    nx: int
    ny: int
    nz: int
    bc_x: int = 0
    bc_y: int = 0
    bc_z: int = 0
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

    def c(self) -> _CParams:
        return _CParams(self.nx, self.ny, self.nz, self.bc_x, self.bc_y, self.bc_z, self.a, self.b,
                        self.R, self.delta, self.kappa, self.tau, self.k_cond, self.p_floor,
                        self.tol, self.max_iter, 0, self.dt)


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        pp = C.POINTER(_CParams)
        lib.orc3_moment_matrix.argtypes = [dp, dp]
        lib.orc3_gauge_matrix.argtypes = [dp, dp, dp]
        lib.orc3_gauge_matrix.restype = C.c_int
        lib.orc3_nonlocal.argtypes = [pp, dp, dp, dp]
        lib.orc3_init.argtypes = [pp, dp, dp, dp, dp, dp, dp]
        lib.orc3_step.argtypes = [pp, dp, dp, dp]
        lib.orc3_step.restype = C.c_int
        lib.orc3_step_nodes.argtypes = [pp, dp, C.POINTER(C.c_int64), C.c_int64, dp]
        lib.orc3_step_nodes.restype = C.c_int
        lib.orc3_macro.argtypes = [pp, dp, dp, dp, dp, C.c_double, dp]
        lib.orc3_collide.argtypes = [pp, dp, dp, dp, dp, dp, C.c_double, dp, dp]
        lib.orc3_collide.restype = C.c_int
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _d(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def weights() -> np.ndarray:
    w1 = np.array([1 / 6, 2 / 3, 1 / 6])
    return np.array([w1[i % 3] * w1[(i // 3) % 3] * w1[i // 9] for i in range(Q)])


def moment_matrix(lam) -> np.ndarray:
    out = np.zeros(Q * Q)
    _load().orc3_moment_matrix(_p(_d(lam)), _p(out))
    return out.reshape(Q, Q)


def gauge_matrix(src, dst) -> np.ndarray:
    out = np.zeros(Q * Q)
    if _load().orc3_gauge_matrix(_p(_d(src)), _p(_d(dst)), _p(out)):
        raise ValueError("singular moment matrix")
    return out.reshape(Q, Q)


def nonlocal_fields(P: Params3, rho, T) -> np.ndarray:
    """(5, nz, ny, nx): F_x, F_y, F_z, rho E_lambda, M_0."""
    out = np.zeros((5, P.nz, P.ny, P.nx))
    cp = P.c()
    _load().orc3_nonlocal(C.byref(cp), _p(_d(rho)), _p(_d(T)), _p(out))
    return out


def init_state(P: Params3, rho, ux, uy, uz, T) -> np.ndarray:
    out = np.zeros((NPLANES, P.nz, P.ny, P.nx))
    cp = P.c()
    _load().orc3_init(C.byref(cp), *[_p(_d(a)) for a in (rho, ux, uy, uz, T)], _p(out))
    return out


def step(P: Params3, state, n: int = 1, stats=None) -> np.ndarray:
    cur = _d(state).copy()
    nxt = np.empty_like(cur)
    st = np.zeros(4)
    cp = P.c()
    for _ in range(n):
        if _load().orc3_step(C.byref(cp), _p(cur), _p(nxt), _p(st)):
            raise FloatingPointError("oracle step failed (singular moment matrix)")
        cur, nxt = nxt, cur
    if stats is not None:
        stats["streams"] = stats.get("streams", 0.0) + st[0]
        stats["nonconv"] = stats.get("nonconv", 0.0) + st[1]
    return cur


def step_nodes(P: Params3, state, nodes) -> np.ndarray:
    """One step at the given flat node indices ((z*ny + y)*nx + x); returns (len, 63)."""
    state = _d(state)
    nodes = np.ascontiguousarray(np.asarray(nodes, dtype=np.int64))
    out = np.zeros((len(nodes), NPLANES))
    cp = P.c()
    if _load().orc3_step_nodes(C.byref(cp), _p(state), nodes.ctypes.data_as(C.POINTER(C.c_int64)),
                               len(nodes), _p(out)):
        raise FloatingPointError("oracle step failed (singular moment matrix)")
    return out


def macro(P: Params3, lam, ft, gt, F=(0.0, 0.0, 0.0), rEl=0.0) -> dict:
    """Macroscopic fields of streamed populations in gauge lam = (theta, ux, uy, uz)."""
    out = np.zeros(13)
    cp = P.c()
    _load().orc3_macro(C.byref(cp), _p(_d(lam)), _p(_d(ft)), _p(_d(gt)), _p(_d(F)), float(rEl), _p(out))
    keys = ["rho", "ux", "uy", "uz", "uhx", "uhy", "uhz", "E", "e", "T", "p", "P", "theta"]
    return dict(zip(keys, out.tolist())) | {"_raw": out}


def collide(P: Params3, lam, ft, gt, mac, F=(0.0, 0.0, 0.0), M0=0.0):
    """Post-collision f, g (27 each) in the streaming gauge lam."""
    fo = np.zeros(Q)
    go = np.zeros(Q)
    raw = mac["_raw"] if isinstance(mac, dict) else _d(mac)
    cp = P.c()
    if _load().orc3_collide(C.byref(cp), _p(_d(lam)), _p(_d(ft)), _p(_d(gt)), _p(_d(raw)), _p(_d(F)),
                            float(M0), _p(fo), _p(go)):
        raise ValueError("singular moment matrix")
    return fo, go


def moments(P: Params3, state) -> dict:
    s = _d(state)
    rho, T = s[PL["rho"]], s[PL["T"]]
    p = rho * P.R * T / (1.0 - P.b * rho) - P.a * rho * rho
    return {"rho": rho.copy(), "ux": s[PL["uhx"]].copy(), "uy": s[PL["uhy"]].copy(),
            "uz": s[PL["uhz"]].copy(), "T": T.copy(), "p": p}
