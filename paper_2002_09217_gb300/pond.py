"""Thin ctypes binding of libpond (``include/pond.h``): argument marshalling only.

Every step of the time step runs in the CUDA kernels of ``libpond.so``; there is
no CPU fallback.  If the library cannot be loaded, or no GPU is usable, the calls
raise.  PyTorch is used for device memory (the caching allocator backs the
library's device buffers) and streams.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build_lib

POND_PERIODIC, POND_ZEROGRAD = 0, 1
POND_D2Q9, POND_D2Q16, POND_D3Q27 = 0, 1, 2
LATTICES = {"d2q9": POND_D2Q9, "d2q16": POND_D2Q16, "d3q27": POND_D3Q27}
POND_VDW, POND_IDEAL, POND_DIETERICI, POND_SIMPLIFIED = 0, 1, 2, 3
POND_FP64, POND_MIXED = 0, 1
NPLANES = 25
STATUS = {0: "POND_OK", 1: "POND_EINVAL", 2: "POND_ENOMEM", 3: "POND_ECUDA", 4: "POND_ENONCONV",
          5: "POND_ETHETA", 6: "POND_ENAN", 7: "POND_ETIMEOUT"}
POND_ENONCONV, POND_ETHETA = 4, 5
# warning-class statuses of the synchronising calls: the call completed and wrote its
# outputs; the status reports a sticky device flag (see include/pond.h)
WARNINGS = (POND_ENONCONV, POND_ETHETA)

_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("bc_x", C.c_int32), ("bc_y", C.c_int32),
                ("nz", C.c_int32), ("bc_z", C.c_int32)]


class Lattice(C.Structure):
    _fields_ = [("kind", C.c_int32)]


class Eos(C.Structure):
    _fields_ = [("kind", C.c_int32), ("a", C.c_double), ("b", C.c_double), ("R", C.c_double),
                ("delta", C.c_double), ("isothermal", C.c_int32), ("T_iso", C.c_double),
                ("beta", C.c_double), ("rho_l", C.c_double), ("rho_v", C.c_double), ("p0", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_iter", C.c_int32), ("tol", C.c_double),
                ("dt", C.c_double), ("k_cond", C.c_double), ("p_floor", C.c_double),
                ("stream", C.c_void_p), ("dalloc", _ALLOC), ("dfree", _FREE),
                ("alloc_ctx", C.c_void_p), ("lanes_per_node", C.c_int32), ("tile_x", C.c_int32),
                ("nonlocal_", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("node_updates", C.c_int64), ("streams", C.c_int64),
                ("nonconverged", C.c_int64), ("clamped", C.c_int64), ("nonfinite", C.c_int64),
                ("stalled", C.c_int64), ("block_streams", C.c_int64), ("max_streams", C.c_int64),
                ("timeouts", C.c_int64), ("region_nodes", C.c_int64), ("pair_streams", C.c_int64)]


class PondError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return build_lib.LIB


def load() -> C.CDLL:
    """Load libpond.so (building it with nvcc first if it is missing or older than any
    of its sources)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not build_lib.up_to_date():
            build_lib.build()
        lib = C.CDLL(build_lib.LIB)
        P = C.c_void_p
        dp = C.POINTER(C.c_double)
        lib.pond_create.argtypes = [C.POINTER(Grid), C.POINTER(Lattice), C.POINTER(Eos), C.c_double,
                                    C.c_double, C.POINTER(Opts), C.POINTER(P)]
        for name, args in [("pond_init_fields", [P, dp, dp, dp, dp]),
                           ("pond_init_fields3", [P, dp, dp, dp, dp, dp]),
                           ("pond_moments3", [P, dp, dp, dp, dp, dp, dp]),
                           ("pond_init_fields_device", [P, P, P, P, P]),
                           ("pond_step", [P, C.c_int64]),
                           ("pond_moments", [P, dp, dp, dp, dp, dp]),
                           ("pond_moments_device", [P, P, P, P, P, P]),
                           ("pond_conservation", [P, dp]),
                           ("pond_get_state", [P, dp]),
                           ("pond_set_state", [P, dp]),
                           ("pond_stats", [P, C.POINTER(Stats), C.c_int32]),
                           ("pond_step_timed", [P, dp])]:
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = C.c_int
        lib.pond_create.restype = C.c_int
        lib.pond_destroy.argtypes = [P]
        lib.pond_destroy.restype = None
        lib.pond_last_error.argtypes = [P]
        lib.pond_last_error.restype = C.c_char_p
        lib.pond_device_bytes.argtypes = [P]
        lib.pond_device_bytes.restype = C.c_size_t
        lib.pond_version.restype = C.c_char_p
        lib.pond_fma_peak.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.POINTER(C.c_double)]
        lib.pond_fma_peak.restype = C.c_int
        lib.pond_conservation_noalloc.argtypes = [C.c_void_p, C.c_int64, dp, C.c_void_p]
        lib.pond_conservation_noalloc.restype = C.c_int
        lib.pond_batch_create.argtypes = [C.c_void_p, C.POINTER(C.c_void_p)]
        lib.pond_batch_create.restype = C.c_int
        for name in ("pond_batch_add", "pond_batch_remove"):
            getattr(lib, name).argtypes = [C.c_void_p, C.c_void_p]
            getattr(lib, name).restype = C.c_int
        lib.pond_batch_step.argtypes = [C.c_void_p, C.c_int64]
        lib.pond_batch_step.restype = C.c_int
        lib.pond_batch_size.argtypes = [C.c_void_p]
        lib.pond_batch_size.restype = C.c_int32
        lib.pond_batch_last_error.argtypes = [C.c_void_p]
        lib.pond_batch_last_error.restype = C.c_char_p
        lib.pond_batch_destroy.argtypes = [C.c_void_p]
        lib.pond_batch_destroy.restype = None
        lib.pond_batch_set_budget.argtypes = [C.c_void_p, C.c_size_t]
        lib.pond_batch_set_budget.restype = C.c_int
        lib.pond_batch_bytes.argtypes = [C.c_void_p]
        lib.pond_batch_bytes.restype = C.c_size_t
        lib.pond_batch_poll.argtypes = [C.c_void_p, C.POINTER(C.c_int32)]
        lib.pond_batch_poll.restype = C.c_int
        _lib = lib
        return lib


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise PondError(3, "no CUDA device available (libpond has no CPU path)")
    return torch


class Simulation:
    """One PonD simulation on the current CUDA device (see include/pond.h).

    precision: "mixed" (FP32 populations and arithmetic, float-float EoS and conserved
    sums) or "fp64".
    """

    def __init__(self, nx: int, ny: int, *, bc_x: int = POND_PERIODIC, bc_y: int = POND_PERIODIC,
                 a: float = 2.0 / 49.0, b: float = 2.0 / 21.0, R: float = 1.0,
                 delta: float = 1.0 / 3.0, kappa: float = 0.0, tau: float = 1.0,
                 precision: str = "mixed", dt: float = 0.5, tol: float | None = None,
                 max_iter: int = 20, k_cond: float = -1.0, p_floor: float = 1e-3 / 6.0,
                 stream=None, torch_alloc: bool = True, ideal: bool = False,
                 lanes_per_node: int = 0, tile_x: int = 0, eos: str = "vdw",
                 isothermal: bool = False, T_iso: float = 0.0, nonlocal_: str = "lagged",
                 eos_params: tuple = (), lattice: str = "d2q9", nz: int = 1,
                 bc_z: int = POND_PERIODIC):
        torch = _torch()
        self._lib = load()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.N = self.nx * self.ny * self.nz
        self.precision = precision
        if precision not in ("mixed", "fp64"):
            raise ValueError("precision must be 'mixed' or 'fp64'")
        if tol is None:
            tol = 1e-6 if precision == "mixed" else 1e-12
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        self._device = self._stream.device
        self._blocks = {}
        if torch_alloc:
            dev, strm = self._device, self._stream

            def _alloc(nbytes, _ctx):
                try:
                    ptr = torch.cuda.caching_allocator_alloc(int(nbytes), dev, strm)
                except RuntimeError:
                    return None
                self._blocks[ptr] = nbytes
                return ptr

            def _free(ptr, _ctx):
                if ptr in self._blocks:
                    del self._blocks[ptr]
                    torch.cuda.caching_allocator_delete(ptr)

            self._cb_alloc, self._cb_free = _ALLOC(_alloc), _FREE(_free)
        else:
            self._cb_alloc, self._cb_free = _ALLOC(), _FREE()
        grid = Grid(self.nx, self.ny, bc_x, bc_y, self.nz, bc_z)
        if lattice not in LATTICES:
            raise ValueError("lattice must be 'd2q9', 'd2q16' or 'd3q27'")
        lat = Lattice(LATTICES[lattice])
        self.lattice = lattice
        self.nplanes = {"d2q9": 25, "d2q16": 39, "d3q27": 63}[lattice]
        # host arrays: (ny, nx) on the two-dimensional lattices, (nz, ny, nx) on D3Q27
        self.shape = (self.nz, self.ny, self.nx) if lattice == "d3q27" else (self.ny, self.nx)
        if eos not in ("vdw", "dieterici", "simplified"):
            raise ValueError("eos must be 'vdw', 'dieterici' or 'simplified'")
        kind = {"dieterici": POND_DIETERICI, "simplified": POND_SIMPLIFIED}.get(
            eos, POND_IDEAL if ideal else POND_VDW)
        sp = tuple(float(v) for v in eos_params) if eos == "simplified" else (0.0, 0.0, 0.0, 0.0)
        eos_c = Eos(kind, a, b, R, delta, 1 if isothermal else 0, float(T_iso), *sp)
        opts = Opts(POND_MIXED if precision == "mixed" else POND_FP64, max_iter, tol, dt, k_cond,
                    p_floor, C.c_void_p(self._stream.cuda_stream), self._cb_alloc, self._cb_free, None,
                    lanes_per_node, tile_x, {"lagged": 0, "current": 1}[nonlocal_])
        self.params = dict(nx=nx, ny=ny, bc_x=bc_x, bc_y=bc_y, a=a, b=b, R=R, delta=delta,
                           kappa=kappa, tau=tau, precision=precision, dt=dt, tol=tol,
                           max_iter=max_iter, k_cond=k_cond, p_floor=p_floor,
                           lanes_per_node=lanes_per_node, tile_x=tile_x, eos=eos,
                           isothermal=isothermal, T_iso=T_iso, nonlocal_=nonlocal_, lattice=lattice)
        ctx = C.c_void_p()
        with torch.cuda.device(self._device):
            st = self._lib.pond_create(C.byref(grid), C.byref(lat), C.byref(eos_c), kappa, tau,
                                       C.byref(opts), C.byref(ctx))
        if st != 0:
            raise PondError(st, "pond_create failed")
        self._ctx = ctx
        self.flags = []          # (status, message) of each warning a sync point returned
        self.last_flag = None    # the last sync point's warning, or None

    # -- helpers ---------------------------------------------------------
    def _check(self, st: int):
        if st != 0:
            raise PondError(st, self._lib.pond_last_error(self._ctx).decode())

    def _check_sync(self, st: int):
        """Status of a synchronising call: the warning-class sticky flags (frame search
        hit max_iter, pressure floor hit) are recorded in ``self.flags`` and do not raise;
        every other non-zero status raises."""
        if st in WARNINGS:
            self.flags.append((STATUS[st], self._lib.pond_last_error(self._ctx).decode()))
            self.last_flag = STATUS[st]
            return
        self.last_flag = None
        self._check(st)

    def _host(self, x) -> np.ndarray:
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(x, dtype=np.float64), self.shape))
        return a

    # -- API ---------------------------------------------------------------
    def init_fields(self, rho, ux, uy, T, uz=None):
        """Host numpy arrays (ny, nx) ((nz, ny, nx) on D3Q27) or CUDA float64 tensors;
        uz (host, D3Q27) defaults to zero."""
        if uz is not None:
            arrs = [self._host(v) for v in (rho, ux, uy, uz, T)]
            self._check(self._lib.pond_init_fields3(self._ctx, *[_dptr(a) for a in arrs]))
            return
        if hasattr(rho, "is_cuda") and rho.is_cuda:
            ts = [t.contiguous() for t in (rho, ux, uy, T)]
            self._check(self._lib.pond_init_fields_device(self._ctx, *[C.c_void_p(t.data_ptr()) for t in ts]))
            return
        arrs = [self._host(v) for v in (rho, ux, uy, T)]
        self._check(self._lib.pond_init_fields(self._ctx, *[_dptr(a) for a in arrs]))

    def step(self, n: int = 1):
        self._check(self._lib.pond_step(self._ctx, int(n)))

    def step_timed(self) -> float:
        """One step; duration of its kernel in milliseconds (CUDA events)."""
        out = np.zeros(1)
        self._check(self._lib.pond_step_timed(self._ctx, _dptr(out)))
        return float(out[0])

    def moments(self) -> dict:
        if self.lattice == "d3q27":
            outs = [np.empty(self.shape) for _ in range(6)]
            self._check_sync(self._lib.pond_moments3(self._ctx, *[_dptr(o) for o in outs]))
            return dict(zip(("rho", "ux", "uy", "uz", "T", "p"), outs))
        outs = [np.empty((self.ny, self.nx)) for _ in range(5)]
        self._check_sync(self._lib.pond_moments(self._ctx, *[_dptr(o) for o in outs]))
        return dict(zip(("rho", "ux", "uy", "T", "p"), outs))

    def moments_device(self, out: dict):
        """Write rho, ux, uy, T, p into given CUDA float64 tensors (keys may be absent)."""
        ptrs = [C.c_void_p(out[k].data_ptr()) if k in out else C.c_void_p() for k in
                ("rho", "ux", "uy", "T", "p")]
        self._check(self._lib.pond_moments_device(self._ctx, *ptrs))

    def conservation(self) -> np.ndarray:
        out = np.zeros(4)
        self._check_sync(self._lib.pond_conservation(self._ctx, _dptr(out)))
        return out

    def get_state(self) -> np.ndarray:
        out = np.empty((self.nplanes,) + self.shape)
        self._check(self._lib.pond_get_state(self._ctx, _dptr(out)))
        return out

    def set_state(self, state):
        s = np.ascontiguousarray(np.asarray(state, dtype=np.float64).reshape((self.nplanes,) + self.shape))
        self._check(self._lib.pond_set_state(self._ctx, _dptr(s)))

    def stats(self, reset: bool = False) -> dict:
        s = Stats()
        st = self._lib.pond_stats(self._ctx, C.byref(s), 1 if reset else 0)
        d = {k: int(getattr(s, k)) for k, _ in Stats._fields_}
        if st not in (0, 6):
            self._check(st)
        d["status"] = STATUS.get(st, st)
        return d

    def device_bytes(self) -> int:
        return int(self._lib.pond_device_bytes(self._ctx))

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.pond_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def conservation_noalloc(d_planes, n_nodes: int, stream=None) -> np.ndarray:
    """Conservation sums of a caller-owned D2Q9 device state in the 25-plane FP64 layout,
    computed without any device allocation (see pond_conservation_noalloc in pond.h).

    d_planes: a contiguous CUDA float64 tensor of exactly 25 * n_nodes values on the
    current device (checked here, since the C ABI cannot see the allocation and the
    kernel reads all 25 planes), or a raw device address, which is NOT checked: the
    caller then guarantees 25 * n_nodes doubles of a D2Q9 state on the current device."""
    lib = load()
    if hasattr(d_planes, "data_ptr"):
        import torch
        n = int(n_nodes)
        if n < 1:
            raise PondError(1, "n_nodes must be positive")
        if (not d_planes.is_cuda or d_planes.device != torch.device("cuda", torch.cuda.current_device())
                or d_planes.dtype != torch.float64 or not d_planes.is_contiguous()
                or d_planes.numel() != NPLANES * n):
            raise PondError(1, "d_planes must be a contiguous float64 tensor of 25 * n_nodes values "
                               "(a D2Q9 state) on the current CUDA device")
        ptr = d_planes.data_ptr()
    else:
        ptr = int(d_planes)
    sp = stream.cuda_stream if stream is not None and hasattr(stream, "cuda_stream") else stream
    out = np.zeros(4)
    st = lib.pond_conservation_noalloc(C.c_void_p(ptr), int(n_nodes), _dptr(out),
                                       C.c_void_p(sp) if sp else None)
    if st != 0:
        raise PondError(st, "pond_conservation_noalloc failed")
    return out


class Batch:
    """Many simulations advanced together, one launch per time step and kernel group
    (see pond_batch_* in pond.h).  Simulations keep their own API for init/moments."""

    def __init__(self, stream=None):
        torch = _torch()
        self._lib = load()
        self._stream = stream if stream is not None else torch.cuda.Stream()
        h = C.c_void_p()
        st = self._lib.pond_batch_create(C.c_void_p(self._stream.cuda_stream), C.byref(h))
        if st != 0:
            raise PondError(st, "pond_batch_create failed")
        self._h = h
        self.members = []

    def _check(self, st):
        if st != 0:
            raise PondError(st, self._lib.pond_batch_last_error(self._h).decode())

    def add(self, sim: Simulation):
        self._check(self._lib.pond_batch_add(self._h, sim._ctx))
        self.members.append(sim)

    def remove(self, sim: Simulation):
        self._check(self._lib.pond_batch_remove(self._h, sim._ctx))
        self.members.remove(sim)

    def step(self, n: int = 1):
        self._check(self._lib.pond_batch_step(self._h, int(n)))

    def set_budget(self, nbytes: int):
        """Device-memory budget of the members (0: no limit); add() then refuses a
        simulation that would exceed it with PondError(POND_ENOMEM)."""
        self._check(self._lib.pond_batch_set_budget(self._h, int(nbytes)))

    def device_bytes(self) -> int:
        return int(self._lib.pond_batch_bytes(self._h))

    def poll(self) -> bool:
        """True when the work of the last step() call has completed (no blocking)."""
        done = C.c_int32()
        self._check(self._lib.pond_batch_poll(self._h, C.byref(done)))
        return bool(done.value)

    def synchronize(self):
        self._stream.synchronize()

    def __len__(self):
        return int(self._lib.pond_batch_size(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.pond_batch_destroy(self._h)
            self._h = None
            self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def from_workload(w, precision: str = "mixed", **kw) -> Simulation:
    """Simulation for an ``inputs.Workload`` (parameters only; call init_fields)."""
    iso = dict(eos=w.eos, isothermal=w.isothermal, T_iso=float(w.T.flat[0]) if w.isothermal else 0.0,
               eos_params=tuple(w.eos_params))
    iso.update(kw)
    return Simulation(w.nx, w.ny, bc_x=w.bc_x, bc_y=w.bc_y, a=w.a, b=w.b, R=w.R, delta=w.delta,
                      kappa=w.kappa, tau=w.tau, precision=precision, dt=w.dt, k_cond=w.k_cond,
                      p_floor=w.p_floor, **iso)


def fma_peak(precision: str = "mixed", iters: int = 20000, stream=None) -> float:
    """Measured FMA-pipe peak of the current GPU in TFLOP/s (FP32 for "mixed", FP64 for
    "fp64"), from pond_fma_peak."""
    lib = load()
    out = C.c_double()
    strm = C.c_void_p(stream.cuda_stream) if stream is not None else None
    st = lib.pond_fma_peak(POND_MIXED if precision == "mixed" else POND_FP64, int(iters), strm, C.byref(out))
    if st != 0:
        raise PondError(st, "pond_fma_peak failed")
    return out.value
