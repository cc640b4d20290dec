"""Helpers shared by the GPU parity tests: oracle runs, error norms, tolerances."""
import numpy as np

import oracle

# per-field relative L-infinity bars: FP64 GPU vs FP64 oracle, mixed FP32/FP64 vs oracle
TOL = {"fp64": 1e-11, "mixed": 1e-5}
# velocity errors are normalised by max(|uhat|, sqrt(max p/rho)): the fluid is often
# nearly at rest, and the speed scale of the populations is the isothermal speed
FIELDS = ("rho", "ux", "uy", "T", "p")


def params_of(w, **over) -> oracle.Params:
    kw = dict(nx=w.nx, ny=w.ny, bc_x=w.bc_x, bc_y=w.bc_y, a=w.a, b=w.b, R=w.R, delta=w.delta,
              kappa=w.kappa, tau=w.tau, dt=w.dt, k_cond=w.k_cond, p_floor=w.p_floor, tol=1e-12,
              max_iter=20, eos=w.eos, isothermal=w.isothermal, eos_params=tuple(w.eos_params),
              T_iso=float(w.T.flat[0]) if w.isothermal else 0.0)
    kw.update(over)
    return oracle.Params(**kw)


def oracle_run(w, steps=None, **over):
    P = params_of(w, **over)
    st = oracle.init_state(P, *w.fields())
    stats = {}
    st = oracle.step(P, st, w.steps if steps is None else steps, stats)
    return P, st, stats


def rel_linf(got: dict, ref: dict) -> dict:
    out = {}
    for k in FIELDS:
        g, r = np.asarray(got[k]), np.asarray(ref[k])
        scale = np.abs(r).max()
        if k in ("ux", "uy"):
            cs = np.sqrt(np.max(np.abs(np.asarray(ref["p"]) / np.asarray(ref["rho"]))))
            scale = max(scale, cs)
        out[k] = float(np.abs(g - r).max() / scale)
    return out


def state_fields(P, rows: np.ndarray) -> dict:
    """Macroscopic fields of node-major state rows (n, 25) (as oracle.moments)."""
    rho, T = rows[:, 21], rows[:, 22]
    p = rho * P.R * T / (1.0 - P.b * rho) - P.a * rho * rho
    return {"rho": rho, "ux": rows[:, 23], "uy": rows[:, 24], "T": T, "p": p}


def sample_nodes(nx: int, ny: int, count: int, seed: int = 7) -> np.ndarray:
    """Corners, edge midpoints and seeded interior nodes (flat indices)."""
    r = np.random.default_rng(seed)
    fixed = [(0, 0), (nx - 1, 0), (0, ny - 1), (nx - 1, ny - 1), (nx // 2, ny // 2),
             (nx // 2, 0), (0, ny // 2), (nx - 1, ny // 2), (nx // 2, ny - 1)]
    pts = {y * nx + x for x, y in fixed}
    while len(pts) < count:
        pts.add(int(r.integers(0, nx * ny)))
    return np.array(sorted(pts), dtype=np.int64)
