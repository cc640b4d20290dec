"""Experiments of the paper run through the GPU path.

Non-classical waves (main text, Fig. 4; SM "Shock tube"): a shock keeps its steepness as
it travels, an expansion fan spreads, so the peak density gradient of each half of the
tube at t*/2 and at t* tells a rarefaction shock (steepness kept) from a rarefaction fan
(steepness halved).

Coexistence (main text, Fig. 2): a liquid slab in its vapour (``inputs.coexistence_slab``)
relaxes to the saturated densities; they are read as the means of the lowest and highest
quarter of the density field, which is independent of where the slab is (it moves in the
advected case).

Speed of sound (main text, Fig. 1; SM "Speed of sound"): a small density bump in a
uniform state (``inputs.sound_pulse``) splits into two sound pulses; the speed of the
right-going one is the slope of its pressure centroid against time.  The measurement
uses only the simulated fields, so it can be set against the closed form
sqrt((dp/drho)_T + T (dp/dT)_rho^2 / (rho^2 C_v)) independently.
"""
from __future__ import annotations

import math

import numpy as np

from . import pond


def pulse_centroid(p: np.ndarray, x0: float) -> float:
    """Centroid of the pressure excess of the right-going pulse: positive part of
    p - p_far over the half domain [x0, x0 + nx/2), where p_far is the pressure at the
    antipode x0 + nx/2 (not yet reached by either pulse).  p: one row of nx values."""
    nx = p.shape[0]
    xs = np.arange(nx, dtype=np.float64)
    far = p[int(round(x0 + nx / 2)) % nx]
    sel = (xs >= x0) & (xs < x0 + nx / 2)
    d = np.clip(p[sel] - far, 0.0, None)
    tot = d.sum()
    return float((xs[sel] * d).sum() / tot) if tot > 0 else float("nan")


def sound_speed(w, precision: str = "mixed", travel=(0.08, 0.3), stream=None, **kw) -> dict:
    """Steps the sound-pulse workload `w` on the GPU, samples the right-going pulse's
    centroid X(t) every ~nx/400 time units until it has travelled travel[1] * nx nodes
    (or w.steps are done), and fits X = X_0 + c t over the samples with
    travel[0] * nx <= X - x0 <= travel[1] * nx.  Returns c and the run's bookkeeping."""
    x0 = w.nx / 4.0
    chunk = max(1, int(math.ceil(w.nx / 400.0 / w.dt)))
    ts, xs = [], []
    done = 0
    with pond.from_workload(w, precision=precision, stream=stream, **kw) as sim:
        sim.init_fields(*w.fields())
        while done < w.steps:
            n = min(chunk, w.steps - done)
            sim.step(n)
            done += n
            p = sim.moments()["p"].mean(axis=0)
            X = pulse_centroid(p, x0)
            ts.append(done * w.dt)
            xs.append(X)
            if X - x0 >= travel[1] * w.nx:
                break
        stats = sim.stats()
    t = np.array(ts)
    X = np.array(xs)
    m = (X - x0 >= travel[0] * w.nx) & (X - x0 <= travel[1] * w.nx)
    if m.sum() < 3:
        raise RuntimeError("sound pulse: too few samples in the fit window (%d)" % m.sum())
    c, _ = np.polyfit(t[m], X[m], 1)
    return {"c": float(c), "samples": int(m.sum()), "steps": done, "time": float(t[-1]),
            "nonfinite": int(stats["nonfinite"])}


def bulk_densities(rho: np.ndarray) -> tuple[float, float]:
    """(vapour, liquid) bulk densities of a field holding half of each phase: the means
    of its lowest and highest quarter of values (interfaces take a small share)."""
    r = np.sort(rho.ravel())
    q = max(1, r.size // 4)
    return float(r[:q].mean()), float(r[-q:].mean())


def coexistence(w, precision: str = "mixed", settle: float = 0.75, samples: int = 8, stream=None,
                **kw) -> dict:
    """Steps the slab workload `w` for settle * w.steps, then averages the bulk densities
    over `samples` snapshots spread over the remaining steps."""
    n_settle = int(settle * w.steps)
    per = max(1, (w.steps - n_settle) // samples)
    rv, rl = [], []
    with pond.from_workload(w, precision=precision, stream=stream, **kw) as sim:
        sim.init_fields(*w.fields())
        sim.step(n_settle)
        for _ in range(samples):
            sim.step(per)
            v, l = bulk_densities(sim.moments()["rho"])
            rv.append(v)
            rl.append(l)
        stats = sim.stats()
    return {"rho_v": float(np.mean(rv)), "rho_l": float(np.mean(rl)),
            "steps": n_settle + samples * per, "nonfinite": int(stats["nonfinite"]),
            "clamped": int(stats["clamped"])}


def wave_steepness(w, precision: str = "mixed", stream=None, **kw) -> dict:
    """Steps the tube workload `w` to half its steps and to all of them; at both times
    returns, for the left and the right half of the tube, the peak |rho(x+1) - rho(x)| and
    where it is, plus the density on both sides of the left half's front (10 nodes
    away)."""
    out = {}
    with pond.from_workload(w, precision=precision, stream=stream, **kw) as sim:
        sim.init_fields(*w.fields())
        done = 0
        for tag, n in (("half", w.steps // 2), ("end", w.steps)):
            sim.step(n - done)
            done = n
            r = sim.moments()["rho"].mean(axis=0)
            g = np.abs(np.diff(r))
            h = w.nx // 2
            il, ir = int(np.argmax(g[:h])), h + int(np.argmax(g[h:]))
            out[tag] = {"left_peak": float(g[il]), "left_at": il, "right_peak": float(g[ir]),
                        "right_at": ir, "left_outer": float(r[max(0, il - 10)]),
                        "left_inner": float(r[min(w.nx - 1, il + 11)])}
        out["nonfinite"] = int(sim.stats()["nonfinite"])
    return out
