"""Benchmark of the PonD van der Waals time step on GB300.

Workload (default): the droplet-shock interaction, 2048 x 1024 nodes, T = 0.8 T_cr, a
liquid droplet of radius 80 at x = 600 hit by a Mach 1.5 shock (Rankine-Hugoniot state of
the van der Waals fluid) from x = 300, zero-gradient boundaries: the largest single-GPU
workload.  One bench "step" = one time step of the whole hot path (non-local terms,
frame search with streaming, collision: one launch of the fused step kernel) over the
grid.  Metric: MLUPS (million node updates per second) in the mixed FP32/FP64 form; the
plain FP64 form of the same workload (its own roofline), the shock tube and the other
workloads, a bounded continuous-batching serving sample and the FP64 CPU oracle are
reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
                  [--workload NAME] [--impl reference] [--no-cpu] [--no-serving]
                  [--no-autotune] [--no-extras]

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events on the
simulation's stream.  The 2048 x 1024 state (268 MB per FP32 buffer) is larger than L2;
for workloads whose state fits in L2 a 512 MiB buffer is written between timed steps.
A step is one kernel launch, so the roofline's kernel time is the same per-step event
time.  The launch shape (lanes per node, tile shape) comes from the autotuner.  Under
torchrun (N > 1) each rank runs an independent replica (the workload does not shard) and
the slowest rank's time counts.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


def peaks() -> dict:
    try:
        with open(MEASURED) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)),
                "src": "measured"}
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM_GBS, "sm_max_mhz": 2070.0, "src": "fallback"}


# FP32 / FP64 ALU peaks of GB300 from unit counts and the maximum SM clock:
# 152 SMs x 128 FP32 lanes x 2 flop/FMA; FP64 at 1/64 of the FP32 rate.
def alu_peak_tflops(precision: str, sm_mhz: float) -> float:
    fp32 = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    return fp32 if precision == "mixed" else fp32 / 64.0


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in the background."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict:
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[3 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload(name: str):
    from paper_2002_09217_gb300 import inputs
    return inputs.config(name)


def bytes_per_update(precision: str, lattice: str = "d2q9") -> int:
    e = 4 if precision == "mixed" else 8
    if lattice == "d2q16":
        # the 44-value record read once (populations, gauge, fields, kept remainders) and
        # written once, rho and T read again by the non-local kernels (2 values), and the
        # nine FP64 non-local planes written and read once
        return (44 + 44 + 2) * e + 2 * 9 * 8
    # state read once (f, g, gauge, rho, T: 23 values) + written once (25 values)
    return 48 * e


# Algorithmic FLOPs of the D2Q9 step kernel's formula (an FMA counts 2).  A stream of a
# node transforms each node of its stencil region (the union of its nine directions'
# 4x4 stencils, counted by the kernel: pond_stats region_nodes) once for all directions:
#  per region node: gauge offsets (9), the per-axis transfer increments from h = e/2 and
#  p = h (2c + e) (42), the nine weight products (9), and per population family the
#  x-transform of the three source rows (45), the sums for the y-transform (9), the
#  increment-form outputs (72) and the weighted accumulation (18) => 348;
#  per stream: departure points, Lagrange weight tables and moment sums of the nine
#  directions (9 x 20) and the moments, EoS and residual (60) => 240;
#  streams of regions wider than 8 nodes take the per-direction path: per stencil pair
#  (9 directions x 16 stencil nodes) gauge offsets (8), six transfer increments (24), the
#  x-increments of three source rows for f and g (30), the f and g components (22),
#  weight and accumulation (7) => 91, plus the same 240 per stream;
#  per node update: the Korteweg tensor, heat flux and their divergences counted once per
#  node (200; the kernel recomputes them at each neighbour) and the collision (1300:
#  transfer rows of both axes ~230, forced g equilibrium ~410, BGK updates ~150, carrying
#  X* into the streaming gauge ~390, exact rest-population remainders ~100).
FLOPS_REGION_NODE = 348
FLOPS_PAIR = 91
FLOPS_DIR = 20
FLOPS_STREAM_EXTRA = 60
FLOPS_NONLOCAL = 200
FLOPS_COLLIDE = 1300


def flops_d2q9(st: dict, updates: int) -> float:
    """FLOPs per node update of the D2Q9 step from its counters (pond_stats)."""
    per_stream = 9 * FLOPS_DIR + FLOPS_STREAM_EXTRA
    pair_streams = st.get("pair_streams", 0)
    total = (st["region_nodes"] * FLOPS_REGION_NODE + st["streams"] * per_stream
             + pair_streams * 9 * 16 * FLOPS_PAIR + updates * (FLOPS_NONLOCAL + FLOPS_COLLIDE))
    return total / max(1, updates)

# The same count for the D2Q16 step (k_q16_step), per node update.  Region stream, per
# region node (the union of the sixteen 4 x 4 departure stencils, 5 x 5 for |v| dt < 1):
# gauge offsets (9), both per-axis increment maps (eight rows of 31 and their offsets 16:
# 264), for f and g the x-increments (128), the y-increments (144) and the weighted
# accumulation (80), the weight products (16) => 990; per region stream: departure floors,
# cubic weights and tables of both axes (220).  Per-pair fallback stream (regions wider
# than 6): per stencil pair (16 directions x 16 stencil nodes) gauge offsets (9), the eight
# increments of the pair's row per axis (16 for their offsets, 82 for the entries), the
# x-increments of the four source rows for f and g (64), the y-increment (24), weight and
# accumulation (11) => 206, per direction departure points and cubic weights (40).  Per
# stream: moments and residual (FP64, 130); per node update: non-local terms (200) and the
# collision (2300: four per-axis increment maps ~700, three tensor-product applications
# ~900, forced g equilibrium ~640, mass and energy defect sums ~70).
FLOPS_Q16_REGION_NODE = 990
FLOPS_Q16_REGION_STREAM = 220
FLOPS_Q16_PAIR = 206
FLOPS_Q16_DIR = 40
FLOPS_Q16_STREAM_EXTRA = 130
FLOPS_Q16_COLLIDE = 2300


def flops_q16(st: dict, updates: int) -> float:
    """FLOPs per node update of the D2Q16 step from its counters (pond_stats)."""
    pair = st.get("pair_streams", 0)
    total = (st["region_nodes"] * FLOPS_Q16_REGION_NODE + (st["streams"] - pair) * FLOPS_Q16_REGION_STREAM
             + st["streams"] * FLOPS_Q16_STREAM_EXTRA + pair * 16 * (FLOPS_Q16_DIR + 16 * FLOPS_Q16_PAIR)
             + updates * (FLOPS_NONLOCAL + FLOPS_Q16_COLLIDE))
    return total / max(1, updates)


# The D3Q27 step (k_q27_step), per node update.  Region stream, per region node (the
# union of the 27 departure stencils of 4 x 4 x 4, 5 x 5 x 5 for |v| dt < 1), for each of the
# two population passes: gauge offsets (11), the three per-axis increment maps (123), the
# weight products (27), x-, y- and z-increments (3 x 135), the running sums of the
# increments (135) and the accumulation (81) => 782, 1564 per node; per region stream:
# departure floors, cubic weights and tables of the three axes (175).  Per-pair fallback
# stream (regions wider than 6): per stencil pair (27 directions x 64 stencil nodes) gauge
# offsets (29), the three per-axis increment rows (60), the x-, y- and z-increments and
# accumulation for f and g (198), weight (2) => 289, per direction three departure points
# and cubic weights (60).  Per stream: moments and residual (FP64, 260); per node update:
# non-local terms (600) and the collision (7000: six per-axis increment maps ~360, three
# three-axis applications ~4800, forced g equilibrium ~1620, defect sums ~300).
FLOPS_Q27_REGION_NODE = 1564
FLOPS_Q27_REGION_STREAM = 175
FLOPS_Q27_PAIR = 289
FLOPS_Q27_DIR = 60
FLOPS_Q27_STREAM_EXTRA = 260
FLOPS_Q27_NONLOCAL = 600
FLOPS_Q27_COLLIDE = 7000


def flops_q27(st: dict, updates: int) -> float:
    """FLOPs per node update of the D3Q27 step from its counters (pond_stats)."""
    pair = st.get("pair_streams", 0)
    total = (st["region_nodes"] * FLOPS_Q27_REGION_NODE + (st["streams"] - pair) * FLOPS_Q27_REGION_STREAM
             + st["streams"] * FLOPS_Q27_STREAM_EXTRA + pair * 27 * (FLOPS_Q27_DIR + 64 * FLOPS_Q27_PAIR)
             + updates * (FLOPS_Q27_NONLOCAL + FLOPS_Q27_COLLIDE))
    return total / max(1, updates)


def d3q27_run(pond, torch, stream, precision, steps, warmup, nx=96, ny=96, nz=64, sm_mhz=2070.0) -> dict:
    """MLUPS of the D3Q27 step on a liquid sphere in its vapour (96 x 96 x 64 nodes, 72-value
    records; 0.6 M nodes x 288 B = 170 MB per FP32 state buffer, larger than L2), with its
    ALU roofline and an end-to-end figure (host fields in, steps, host fields out)."""
    import numpy as np
    from paper_2002_09217_gb300 import inputs
    w = inputs.droplet3d(n=nx, ny=ny, nz=nz, radius=20.0)
    sim = pond.Simulation(w.nx, w.ny, stream=stream, **inputs.from_workload3(w, precision))
    sim.init_fields(w.rho, w.ux, w.uy, w.T)
    sim.step(warmup)
    stream.synchronize()
    sim.stats(reset=True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    sim.step(steps)
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b) / steps
    st = sim.stats()
    its = st["streams"] / max(1, st["node_updates"])
    t0 = time.perf_counter()
    sim.init_fields(*[np.ascontiguousarray(x) for x in (w.rho, w.ux, w.uy, w.T)], uz=w.uz)
    sim.step(steps)
    sim.moments()
    e2e = w.nodes * steps / (time.perf_counter() - t0) / 1e6
    sim.close()
    fl = flops_q27(st, st["node_updates"])
    achieved = w.nodes * fl / (ms * 1e-3) / 1e12
    peak = alu_peak_tflops(precision, sm_mhz)
    return {"workload": w.name, "mlups": w.nodes / ms / 1e3, "ms_per_step": ms, "streams_per_node": its,
            "e2e_mlups": e2e,
            "roofline": {"bound": "alu", "kernel": "k_q27_step (+ two non-local kernels, timed together)",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "flops_per_update": fl}}


# DRAM bytes per launch of k_pond_step (dram__bytes_read.sum + dram__bytes_write.sum) from
# one ncu capture of the bench workload; they hold only for the kernel source they were
# taken on (sha256 over the two kernel headers), any other source reports null.
NCU_TRAFFIC = {"kernel_sha256": "804944b3cf14dfdb4985ac6b9233784f0279b3f7c34f8b526fea166cf068bb7f",
               "bytes": {"dropletshock2048x1024/mixed": 637875968.0,
                         "dropletshock2048x1024/fp64": 1170719488.0}}


def kernel_sha256() -> str:
    h = hashlib.sha256()
    for f in ("pond_step.cuh", "pond_kernels.cuh"):
        with open(os.path.join(ROOT, "paper_2002_09217_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def ncu_traffic(w, precision):
    if kernel_sha256() != NCU_TRAFFIC["kernel_sha256"]:
        return None
    return NCU_TRAFFIC["bytes"].get("%s/%s" % (w.name, precision))


def oracle_mlups(w, steps: int, lattice: str = "d2q9", warmup: int = 1) -> dict:
    import oracle
    P = oracle.Params(nx=w.nx, ny=w.ny, bc_x=w.bc_x, bc_y=w.bc_y, a=w.a, b=w.b, R=w.R,
                      delta=w.delta, kappa=w.kappa, tau=w.tau, dt=w.dt, k_cond=w.k_cond,
                      p_floor=w.p_floor, tol=1e-12, max_iter=20, eos=w.eos, isothermal=w.isothermal,
                      eos_params=tuple(w.eos_params),
                      T_iso=float(w.T.flat[0]) if w.isothermal else 0.0, lattice=lattice)
    st = oracle.init_state(P, *w.fields())
    st = oracle.step(P, st, max(1, warmup))   # warm-up (page-in, thread pool)
    t0 = time.perf_counter()
    st = oracle.step(P, st, steps)
    dt = time.perf_counter() - t0
    return {"value": w.nodes * steps / dt / 1e6, "unit": "MLUPS", "cores": oracle.num_threads(),
            "kind": "oracle", "seconds": dt,
            "sample": "%d time steps of the full %dx%d grid (FP64 oracle, %s, OpenMP over nodes)"
                      % (steps, w.nx, w.ny, lattice.upper()), "state": st, "params": P}


L2_BYTES = 129e6


def state_bytes(w, precision: str) -> float:
    """Bytes of one state buffer (32-value records) of a D2Q9 workload."""
    return w.nodes * 32 * (4 if precision == "mixed" else 8)


def run_form(w, pond, torch, stream, flush, precision, steps, warmup, shape, ws):
    """Timed steps of one precision form: per-step CUDA events; the L2 is flushed between
    timed steps when the state fits in it.  Returns the per-step times, the counters and
    the mean kernel time (the step is one launch: the same events)."""
    sim = pond.from_workload(w, precision=precision, stream=stream, **shape)
    dev_fields = [torch.tensor(a, device=stream.device, dtype=torch.float64) for a in w.fields()]
    with torch.cuda.stream(stream):
        sim.init_fields(*dev_fields)
        sim.step(warmup)
    stream.synchronize()
    sim.stats(reset=True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    do_flush = state_bytes(w, precision) < 2 * L2_BYTES
    with torch.cuda.stream(stream):
        for k in range(steps):
            if do_flush:
                flush.fill_(float(k))
            evs[k][0].record(stream)
            sim.step(1)
            evs[k][1].record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in evs]
    st = sim.stats()
    sim.close()
    return ms, st, sum(ms) / len(ms)


def roofline(w, precision, its, kernel_ms, pk, lattice="d2q9", st=None, updates=0):
    if lattice == "d2q16":
        fl = flops_q16(st, updates)
        kernel, traffic = "k_q16_step (+ two non-local kernels, timed together)", None
    else:
        fl = flops_d2q9(st, updates)
        kernel, traffic = "k_pond_step", ncu_traffic(w, precision)
    achieved = w.nodes * fl / (kernel_ms * 1e-3) / 1e12
    peak = alu_peak_tflops(precision, pk["sm_max_mhz"])
    out = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak,
           "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
           "peak_src": "%s: 152 SM x 128 lanes x 2 flop x %.0f MHz%s" % (
               "FP32" if precision == "mixed" else "FP64", pk["sm_max_mhz"],
               "" if precision == "mixed" else " / 64"),
           "flops_per_update": fl, "kernel_ms": kernel_ms}
    fma = pk.get("fma_" + precision)
    if fma:
        # the same GPU's FMA-chain microbenchmark (pond_fma_peak), beside the derived peak
        out["peak_measured_fma"] = fma
        out["frac_of_measured_fma"] = achieved / fma
    return out


def end_to_end(w, pond, torch, stream, precision, shape, n_seg: int, reps: int) -> dict:
    import numpy as np
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in w.fields()]
    sim = pond.from_workload(w, precision=precision, stream=stream, **shape)
    times = []
    for r in range(reps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.init_fields(*[h.numpy() for h in host])
        sim.step(n_seg)
        sim.moments()
        times.append(time.perf_counter() - t0)
    sim.close()
    t = statistics.median(times[1:])
    return {"value": w.nodes * n_seg / t / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": 4 * w.nodes * 8 / n_seg, "d2h_bytes_per_step": 5 * w.nodes * 8 / n_seg,
            "segment_steps": n_seg,
            "note": "per call: init from pinned host (4 fields), %d steps, 5 fields back to host" % n_seg}


def serving_run(torch, rank: int, ws: int, n_req: int = 32, side_cap: int = 256,
                steps_scale: dict | None = None, tr_min: float = 0.8, rate: float = 200.0,
                budget: int = 8 << 30, check: int = 0) -> dict:
    """The seeded serving mix served by the batching server, scaled as stated in the
    returned `sample` (sides capped at side_cap, step counts times steps_scale per
    precision, temperatures raised to tr_min; None/1.0 leaves a quantity as specified).
    With several ranks each serves its placement share (no data exchange).  `check`
    requests (a seeded subset, half of each precision) keep their final state for the
    accuracy check (serving_accuracy)."""
    import dataclasses
    import random
    from paper_2002_09217_gb300 import inputs, placement, serving
    steps_scale = steps_scale or {"mixed": 0.1, "fp64": 0.1}
    reqs = inputs.serving_requests(n=n_req, rate=rate)
    reqs = [dataclasses.replace(r, side=min(r.side, side_cap) if side_cap else r.side,
                                steps=max(100, int(round(r.steps * steps_scale[r.precision]))),
                                T_r=max(r.T_r, tr_min) if tr_min else r.T_r) for r in reqs]
    mine = placement.my_share(reqs, rank, ws) if ws > 1 else reqs
    keep = set()
    if check:
        rng = random.Random(20020921)
        for prec in ("mixed", "fp64"):
            ids = [r.rid for r in mine if r.precision == prec]
            keep |= set(rng.sample(ids, min(len(ids), check // 2)))
    server = serving.Server(hbm_budget=budget, chunk=50, keep_fields=False, keep_state=keep)
    t0 = time.perf_counter()
    results = server.run(mine)
    wall = time.perf_counter() - t0
    server.close()
    util = server.used_seconds / max(1e-9, wall) / budget
    if ws > 1:
        import torch.distributed as dist
        gathered = [None] * ws
        dist.all_gather_object(gathered, (results, wall))
        results = [r for part, _ in gathered for r in part]
        wall = max(w for _, w in gathered)
    summ = serving.summarize(results, wall)
    summ["nonfinite_requests"] = sum(1 for r in results if r.status.get("nonfinite", 0))
    by_rid = {q.rid: q for q in reqs}
    summ["nonfinite"] = [{"rid": r.rid, "kind": by_rid[r.rid].kind, "T_r": float(by_rid[r.rid].T_r),
                          "mach": float(by_rid[r.rid].mach), "side": by_rid[r.rid].side, "steps": r.steps,
                          "precision": r.precision} for r in results if r.status.get("nonfinite", 0)]
    summ["budget_bytes"] = budget
    summ["budget_mean_use"] = util
    summ["budget_peak_use"] = server.peak_bytes / budget
    summ["refused_after_create"] = server.refused
    scaled = ", ".join("%s steps x %g" % (k, v) for k, v in steps_scale.items() if v != 1.0) or "steps as specified"
    summ["sample"] = ("%d requests of the seeded mix (sides %s, %s, T_r %s), mixed and FP64 "
                      "as drawn, Poisson %g/s, %.1f GiB budget" % (
                          n_req, "<= %d" % side_cap if side_cap else "64..1024 as drawn", scaled,
                          ">= %g" % tr_min if tr_min else "0.70..0.95 as drawn", rate, budget / 2 ** 30))
    summ["_kept"] = [r for r in results if r.state is not None]
    return summ


def serving_accuracy(pond, kept, nsample: int = 64) -> dict:
    """One-step check of served results: each kept final state is stepped once more on the
    GPU (alone, its own precision) and by the FP64 oracle at sampled nodes (half in
    interfaces and fronts); relative L-infinity per request against the bar of its form."""
    import numpy as np
    import oracle
    bars = {"mixed": 1e-5, "fp64": 1e-11}
    rows = []
    for r in kept:
        w = r.workload
        P = oracle.Params(nx=w.nx, ny=w.ny, bc_x=w.bc_x, bc_y=w.bc_y, a=w.a, b=w.b, R=w.R, delta=w.delta,
                          kappa=w.kappa, tau=w.tau, dt=w.dt, k_cond=w.k_cond, p_floor=w.p_floor,
                          tol=1e-12 if r.precision == "fp64" else 1e-6, max_iter=20)
        st = r.state.reshape(25, -1)
        if not np.isfinite(st).all():
            rows.append({"rid": r.rid, "precision": r.precision, "finite": False})
            continue
        rho = st[21].reshape(w.ny, w.nx)
        g = (np.abs(np.roll(rho, -1, 1) - np.roll(rho, 1, 1)) + np.abs(np.roll(rho, -1, 0) - np.roll(rho, 1, 0))).ravel()
        rng = np.random.default_rng(r.rid)
        steep = rng.choice(np.argsort(g)[::-1][: 8 * nsample], nsample // 2, replace=False)
        nodes = np.unique(np.concatenate([steep, rng.choice(w.nodes, nsample // 2, replace=False)]))
        with pond.from_workload(w, precision=r.precision) as sim:
            sim.set_state(r.state)
            sim.step(1)
            got = sim.get_state().reshape(25, -1)[:, nodes].T
        ref = oracle.step_nodes(P, r.state, nodes)
        err = 0.0
        for k, col in (("rho", 21), ("T", 22)):
            err = max(err, float(np.abs(got[:, col] - ref[:, col]).max() / np.abs(ref[:, col]).max()))
        cs = float(np.sqrt(np.max(np.abs(ref[:, 18]) * (1.0 / 3.0))))
        for col in (23, 24):
            err = max(err, float(np.abs(got[:, col] - ref[:, col]).max() / max(np.abs(ref[:, col]).max(), cs)))
        rows.append({"rid": r.rid, "precision": r.precision, "side": w.nx, "steps": r.steps, "T_r": round(w.T_r, 2),
                     "linf": err, "within_bar": err <= bars[r.precision], "finite": True})
    return {"checked": len(rows), "within_bar": sum(1 for x in rows if x.get("within_bar")),
            "max_linf": {p: max([x["linf"] for x in rows if x["precision"] == p and x.get("finite")] or [0.0])
                         for p in ("mixed", "fp64")},
            "requests": rows, "nodes_per_request": nsample}


def serving_sample(torch, rank: int, ws: int, n_req: int = 32) -> dict:
    """Bounded sample for the default bench run: sides <= 256, steps / 10, T_r >= 0.8,
    arrivals at 200 requests/s, 8 GiB budget."""
    summ = serving_run(torch, rank, ws, n_req=n_req)
    summ.pop("_kept", None)
    return summ


def other_configs(pond, torch, stream, sm_mhz: float = 2070.0, skip: str = "") -> dict:
    """MLUPS of the other full-size workloads (default launch shape, a few back-to-back
    steps after warm-up; the larger ones exceed L2 by themselves), both forms."""
    from paper_2002_09217_gb300 import inputs
    out = {}
    for name, steps in (("slab128x4", 200), ("shocktube2048x4", 200), ("droplet512x512", 20),
                        ("dropletshock2048x1024", 10)):
        if name == skip:
            continue
        w = inputs.config(name)
        for prec in ("mixed", "fp64"):
            n = steps if prec == "mixed" or w.nodes < 10000 else max(3, steps // 5)
            sim = pond.from_workload(w, precision=prec, stream=stream)
            sim.init_fields(*w.fields())
            sim.step(3)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim.step(n)
            b.record(stream)
            b.synchronize()
            ms = a.elapsed_time(b) / n
            st = sim.stats()
            sim.close()
            out["%s/%s" % (name, prec)] = {"mlups": w.nodes / ms / 1e3, "ms_per_step": ms,
                                           "streams_per_node": st["streams"] / max(1, st["node_updates"])}
    # the D2Q16 lattice on the 512 x 512 droplet (three launches per step: the two
    # non-local kernels and the node step); achieved FLOP/s of the step from the formula's
    # count above against the ALU peak of its precision
    w = inputs.config("droplet512x512")
    for prec, steps in (("mixed", 20), ("fp64", 3)):
        sim = pond.from_workload(w, precision=prec, stream=stream, lattice="d2q16")
        sim.init_fields(*w.fields())
        sim.step(3)
        sim.stats(reset=True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.step(steps)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b) / steps
        st = sim.stats()
        sim.close()
        its = st["streams"] / max(1, st["node_updates"])
        fl = flops_q16(st, st["node_updates"])
        achieved = w.nodes * fl / (ms * 1e-3) / 1e12
        peak = alu_peak_tflops(prec, sm_mhz)
        out["%s/d2q16/%s" % (w.name, prec)] = {
            "mlups": w.nodes / ms / 1e3, "ms_per_step": ms, "streams_per_node": its,
            "roofline": {"bound": "alu", "kernel": "k_q16_step (+ two non-local kernels)",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "flops_per_update": fl}}
    # the D3Q27 lattice on a 96 x 96 x 64 liquid sphere
    for prec, steps in (("mixed", 5), ("fp64", 2)):
        out["droplet3d96x96x64/d3q27/%s" % prec] = d3q27_run(pond, torch, stream, prec, steps, 2, sm_mhz=sm_mhz)
    # the two-pass step (current-time non-local terms) on the slab: two launches per step
    w = inputs.config("slab128x4")
    sim = pond.from_workload(w, precision="mixed", stream=stream, nonlocal_="current")
    sim.init_fields(*w.fields())
    sim.step(3)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    sim.step(200)
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b) / 200
    sim.close()
    out["slab128x4/mixed/current_time"] = {"mlups": w.nodes / ms / 1e3, "ms_per_step": ms}
    # the speed-of-sound experiment (saturated liquid at 0.9 T_cr): pulse speed from the
    # simulated pressure field, sampled every ~5 time units (closed form: 0.53588)
    from paper_2002_09217_gb300 import experiments
    w = inputs.sound_pulse(0.9, "liquid", nx=2048, width=12.0)
    t0 = time.perf_counter()
    res = experiments.sound_speed(w, "mixed", stream=stream)
    el = time.perf_counter() - t0
    out["%s/mixed" % w.name] = {"c_measured": res["c"], "steps": res["steps"], "wall_s": el,
                                "mlups_incl_sampling": w.nodes * res["steps"] / el / 1e6}
    # the anomalous shock tube (delta = 0.0125): steepness of the left (rarefaction shock)
    # and right fronts at t*/2 and t*
    w = inputs.nonclassical_tube("fig4", nx=1024)
    t0 = time.perf_counter()
    res = experiments.wave_steepness(w, "mixed", stream=stream)
    el = time.perf_counter() - t0
    out["%s/mixed" % w.name] = {"left_peak_half": res["half"]["left_peak"], "left_peak_end": res["end"]["left_peak"],
                                "steps": w.steps, "wall_s": el, "mlups_incl_reads": w.nodes * w.steps / el / 1e6}
    # the coexistence experiment (flat slab at 0.9 T_cr, delta = 1/3): saturated densities
    # from the relaxed field (Maxwell: 1.490096 / 5.800446)
    w = inputs.coexistence_slab(0.9, nx=256, steps=4000)
    t0 = time.perf_counter()
    res = experiments.coexistence(w, "mixed", stream=stream)
    el = time.perf_counter() - t0
    out["%s/mixed" % w.name] = {"rho_v": res["rho_v"], "rho_l": res["rho_l"], "steps": res["steps"],
                                "wall_s": el}
    return out


def parity_vs_oracle(w, pond, stream, precision, shape, res, steps) -> dict:
    import numpy as np
    import oracle
    ref = oracle.moments(res["params"], res["state"])
    sim = pond.from_workload(w, precision=precision, stream=stream, **shape)
    sim.init_fields(*w.fields())
    sim.step(steps)
    got = sim.moments()
    sim.close()
    out = {}
    cs = float(np.sqrt(np.max(np.abs(ref["p"] / ref["rho"]))))
    for k in ("rho", "ux", "uy", "T", "p"):
        scale = np.abs(ref[k]).max()
        if k in ("ux", "uy"):
            scale = max(scale, cs)
        out[k] = float(np.abs(got[k] - ref[k]).max() / scale)
    # the velocity figures above are normalised by max(|uhat|, sqrt(max p/rho)); beside them
    # the plain relative L-infinity |got - ref|max / |ref|max and the ratio of the largest
    # speed to that scale (the two agree where the ratio is >= 1)
    for k in ("ux", "uy"):
        umax = float(np.abs(ref[k]).max())
        out[k + "_plain"] = float(np.abs(got[k] - ref[k]).max() / umax) if umax > 0 else None
        out[k + "_max_over_cs"] = umax / cs
    out["steps"] = steps
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="dropletshock2048x1024")
    ap.add_argument("--lattice", default="d2q9", choices=["d2q9", "d2q16", "d3q27"],
                    help="velocity set (D2Q16: the three-launch plane step, no autotuning; "
                         "D3Q27: a 96 x 96 x 64 sphere, its own short line)")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving sample")
    ap.add_argument("--no-autotune", action="store_true", help="use the default launch shape")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64 form, the other workloads / experiments and the FMA peak")
    ap.add_argument("--cpu-steps", type=int, default=0, help="oracle sample steps (0 = auto)")
    ap.add_argument("--serving-config5", action="store_true",
                    help="serve the 256-request mix (sides, temperatures and mixed step counts as "
                         "drawn; FP64 step counts / --fp64-steps-div) and print its summary line")
    ap.add_argument("--fp64-steps-div", type=float, default=10.0)
    ap.add_argument("--serving-rate", type=float, default=0.5, help="Poisson arrivals per second")
    ap.add_argument("--serving-budget-gib", type=float, default=8.0)
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    ws, rank, local = dist_env()

    import torch
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    w = workload(args.workload)

    if args.impl == "reference" and args.lattice == "d3q27":
        # the 3-D oracle on a bounded sample of the 96 x 96 x 64 sphere: one step of 2,000
        # nodes (the whole grid's moments and non-local terms included)
        if rank == 0:
            import numpy as np
            from oracle import core3d
            from paper_2002_09217_gb300 import inputs
            w3 = inputs.droplet3d(n=96, ny=96, nz=64, radius=20.0)
            P3 = core3d.Params3(nx=w3.nx, ny=w3.ny, nz=w3.nz, a=w3.a, b=w3.b, R=w3.R, delta=w3.delta,
                                kappa=w3.kappa, tau=w3.tau, k_cond=w3.k_cond, p_floor=w3.p_floor,
                                tol=1e-12, dt=w3.dt)
            st = core3d.init_state(P3, *w3.fields())
            nodes = np.random.default_rng(3).choice(w3.nodes, 2000, replace=False)
            t0 = time.perf_counter()
            core3d.step_nodes(P3, st, nodes)
            el = time.perf_counter() - t0
            v = len(nodes) / el / 1e6
            import oracle
            line = {"impl": "reference", "metric": "MLUPS", "value": v, "unit": "MLUPS", "n_gpus": ws,
                    "steps": 1, "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                    "dtype": "f64", "data": "synthetic",
                    "config": {"workload": w3.name, "nx": w3.nx, "ny": w3.ny, "nz": w3.nz, "lattice": "d3q27"},
                    "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": oracle.num_threads(), "kind": "oracle",
                                     "sample": "one step of 2,000 sampled nodes of the 96x96x64 sphere (3-D FP64 oracle)"},
                    "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
            print(json.dumps(line), flush=True)
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    if args.impl == "reference":
        if rank == 0:
            # full-grid oracle steps, bounded: a 2048 x 1024 step takes ~10 s on 16 cores
            steps = max(1, min(args.steps, 20 if w.nodes < 100000 else 3))
            res = oracle_mlups(w, steps, args.lattice, warmup=args.warmup)
            line = {"impl": "reference", "metric": "MLUPS", "value": res["value"], "unit": "MLUPS",
                    "n_gpus": ws, "steps": steps, "warmup": args.warmup, "higher_is_better": True,
                    "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                    "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "dt": w.dt, "precision": "fp64",
                               "launch_shape": "n/a (CPU oracle)", "lattice": args.lattice,
                               "l2": "n/a (CPU)", "parallelism": "replicas" if ws > 1 else "single"},
                    "cpu_baseline": {k: res[k] for k in ("value", "unit", "cores", "kind", "sample")},
                    "e2e": {"value": res["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                            "d2h_bytes_per_step": 0}}
            print(json.dumps(line), flush=True)
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    from paper_2002_09217_gb300 import autotune, pond
    torch.cuda.set_device(local)
    if args.serving_config5:
        # the serving configuration: 256 seeded requests, served by footprint admission and
        # continuous batching; then a one-step oracle check of a seeded subset of results
        clocks = ClockSampler(local)
        with clocks:
            summ = serving_run(torch, rank, ws, n_req=256, side_cap=0,
                               steps_scale={"mixed": 1.0, "fp64": 1.0 / args.fp64_steps_div}, tr_min=0.0,
                               rate=args.serving_rate, budget=int(args.serving_budget_gib * 2 ** 30), check=16)
        kept = summ.pop("_kept")
        if rank == 0:
            line = {"metric": "serving sims/s", "value": summ["sims_per_s"], "unit": "sims/s", "n_gpus": ws,
                    "higher_is_better": True, "data": "synthetic", "config": {"workload": "serving256"},
                    "serving": summ, "clocks": clocks.summary()}
            if not args.no_cpu:
                line["accuracy"] = serving_accuracy(pond, kept)
            print(json.dumps(line), flush=True)
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    pk = peaks()
    for prec, iters in (("mixed", 200000), ("fp64", 20000)):
        pk["fma_" + prec] = None
        if not args.no_extras:
            try:
                pk["fma_" + prec] = pond.fma_peak(prec, iters, stream)
            except pond.PondError:
                pass

    if args.lattice == "d3q27":
        # the three-dimensional lattice: its own short line on a 96 x 96 x 64 sphere
        steps = max(1, min(args.steps, 20))
        clocks = ClockSampler(local)
        with clocks:
            r = d3q27_run(pond, torch, stream, args.precision, steps, args.warmup, sm_mhz=pk["sm_max_mhz"])
        nodes = 96 * 96 * 64
        line = {"metric": "MLUPS", "value": ws * r["mlups"], "unit": "MLUPS", "n_gpus": ws, "steps": steps,
                "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
                "config": {"workload": r["workload"], "nx": 96, "ny": 96, "nz": 64, "lattice": "d3q27",
                           "precision": args.precision, "l2": "inputs larger than L2 (170 MB per FP32 buffer)"},
                "frame_search_streams_per_node": r["streams_per_node"], "gpu_launches": 3 * steps,
                "roofline": r["roofline"], "clocks": clocks.summary(),
                "e2e": {"value": ws * r["e2e_mlups"], "unit": "MLUPS", "h2d_bytes_per_step": 5 * nodes * 8 / steps,
                        "d2h_bytes_per_step": 6 * nodes * 8 / steps}}
        if rank == 0:
            print(json.dumps(line), flush=True)
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    def shape_for(prec):
        if args.lattice != "d2q9":
            return {"lattice": args.lattice}
        if args.no_autotune:
            return {}
        best = autotune.tune(w, prec, stream=stream)
        return {"lanes_per_node": best["lanes_per_node"], "tile_x": best["tile_x"]}

    shape = shape_for(args.precision)
    big = state_bytes(w, args.precision) >= 2 * L2_BYTES
    clocks = ClockSampler(local)
    with clocks:
        ms, st, kms = run_form(w, pond, torch, stream, flush, args.precision, args.steps,
                               args.warmup, shape, ws)
    total_ms = sum(ms)
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = ws * w.nodes * args.steps / (total_ms * 1e-3) / 1e6
    its = st["streams"] / max(1, w.nodes * args.steps)

    line = {
        "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        # the mixed form's step computes in FP32 (its EoS and conserved sums in float-float
        # pairs of FP32); the FP64 form in FP64
        "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "dt": w.dt, "precision": args.precision,
                   "launch_shape": shape or "default", "lattice": args.lattice,
                   "l2": ("inputs larger than L2 (%.0f MB per state buffer)" % (state_bytes(w, args.precision) / 1e6)
                          if big else "flushed between timed steps (512 MiB write)"),
                   "parallelism": "replicas" if ws > 1 else "single"},
        "frame_search_streams_per_node": its,
        "gpu_launches": args.steps * (3 if args.lattice == "d2q16" else 1),
        "roofline": roofline(w, args.precision, its, kms, pk, args.lattice, st, w.nodes * args.steps),
        "region_nodes_per_stream": st["region_nodes"] / max(1, st["streams"] - st["pair_streams"]),
        # streams a block runs (its nodes search in lockstep) per node's own streams
        "block_stream_ratio": st["block_streams"] * 16 / max(1, st["streams"]),
        "hbm": {"bytes_per_update": bytes_per_update(args.precision, args.lattice),
                "achieved_gbs": value / ws * 1e6 * bytes_per_update(args.precision, args.lattice) / 1e9,
                "peak_gbs": pk["hbm_gbs"], "peak_src": pk["src"]},
        "clocks": clocks.summary(),
    }
    line["e2e"] = end_to_end(w, pond, torch, stream, args.precision, shape, n_seg=100, reps=5)

    if args.precision == "mixed" and not args.no_extras:
        # the plain FP64 form of the same workload (fewer steps: the FP64 pipes are 1/64)
        shape64 = shape_for("fp64")
        n64 = 30 if w.nodes < 1000000 else 8
        ms64, st64, kms64 = run_form(w, pond, torch, stream, flush, "fp64", n64, 3, shape64, 1)
        its64 = st64["streams"] / max(1, w.nodes * n64)
        line["fp64"] = {"value": w.nodes * n64 / (sum(ms64) * 1e-3) / 1e6, "unit": "MLUPS", "steps": n64,
                        "ms_per_step": sum(ms64) / n64, "launch_shape": shape64 or "default",
                        "frame_search_streams_per_node": its64,
                        "hbm": {"bytes_per_update": bytes_per_update("fp64", args.lattice)},
                        "roofline": roofline(w, "fp64", its64, kms64, pk, args.lattice, st64, w.nodes * n64),
                        "e2e": end_to_end(w, pond, torch, stream, "fp64", shape64, n_seg=10, reps=2)}

    if rank == 0 and not args.no_extras:
        line["other_configs"] = other_configs(pond, torch, stream, pk["sm_max_mhz"], skip=w.name)

    if not args.no_serving:
        serv = serving_sample(torch, rank, ws)
        if rank == 0:
            line["serving"] = serv

    if rank == 0 and not args.no_cpu:
        cpu_steps = args.cpu_steps or max(1, min(40, int(3e5 // w.nodes)))
        res = oracle_mlups(w, cpu_steps, args.lattice)
        line["cpu_baseline"] = {k: res[k] for k in ("value", "unit", "cores", "kind", "sample")}
        # this run's GPU path against the oracle sample (same steps from the same start,
        # every node compared), in the bench's form and in FP64
        line["linf_vs_oracle"] = parity_vs_oracle(w, pond, stream, args.precision, shape, res,
                                                  cpu_steps + 1)
        if args.precision == "mixed" and not args.no_extras and args.lattice == "d2q9":
            line["fp64"]["linf_vs_oracle"] = parity_vs_oracle(w, pond, stream, "fp64", shape_for("fp64"),
                                                              res, cpu_steps + 1)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
