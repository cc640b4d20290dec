"""Benchmark of the PonD van der Waals time step on GB300.

Workload (default): the supercritical real-gas shock tube, 2048 x 4 nodes,
T = 1.1 T_cr, density ratio 4 with a tanh step of width 4, zero-gradient ends in x.
One bench "step" = one time step of the whole hot path (non-local terms, frame
search with streaming, collision) over the grid.  Metric: MLUPS (million node
updates per second) in the mixed FP32/FP64 form; the plain FP64 form is reported
beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
                  [--impl reference] [--no-cpu]

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events on the
simulation's stream, with the L2 flushed (a 512 MiB buffer written) between timed
steps because the state (a few MB) is far smaller than L2.  Under torchrun (N > 1)
each rank runs an independent replica (the workload does not shard) and the
slowest rank's time counts.
"""
from __future__ import annotations

import argparse
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


def bytes_per_update(precision: str) -> int:
    # state read once (f, g, gauge, rho, T: 23 values) + written once (25 values)
    return 48 * (4 if precision == "mixed" else 8)


def flops_per_stream() -> int:
    """Algorithmic FLOPs of one streaming pass of one node (the kernel's formula):
    per direction: departure point + two cubic Lagrange bases (24), and per stencil
    node: sqrt(theta_n) + 6 transfer coefficients (4 each) + f and g components
    (2 x (9 + 3) FMA) + 2 interpolation FMA => 16 x (1 + 24 + 48 + 4) = 1232."""
    return 9 * (24 + 16 * (1 + 24 + 48 + 4))


FLOPS_PER_ITER_EXTRA = 60        # moments and residual per frame-search pass
FLOPS_COLLIDE = 700              # equilibria, sources and the 3x3 (x) 3x3 map of g


def oracle_mlups(w, steps: int) -> dict:
    import numpy as np  # noqa: F401
    import oracle
    P = oracle.Params(nx=w.nx, ny=w.ny, bc_x=w.bc_x, bc_y=w.bc_y, a=w.a, b=w.b, R=w.R,
                      delta=w.delta, kappa=w.kappa, tau=w.tau, dt=w.dt, k_cond=w.k_cond,
                      p_floor=w.p_floor, tol=1e-12, max_iter=20)
    st = oracle.init_state(P, *w.fields())
    st = oracle.step(P, st, 1)          # warm-up (page-in, thread pool)
    t0 = time.perf_counter()
    st = oracle.step(P, st, steps)
    dt = time.perf_counter() - t0
    return {"value": w.nodes * steps / dt / 1e6, "unit": "MLUPS", "cores": oracle.num_threads(),
            "kind": "oracle", "seconds": dt,
            "sample": "%d time steps of the full %dx%d grid (FP64 oracle, OpenMP over nodes)"
                      % (steps, w.nx, w.ny), "state": st, "params": P}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="shocktube2048x4")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-steps", type=int, default=0, help="oracle sample steps (0 = auto)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    ws, rank, local = dist_env()

    import torch
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    w = workload(args.workload)

    if args.impl == "reference":
        if rank == 0:
            steps = max(1, min(args.steps, 20))
            res = oracle_mlups(w, steps)
            line = {"impl": "reference", "metric": "MLUPS", "value": res["value"], "unit": "MLUPS",
                    "n_gpus": ws, "steps": steps, "warmup": 1, "higher_is_better": True,
                    "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                    "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "dt": w.dt},
                    "cpu_baseline": {k: res[k] for k in ("value", "unit", "cores", "kind", "sample")},
                    "e2e": {"value": res["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                            "d2h_bytes_per_step": 0}}
            print(json.dumps(line), flush=True)
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    from paper_2002_09217_gb300 import pond
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed_run(precision: str, steps: int, warmup: int):
        sim = pond.from_workload(w, precision=precision, stream=stream)
        dev_fields = [torch.tensor(a, device=dev, dtype=torch.float64) for a in w.fields()]
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
        with torch.cuda.stream(stream):
            for k in range(steps):
                flush.fill_(float(k))
                evs[k][0].record(stream)
                sim.step(1)
                evs[k][1].record(stream)
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in evs]
        st = sim.stats()
        return sim, ms, st

    clocks = ClockSampler(local)
    with clocks:
        sim, ms, st = timed_run(args.precision, args.steps, args.warmup)
    total_ms = sum(ms)
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = ws * w.nodes * args.steps / (total_ms * 1e-3) / 1e6
    its = st["streams"] / max(1, w.nodes * args.steps)

    # per-kernel time of the dominant kernel (k_step) from events around one launch:
    # the step is 3 launches; time the frame-search kernel alone via a second sim call
    kstep_ms = kernel_time(sim, flush, stream, torch, reps=min(args.steps, 50))

    # end to end through the public API with host buffers: init from pinned host arrays,
    # n_seg time steps, moments back to host, per call
    e2e = end_to_end(w, pond, torch, stream, args.precision, n_seg=100, reps=5)

    pk = peaks()
    sm_mhz = clocks.summary().get("sm_mhz") or pk["sm_max_mhz"]
    fl_update = its * (flops_per_stream() + FLOPS_PER_ITER_EXTRA) + FLOPS_COLLIDE
    achieved_tf = w.nodes * fl_update / (kstep_ms * 1e-3) / 1e12
    peak_tf = alu_peak_tflops(args.precision, pk["sm_max_mhz"])

    line = {
        "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "dt": w.dt, "precision": args.precision,
                   "l2": "flushed between timed steps (512 MiB write)",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "frame_search_streams_per_node": its,
        "gpu_launches": args.steps,
        "roofline": {"bound": "alu", "kernel": "k_pond_step", "achieved": achieved_tf, "peak": peak_tf,
                     "unit": "TFLOP/s", "frac": achieved_tf / peak_tf, "traffic": None,
                     "peak_src": "FP32 %s: 152 SM x 128 lanes x 2 x %.0f MHz" % (
                         "" if args.precision == "mixed" else "/64 (FP64)", pk["sm_max_mhz"]),
                     "flops_per_update": fl_update, "kernel_ms": kstep_ms},
        "hbm": {"bytes_per_update": bytes_per_update(args.precision),
                "achieved_gbs": value * 1e6 * bytes_per_update(args.precision) / 1e9,
                "peak_gbs": pk["hbm_gbs"], "peak_src": pk["src"]},
        "clocks": clocks.summary(),
        "e2e": e2e,
    }
    if rank == 0 and not args.no_cpu:
        cpu_steps = args.cpu_steps or max(1, min(40, int(3e5 // w.nodes)))
        res = oracle_mlups(w, cpu_steps)
        line["cpu_baseline"] = {k: res[k] for k in ("value", "unit", "cores", "kind", "sample")}
        # parity of this run's GPU path against the oracle sample (same steps, fresh start)
        line["linf_vs_oracle"] = parity_vs_oracle(w, pond, torch, stream, args.precision, res, cpu_steps + 1)
    sim.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def kernel_time(sim, flush, stream, torch, reps: int) -> float:
    """Average duration of the fused step kernel, timed by the library itself with CUDA
    events on the context stream, L2 flushed before each launch."""
    acc = 0.0
    for k in range(reps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
        acc += sim.step_timed() / reps
    return acc


def end_to_end(w, pond, torch, stream, precision, n_seg: int, reps: int) -> dict:
    import numpy as np
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in w.fields()]
    outs = {k: torch.empty((w.ny, w.nx), dtype=torch.float64).pin_memory() for k in ("rho", "ux", "uy", "T", "p")}
    sim = pond.from_workload(w, precision=precision, stream=stream)
    times = []
    for r in range(reps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.init_fields(*[h.numpy() for h in host])
        sim.step(n_seg)
        m = sim.moments()
        for k in outs:
            outs[k].numpy()[...] = m[k]
        times.append(time.perf_counter() - t0)
    sim.close()
    t = statistics.median(times[1:])
    return {"value": w.nodes * n_seg / t / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": 4 * w.nodes * 8 / n_seg, "d2h_bytes_per_step": 5 * w.nodes * 8 / n_seg,
            "segment_steps": n_seg,
            "note": "per call: init from pinned host (4 fields), %d steps, 5 fields back to host" % n_seg}


def parity_vs_oracle(w, pond, torch, stream, precision, res, steps) -> dict:
    import numpy as np
    import oracle
    ref = oracle.moments(res["params"], res["state"])
    sim = pond.from_workload(w, precision=precision, stream=stream)
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
    out["steps"] = steps
    return out


if __name__ == "__main__":
    main()
