"""Continuous-batching serving loop for PonD simulation requests.

Requests (``inputs.Request``) arrive over time.  The server admits an arrived request
when the device memory it needs fits the budget, initialises it on the GPU and adds it to
the running batch of its precision.  Each precision has its own batch on its own CUDA
stream, the mixed one at higher priority, so the fast mixed-precision requests do not
wait for the FP64 ones (which run at the FP64 pipe's 1/64 rate on GB300) and the two
groups' kernels overlap on the device.  Whenever a batch's previous chunk of steps has
finished (``pond_batch_poll``, which does not block), the server retires its requests that
reached their step count (fields back to the host), frees their memory, admits more and
launches the batch's next chunk with ``pond_batch_step`` (one launch per time step and
kernel group, graph-replayed).  Admission is checked twice: against an estimate before the
simulation's memory is taken, and by the batch itself (``pond_batch_set_budget``), which
refuses a member whose exact device bytes would exceed the budget.
Latency of a request = completion time - arrival time.

The per-node arithmetic does not depend on the batch, so a request's result is the same
stepped alone or in the mix (checked by the tests).
"""
from __future__ import annotations

import dataclasses
import heapq
import time

import numpy as np

from . import inputs, pond


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    completed: float
    steps: int
    nodes: int
    precision: str
    fields: dict | None
    status: dict
    state: object = None      # the final state (25 planes) when the server keeps it
    workload: object = None   # the request's inputs.Workload

    @property
    def latency(self) -> float:
        return self.completed - self.arrival


def footprint_bytes(nodes: int, precision: str) -> int:
    """Estimated device bytes of one D2Q9 simulation before it is created: two state
    buffers of 32-value records, a 6-plane FP64 staging buffer and the reduction partials
    and counters (as pond_create allocates).  Once created, the server charges the
    library's exact figure (pond_device_bytes) instead."""
    esize = 4 if precision == "mixed" else 8
    blocks = min(1024, max(1, (nodes + 255) // 256))
    return 2 * 32 * nodes * esize + 6 * nodes * 8 + (8 * blocks + 8) * 8 + 4096


class Server:
    """Admits requests by device-memory footprint and steps them in one batch."""

    PRECISIONS = ("mixed", "fp64")

    def __init__(self, hbm_budget: int, chunk: int = 50, max_resident: int = 64,
                 keep_fields: bool = True, keep_state: bool = False):
        import torch
        self.torch = torch
        self.budget = int(hbm_budget)
        self.chunk = int(chunk)
        self.max_resident = int(max_resident)
        self.keep_fields = keep_fields
        # also return the full final state of every request (True) or of the requests
        # whose ids are in a given set
        self.keep_state = keep_state
        self.peak_bytes = 0
        # the mixed stream at higher priority: an FP64 group launch holds tens of thousands
        # of slow blocks, and the block scheduler would otherwise dispatch them ahead of the
        # mixed group's
        self.streams = {"mixed": torch.cuda.Stream(priority=-1), "fp64": torch.cuda.Stream(priority=0)}
        self.batches = {k: pond.Batch(self.streams[k]) for k in self.PRECISIONS}
        for b in self.batches.values():
            b.set_budget(self.budget)
        self.refused = 0          # admissions the batch refused after creation (budget)

    def _start(self, req, now, used):
        """Create, initialise and batch a request's simulation; None if the exact device
        bytes (pond_device_bytes) or the batch's own budget check refuse it while other
        requests hold memory."""
        w = inputs.request_workload(req)
        sim = pond.from_workload(w, precision=req.precision, stream=self.streams[req.precision])
        nbytes = sim.device_bytes()
        if used > 0 and used + nbytes > self.budget:
            sim.close()
            return None
        sim.init_fields(*w.fields())
        try:
            self.batches[req.precision].add(sim)
        except pond.PondError as e:
            sim.close()
            if e.status != 2:
                raise
            return None
        return {"req": req, "sim": sim, "left": req.steps, "admitted": now, "nodes": w.nodes,
                "bytes": nbytes, "w": w}

    def run(self, requests, time_scale: float = 1.0) -> list[Result]:
        """Serve the requests; arrival times are in seconds after the start, multiplied
        by time_scale.  Returns one Result per request, in completion order."""
        torch = self.torch
        pending = [(r.arrival * time_scale, r.rid, r) for r in requests]
        heapq.heapify(pending)
        waiting = []                                   # arrived, not yet admitted (FIFO)
        running = {k: [] for k in self.PRECISIONS}
        inflight = {k: False for k in self.PRECISIONS}  # a batch's last chunk may still run
        used = 0
        results = []
        t0 = time.perf_counter()
        self.used_seconds = 0.0        # integral of resident bytes over time (byte-seconds)
        t_prev = t0
        while pending or waiting or any(running.values()):
            t_now = time.perf_counter()
            self.used_seconds += used * (t_now - t_prev)
            t_prev = t_now
            now = t_now - t0
            while pending and pending[0][0] <= now:
                waiting.append(heapq.heappop(pending)[2])
            busy = False
            for k in self.PRECISIONS:
                if inflight[k] and not self.batches[k].poll():
                    busy = True
                    continue
                inflight[k] = False
                # retire what the finished chunk completed (its stream is idle)
                for it in [it for it in running[k] if it["left"] == 0]:
                    sim = it["sim"]
                    self.batches[k].remove(sim)
                    try:
                        fields = sim.moments() if self.keep_fields else None
                    except pond.PondError as e:
                        if e.status != 6:
                            raise
                        fields = None            # a diverged request: reported, not returned
                    status = sim.stats()
                    status["flags"] = [f for f, _ in sim.flags]
                    ks = self.keep_state
                    if ks is True or (ks and it["req"].rid in ks):
                        it["state"] = sim.get_state()
                    sim.close()
                    req = it["req"]
                    results.append(Result(req.rid, req.arrival * time_scale, it["admitted"],
                                          time.perf_counter() - t0, req.steps, it["nodes"],
                                          req.precision, fields, status, it.get("state"), it["w"]))
                    used -= it["bytes"]
                    running[k].remove(it)
            # admission by footprint, in arrival order: the estimate first (nothing is
            # allocated for a request that cannot fit), then the exact bytes once created;
            # a request larger than the budget runs when nothing else is resident
            while waiting and sum(len(v) for v in running.values()) < self.max_resident:
                req = waiting[0]
                need = footprint_bytes(req.side * req.side, req.precision)
                if used + need > self.budget and any(running.values()):
                    break
                k = req.precision
                if inflight[k]:
                    break                  # its batch is stepping; it joins after the chunk
                item = self._start(req, time.perf_counter() - t0, used)
                if item is None:
                    self.refused += 1
                    if not any(running.values()):
                        raise RuntimeError("request %d cannot be admitted with nothing resident" % req.rid)
                    break                  # over the budget: wait for memory to free up
                waiting.pop(0)
                running[k].append(item)
                used += item["bytes"]
                self.peak_bytes = max(self.peak_bytes, used)
            for k in self.PRECISIONS:
                if not inflight[k] and running[k]:
                    n = min(self.chunk, min(it["left"] for it in running[k]))
                    self.batches[k].step(n)
                    for it in running[k]:
                        it["left"] -= n
                    inflight[k] = True
                    busy = True
            if not busy and not waiting:
                if pending:
                    time.sleep(max(0.0, min(0.01, pending[0][0] - (time.perf_counter() - t0))))
            elif busy:
                time.sleep(0.0002)
        for k in self.PRECISIONS:
            self.batches[k].synchronize()
        return results

    def close(self):
        for b in self.batches.values():
            b.close()


def summarize(results: list[Result], wall: float) -> dict:
    lat = np.array([r.latency for r in results])
    nodes = sum(r.nodes * r.steps for r in results)
    by = {}
    for prec in sorted({r.precision for r in results}):
        l = np.array([r.latency for r in results if r.precision == prec])
        by[prec] = {"requests": int(l.size), "p50_latency_s": float(np.percentile(l, 50)),
                    "p99_latency_s": float(np.percentile(l, 99))}
    return {"requests": len(results), "sims_per_s": len(results) / wall,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "node_updates": int(nodes), "mlups": nodes / wall / 1e6, "wall_s": wall,
            "by_precision": by}
