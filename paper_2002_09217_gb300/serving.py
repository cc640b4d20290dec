"""Continuous-batching serving loop for PonD simulation requests.

Requests (``inputs.Request``) arrive over time.  The server admits an arrived request
when the device memory it needs fits the budget, initialises it on the GPU and adds it to
the running batch; every scheduler turn advances all resident simulations together with
``pond_batch_step`` (one launch per time step and kernel group, graph-replayed), retires
those that reached their step count (fields back to the host), frees their memory and
admits more.  Requests that arrive while others run join at the next turn, so their work
overlaps on the device.  Latency of a request = completion time - arrival time.

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

    @property
    def latency(self) -> float:
        return self.completed - self.arrival


def footprint_bytes(nodes: int, precision: str) -> int:
    """Device bytes of one simulation: two state buffers of 32-value records, a 5-plane
    FP64 staging buffer and small reduction/counter blocks (as pond_create allocates)."""
    esize = 4 if precision == "mixed" else 8
    return 2 * 32 * nodes * esize + 5 * nodes * 8 + 65536


class Server:
    """Admits requests by device-memory footprint and steps them in one batch."""

    def __init__(self, hbm_budget: int, chunk: int = 50, max_resident: int = 64,
                 keep_fields: bool = True):
        import torch
        self.torch = torch
        self.budget = int(hbm_budget)
        self.chunk = int(chunk)
        self.max_resident = int(max_resident)
        self.keep_fields = keep_fields
        self.stream = torch.cuda.Stream()
        self.batch = pond.Batch(self.stream)

    def _start(self, req, now):
        w = inputs.request_workload(req)
        sim = pond.from_workload(w, precision=req.precision, stream=self.stream)
        sim.init_fields(*w.fields())
        self.batch.add(sim)
        return {"req": req, "sim": sim, "left": req.steps, "admitted": now, "nodes": w.nodes,
                "bytes": footprint_bytes(w.nodes, req.precision)}

    def run(self, requests, time_scale: float = 1.0) -> list[Result]:
        """Serve the requests; arrival times are in seconds after the start, multiplied
        by time_scale.  Returns one Result per request, in completion order."""
        pending = [(r.arrival * time_scale, r.rid, r) for r in requests]
        heapq.heapify(pending)
        waiting = []          # arrived, not yet admitted (FIFO)
        running = []
        used = 0
        results = []
        t0 = time.perf_counter()
        while pending or waiting or running:
            now = time.perf_counter() - t0
            while pending and pending[0][0] <= now:
                waiting.append(heapq.heappop(pending)[2])
            # admission by footprint, in arrival order
            while waiting and len(running) < self.max_resident:
                req = waiting[0]
                need = footprint_bytes(req.side * req.side, req.precision)
                if used + need > self.budget and running:
                    break
                waiting.pop(0)
                item = self._start(req, now)
                running.append(item)
                used += item["bytes"]
            if not running:
                if pending:
                    time.sleep(max(0.0, min(0.01, pending[0][0] - now)))
                continue
            n = min(self.chunk, min(it["left"] for it in running))
            self.batch.step(n)
            for it in running:
                it["left"] -= n
            done = [it for it in running if it["left"] == 0]
            if done:
                self.batch.synchronize()
                for it in done:
                    sim = it["sim"]
                    self.batch.remove(sim)
                    fields = sim.moments() if self.keep_fields else None
                    status = sim.stats()
                    sim.close()
                    req = it["req"]
                    results.append(Result(req.rid, req.arrival * time_scale, it["admitted"],
                                          time.perf_counter() - t0, req.steps, it["nodes"],
                                          req.precision, fields, status))
                    used -= it["bytes"]
                    running.remove(it)
        self.batch.synchronize()
        return results

    def close(self):
        self.batch.close()


def summarize(results: list[Result], wall: float) -> dict:
    lat = np.array([r.latency for r in results])
    nodes = sum(r.nodes * r.steps for r in results)
    return {"requests": len(results), "sims_per_s": len(results) / wall,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "node_updates": int(nodes), "mlups": nodes / wall / 1e6, "wall_s": wall}
