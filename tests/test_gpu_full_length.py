"""Parity at the workloads' own step counts, and how the difference to the FP64 oracle
grows with the number of steps.

- The 2048 x 4 supercritical shock tube for all 5,000 of its steps, element by element,
  in both forms against one oracle run.
- The 512 x 512 droplet after 20,000 steps and the 2048 x 1024 droplet-shock after
  10,000: the GPU runs (mixed form) to one step short of the count, and the last step is
  compared at >= 256 sampled nodes, half of them in interfaces or shock fronts, with the
  oracle stepping those nodes from the GPU's own state.  The FP64 form takes the same
  last step from the same state (set_state into an FP64 context): the full FP64 runs,
  at the FP64 pipe's rate, would take 5 and 10 minutes of GPU time.
- Growth curves on reduced analogues (a 64 x 64 droplet for 4,000 steps, a 128 x 64
  droplet-shock for 2,000): the full fields of both forms against the oracle at every
  500 steps.

Bars: FP64 <= 1e-11, mixed FP32/FP64 <= 1e-5 relative L-infinity per field.
"""
import numpy as np
import pytest

import oracle
from paper_2002_09217_gb300 import inputs

from parity_util import TOL, oracle_run, params_of, rel_linf, sample_nodes, state_fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pond():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2002_09217_gb300 import pond as mod
    mod.load()
    return mod


@pytest.fixture(scope="module")
def tube_oracle():
    w = inputs.shock_tube()
    P, st, stats = oracle_run(w)
    return w, oracle.moments(P, st)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_shocktube2048x4_all_5000_steps(pond, tube_oracle, precision):
    w, ref = tube_oracle
    with pond.from_workload(w, precision=precision) as sim:
        sim.init_fields(*w.fields())
        sim.step(w.steps)
        got = sim.moments()
        st = sim.stats()
    err = rel_linf(got, ref)
    print("shocktube2048x4 %s after %d steps: %s" % (precision, w.steps, err))
    assert st["nonfinite"] == 0
    assert max(err.values()) <= TOL[precision], err


def interface_and_other_nodes(state, nx, ny, count=256, seed=11):
    """Half the sample where the density changes fastest (interfaces, shock fronts),
    half from sample_nodes (corners, edge midpoints, seeded interior)."""
    rho = state[21].reshape(ny, nx)
    gx = np.abs(np.roll(rho, -1, 1) - np.roll(rho, 1, 1))
    gy = np.abs(np.roll(rho, -1, 0) - np.roll(rho, 1, 0))
    g = (gx + gy).reshape(-1)
    steep = np.argsort(g)[::-1][: 8 * count]
    rng = np.random.default_rng(seed)
    pick = set(int(i) for i in rng.choice(steep, count // 2, replace=False))
    for i in sample_nodes(nx, ny, count):
        if len(pick) >= count:
            break
        pick.add(int(i))
    return np.array(sorted(pick), dtype=np.int64)


def last_step_check(pond, w, steps):
    """Mixed run to steps - 1, then the last step in both forms from that state,
    compared at sampled nodes with the oracle's step of those nodes."""
    with pond.from_workload(w, precision="mixed") as sim:
        sim.init_fields(*w.fields())
        sim.step(steps - 1)
        prev = sim.get_state()
        sim.step(1)
        nxt = {"mixed": sim.get_state().reshape(25, -1)}
        st = sim.stats()
    assert st["nonfinite"] == 0, st
    with pond.from_workload(w, precision="fp64") as sim:
        sim.set_state(prev)
        sim.step(1)
        nxt["fp64"] = sim.get_state().reshape(25, -1)
    nodes = interface_and_other_nodes(prev.reshape(25, -1), w.nx, w.ny)
    out = {}
    for prec in ("mixed", "fp64"):
        P = params_of(w, tol=(1e-12 if prec == "fp64" else 1e-6))
        rows = oracle.step_nodes(P, prev, nodes)
        out[prec] = rel_linf(state_fields(P, nxt[prec][:, nodes].T), state_fields(P, rows))
    return out, len(nodes)


def test_droplet512_last_of_20000_steps(pond):
    w = inputs.droplet()
    err, n = last_step_check(pond, w, w.steps)
    print("droplet512x512 step %d at %d nodes: %s" % (w.steps, n, err))
    assert n >= 256
    for prec in ("mixed", "fp64"):
        assert max(err[prec].values()) <= TOL[prec], (prec, err[prec])


def test_dropletshock2048x1024_last_of_10000_steps(pond):
    w = inputs.droplet_shock()
    err, n = last_step_check(pond, w, w.steps)
    print("dropletshock2048x1024 step %d at %d nodes: %s" % (w.steps, n, err))
    assert n >= 256
    for prec in ("mixed", "fp64"):
        assert max(err[prec].values()) <= TOL[prec], (prec, err[prec])


def growth_curve(pond, w, every):
    """Full-field rel. L-infinity of both forms against the oracle every `every` steps."""
    P = params_of(w)
    ref_state = oracle.init_state(P, *w.fields())
    sims = {prec: pond.from_workload(w, precision=prec) for prec in ("fp64", "mixed")}
    curve = []
    try:
        for s in sims.values():
            s.init_fields(*w.fields())
        done = 0
        while done < w.steps:
            n = min(every, w.steps - done)
            ref_state = oracle.step(P, ref_state, n)
            done += n
            ref = oracle.moments(P, ref_state)
            row = {"steps": done}
            for prec, s in sims.items():
                s.step(n)
                row[prec] = max(rel_linf(s.moments(), ref).values())
            curve.append(row)
    finally:
        for s in sims.values():
            s.close()
    return curve


@pytest.mark.parametrize("case", ["droplet64", "dropletshock128x64"])
def test_growth_of_the_difference_on_reduced_analogues(pond, case):
    if case == "droplet64":
        w = inputs.droplet(n=64, Tr=0.85, radius=10.0, steps=4000)
    else:
        w = inputs.droplet_shock(nx=128, ny=64, Tr=0.8, radius=10.0, xc=60.0, x_shock=25.0, steps=2000)
    curve = growth_curve(pond, w, 500)
    for row in curve:
        print("%s %s" % (case, row))
    final = curve[-1]
    assert final["fp64"] <= TOL["fp64"], curve
    assert final["mixed"] <= TOL["mixed"], curve
