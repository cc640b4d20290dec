"""Batched stepping and the continuous-batching server: every simulation's result must be
the same stepped alone or inside a batch whose membership changes while it runs."""
import dataclasses

import numpy as np
import pytest

from paper_2002_09217_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pond():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2002_09217_gb300 import pond as mod
    mod.load()
    return mod


def _cases():
    return [
        (inputs.droplet(n=40, ny=36, Tr=0.9, radius=8.0), "mixed", {}),
        (inputs.slab(nx=64, ny=5, Tr=0.9), "mixed", {"lanes_per_node": 16}),
        (inputs.shock_in_vapour(n=32, Tr=0.8, Mach=1.5), "fp64", {}),
        (inputs.shock_tube(nx=96, ny=3, width=2.0), "mixed", {"tile_x": 8}),
        (inputs.droplet(n=24, ny=20, Tr=0.85, radius=5.0), "fp64", {"tile_x": 16}),
    ]


def _alone(pond, w, prec, kw, steps):
    with pond.from_workload(w, precision=prec, **kw) as sim:
        sim.init_fields(*w.fields())
        sim.step(steps)
        return sim.moments()


def test_batch_with_changing_membership_equals_alone(pond):
    cases = _cases()
    batch = pond.Batch()
    sims = []
    for w, prec, kw in cases:
        s = pond.from_workload(w, precision=prec, **kw)
        s.init_fields(*w.fields())
        sims.append(s)
    steps = [0] * len(cases)
    # join two, step, join the rest, step, let one leave, step, let it come back, step
    for k in (0, 1):
        batch.add(sims[k])
    batch.step(7)
    for k in (0, 1):
        steps[k] += 7
    for k in (2, 3, 4):
        batch.add(sims[k])
    batch.step(5)
    for k in range(5):
        steps[k] += 5
    batch.remove(sims[1])
    batch.step(4)
    for k in (0, 2, 3, 4):
        steps[k] += 4
    batch.add(sims[1])
    batch.step(3)
    for k in range(5):
        steps[k] += 3
    batch.synchronize()
    with pytest.raises(pond.PondError):
        sims[0].step(1)          # a batched context is stepped by its batch only
    for (w, prec, kw), sim, n in zip(cases, sims, steps):
        got = sim.moments()
        ref = _alone(pond, w, prec, kw, n)
        for key in ref:
            np.testing.assert_array_equal(got[key], ref[key], err_msg="%s %s" % (w.name, key))
    batch.close()
    for s in sims:
        s.close()


def test_serving_results_equal_alone(pond):
    from paper_2002_09217_gb300 import serving
    reqs = inputs.serving_requests(n=10, rate=200.0, seed=77)
    # small and short requests so that the FP64 ones finish quickly
    reqs = [dataclasses.replace(r, side=min(r.side, 48), steps=20 + (r.steps % 40),
                                T_r=max(r.T_r, 0.8)) for r in reqs]
    server = serving.Server(hbm_budget=64 << 20, chunk=7)
    results = server.run(reqs)
    server.close()
    assert sorted(r.rid for r in results) == [r.rid for r in reqs]
    by_id = {r.rid: r for r in reqs}
    for res in results:
        req = by_id[res.rid]
        w = inputs.request_workload(req)
        ref = _alone(pond, w, req.precision, {}, req.steps)
        for key in ref:
            np.testing.assert_array_equal(res.fields[key], ref[key], err_msg="request %d %s" % (res.rid, key))
        assert res.latency >= 0.0
    summary = serving.summarize(results, max(r.completed for r in results))
    assert summary["requests"] == len(reqs) and summary["p99_latency_s"] >= summary["p50_latency_s"]


def test_batch_mixing_equations_of_state_equals_alone(pond):
    """One batch group holding a van der Waals, an isothermal Dieterici, a double-well and
    a non-classical (delta = 0.0125) simulation: each uses its own parameters from the
    work list, so each result equals its alone run bit for bit."""
    cases = [
        (inputs.droplet(n=32, ny=24, Tr=0.9, radius=6.0), {}),
        (inputs.dieterici_slab(0.8, nx=48, ny=4, steps=0), {}),
        (inputs.simplified_eos("slab", nx=40, ny=4, steps=0), {}),
        (dataclasses.replace(inputs.nonclassical_tube("fig4", nx=64, ny=2), steps=0), {}),
    ]
    steps = 9
    batch = pond.Batch()
    sims = []
    for w, kw in cases:
        s = pond.from_workload(w, precision="mixed", **kw)
        s.init_fields(*w.fields())
        batch.add(s)
        sims.append(s)
    batch.step(steps)
    batch.synchronize()
    for (w, kw), sim in zip(cases, sims):
        got = sim.moments()
        ref = _alone(pond, w, "mixed", kw, steps)
        for key in ref:
            np.testing.assert_array_equal(got[key], ref[key], err_msg="%s %s" % (w.name, key))
    batch.close()
    for s in sims:
        s.close()


def test_batch_with_d2q16_members_equals_alone(pond):
    """D2Q16 simulations (their own three launches on the batch stream, inside the batch's
    graph) next to a D2Q9 group, with one leaving and rejoining between odd step counts:
    each equals its alone run bit for bit."""
    cases = [
        (inputs.droplet(n=40, ny=28, Tr=0.9, radius=6.0), "mixed", {"lattice": "d2q16"}),
        (inputs.slab(nx=48, ny=5, Tr=0.9), "fp64", {"lattice": "d2q16"}),
        (inputs.droplet(n=32, ny=24, Tr=0.9, radius=6.0), "mixed", {}),
    ]
    batch = pond.Batch()
    sims = []
    for w, prec, kw in cases:
        s = pond.from_workload(w, precision=prec, **kw)
        s.init_fields(*w.fields())
        batch.add(s)
        sims.append(s)
    steps = [5, 5, 5]
    batch.step(5)
    batch.remove(sims[0])
    batch.step(4)
    steps[1] += 4
    steps[2] += 4
    batch.add(sims[0])
    batch.step(3)
    steps = [n + 3 for n in steps]
    batch.synchronize()
    for (w, prec, kw), sim, n in zip(cases, sims, steps):
        got = sim.moments()
        ref = _alone(pond, w, prec, kw, n)
        for key in ref:
            np.testing.assert_array_equal(got[key], ref[key], err_msg="%s %s %s" % (w.name, kw, key))
    batch.close()
    for s in sims:
        s.close()


def test_served_states_pass_a_one_step_oracle_check(pond):
    """Accuracy of served results: the final states the server returns (mixed and FP64
    requests of the seeded mix, temperatures as drawn, 0.70..0.95) are stepped once more
    on the GPU and by the oracle at sampled nodes; each stays within its form's bar."""
    import oracle
    from parity_util import TOL, params_of, rel_linf, sample_nodes, state_fields
    from paper_2002_09217_gb300 import serving
    reqs = inputs.serving_requests(n=8, rate=200.0, seed=91)
    reqs = [dataclasses.replace(r, side=min(r.side, 64), steps=30 + (r.steps % 50)) for r in reqs]
    server = serving.Server(hbm_budget=256 << 20, chunk=11, keep_fields=False, keep_state=True)
    results = server.run(reqs)
    server.close()
    assert len(results) == len(reqs)
    precs = set()
    for res in results:
        w = res.workload
        assert np.isfinite(res.state).all(), res.rid
        with pond.from_workload(w, precision=res.precision) as sim:
            sim.set_state(res.state)
            sim.step(1)
            nxt = sim.get_state().reshape(25, -1)
        P = params_of(w, tol=(1e-12 if res.precision == "fp64" else 1e-6))
        nodes = sample_nodes(w.nx, w.ny, 48)
        rows = oracle.step_nodes(P, res.state, nodes)
        err = rel_linf(state_fields(P, nxt[:, nodes].T), state_fields(P, rows))
        assert max(err.values()) <= TOL[res.precision], (res.rid, res.precision, err)
        precs.add(res.precision)
    assert precs == {"mixed", "fp64"}
