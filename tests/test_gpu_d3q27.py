"""D3Q27 GPU path (libpond with lattice POND_D3Q27, through its C ABI) against the 3-D
FP64 oracle: element by element on small 3-D grids (ragged 32 x 4 patches, the
128 x 1 strips of grids of fewer than four rows, zero-gradient z ends, a single node, a
moving fluid), conservation sums and the full state, checkpoint/resume, and one-step
checks at sampled nodes of a 96 x 96 x 64 droplet from the GPU's own state.  Bars as on
D2Q9: FP64 <= 1e-11, mixed <= 1e-5 relative L-infinity per field."""
import dataclasses

import numpy as np
import pytest

from oracle import core3d as o3
from paper_2002_09217_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-11, "mixed": 1e-5}
FIELDS = ("rho", "ux", "uy", "uz", "T", "p")


@pytest.fixture(scope="module")
def pond():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2002_09217_gb300 import pond as mod
    mod.load()
    return mod


def params3(w, **over):
    kw = dict(nx=w.nx, ny=w.ny, nz=w.nz, bc_x=w.bc_x, bc_y=w.bc_y, bc_z=w.bc_z, a=w.a, b=w.b, R=w.R,
              delta=w.delta, kappa=w.kappa, tau=w.tau, k_cond=w.k_cond, p_floor=w.p_floor, tol=1e-12,
              max_iter=20, dt=w.dt)
    kw.update(over)
    return o3.Params3(**kw)


def rel_err(got, ref):
    out = {}
    cs = np.sqrt(np.max(np.abs(ref["p"] / ref["rho"])))
    for k in FIELDS:
        scale = np.abs(ref[k]).max()
        if k in ("ux", "uy", "uz"):
            scale = max(scale, cs)
        out[k] = float(np.abs(np.asarray(got[k]) - ref[k]).max() / scale)
    return out


def sim_of(pond, w, precision):
    return pond.Simulation(w.nx, w.ny, **inputs.from_workload3(w, precision))


def moving(w, amp=0.03):
    z, y, x = np.meshgrid(np.arange(w.nz), np.arange(w.ny), np.arange(w.nx), indexing="ij")
    ux = amp * np.sin(2 * np.pi * (y + 0.5) / w.ny)
    uy = amp * np.cos(2 * np.pi * (z + 0.5) / w.nz)
    uz = amp * np.sin(2 * np.pi * (x + 0.5) / w.nx)
    return dataclasses.replace(w, ux=ux, uy=uy, uz=uz)


def cases():
    yield "droplet16", inputs.droplet3d(n=16, radius=4.0, steps=5)
    yield "droplet_ragged33x6x5", inputs.droplet3d(n=33, ny=6, nz=5, radius=2.0, steps=4)
    yield "strip40x2x3_zerograd_z", inputs.droplet3d(n=40, ny=2, nz=3, radius=3.0, bc_z=1, steps=4)
    yield "moving12x10x8", moving(inputs.droplet3d(n=12, ny=10, nz=8, radius=3.0, steps=5))
    yield "single_node", inputs.droplet3d(n=1, radius=0.5, steps=3)
    yield "hot_bump10x8x6_wide_regions", wide_region_bump()


def wide_region_bump():
    """A 10 x 8 x 6 droplet's density field at three times its temperature (2.55 T_cr) with
    dt = 1: sqrt(theta / T_L) dt up to 1.11, so that about half of the nodes have departure
    floors spread over three nodes (regions wider than 6) and take the per-pair stream."""
    w = inputs.droplet3d(n=10, ny=8, nz=6, radius=3.0, steps=4)
    return dataclasses.replace(w, name="hot_bump10x8x6_dt1", dt=1.0, T=w.T * 3.0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", [c[0] for c in cases()])
def test_small_grids_match_oracle(pond, case, precision):
    w = dict(cases())[case]
    P = params3(w)
    stats = {}
    ref = o3.moments(P, o3.step(P, o3.init_state(P, *w.fields()), w.steps, stats))
    with sim_of(pond, w, precision) as sim:
        sim.init_fields(w.rho, w.ux, w.uy, w.T, uz=w.uz)
        sim.step(w.steps)
        got = sim.moments()
        st = sim.stats()
    err = rel_err(got, ref)
    assert max(err.values()) <= TOL[precision], err
    assert st["nonfinite"] == 0
    if precision == "fp64":
        assert abs(st["streams"] - stats["streams"]) <= 0.01 * stats["streams"] + 2


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_region_and_pair_streams_are_both_taken(pond, precision):
    """Every stream of a usual workload (|v| dt < 1) takes the region stream over at most
    6 x 6 x 6 nodes; the hot bump sends streams down both paths."""
    for w, both in ((inputs.droplet3d(n=16, radius=4.0, steps=3), False), (wide_region_bump(), True)):
        with sim_of(pond, w, precision) as sim:
            sim.init_fields(w.rho, w.ux, w.uy, w.T, uz=w.uz)
            sim.step(w.steps)
            st = sim.stats()
        if both:
            assert 0 < st["pair_streams"] < st["streams"], st
            assert st["region_nodes"] > 0
        else:
            assert st["pair_streams"] == 0
            assert 63 * st["streams"] <= st["region_nodes"] <= 216 * st["streams"], st


def test_full_state_and_conservation_sums_match_oracle(pond):
    w = moving(inputs.droplet3d(n=12, ny=10, nz=8, radius=3.0, steps=4))
    P = params3(w)
    st = o3.step(P, o3.init_state(P, *w.fields()), w.steps)
    with sim_of(pond, w, "fp64") as sim:
        sim.init_fields(w.rho, w.ux, w.uy, w.T, uz=w.uz)
        sim.step(w.steps)
        got = sim.get_state()
        sums = sim.conservation()
    assert got.shape == st.shape == (63, 8, 10, 12)
    scale = np.abs(st).reshape(63, -1).max(axis=1)
    scale[scale == 0] = 1.0
    assert (np.abs(got - st).reshape(63, -1).max(axis=1) / scale).max() <= 1e-11
    L = o3.PL
    rho = st[L["rho"]]
    want = [rho.sum(), (rho * st[L["uhx"]]).sum(), (rho * st[L["uhy"]]).sum(), 0.5 * st[L["g"]:L["g"] + 27].sum()]
    np.testing.assert_allclose(sums, want, rtol=1e-11, atol=1e-11 * abs(want[0]))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_checkpoint_resume(pond, precision):
    w = inputs.droplet3d(n=20, ny=16, nz=12, radius=4.0, steps=6)
    with sim_of(pond, w, precision) as a:
        a.init_fields(w.rho, w.ux, w.uy, w.T)
        a.step(3)
        ck = a.get_state()
        a.step(3)
        ref, ref_m = a.get_state(), a.moments()
    with sim_of(pond, w, precision) as b:
        b.set_state(ck)
        b.step(3)
        if precision == "fp64":
            np.testing.assert_array_equal(b.get_state(), ref)
        else:
            err = rel_err(b.moments(), ref_m)
            assert max(err.values()) <= 1e-6, err


def test_batches_refuse_d3q27(pond):
    w = inputs.droplet3d(n=8, radius=2.0, steps=1)
    with sim_of(pond, w, "fp64") as sim:
        sim.init_fields(w.rho, w.ux, w.uy, w.T)
        b = pond.Batch()
        with pytest.raises(pond.PondError):
            b.add(sim)
        b.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_droplet_sampled_nodes(pond, precision):
    """96 x 96 x 64 droplet (the D3Q27 bench workload): after 3 GPU steps, one more GPU
    step equals the oracle's step of sampled nodes from the GPU's state."""
    w = inputs.droplet3d(n=96, ny=96, nz=64, radius=20.0, steps=3)
    P = params3(w)
    with sim_of(pond, w, precision) as sim:
        sim.init_fields(w.rho, w.ux, w.uy, w.T)
        sim.step(w.steps)
        prev = sim.get_state()
        sim.step(1)
        now = sim.get_state()
    r = np.random.default_rng(11)
    nodes = np.unique(np.concatenate([[0, w.nodes - 1, w.nodes // 2], r.integers(0, w.nodes, 40)]))
    rows = o3.step_nodes(P, prev, nodes)
    flat = now.reshape(63, -1)[:, nodes].T
    L = o3.PL

    def fields(rw):
        m = {"rho": rw[:, L["rho"]], "ux": rw[:, L["uhx"]], "uy": rw[:, L["uhy"]], "uz": rw[:, L["uhz"]],
             "T": rw[:, L["T"]]}
        m["p"] = m["rho"] * P.R * m["T"] / (1.0 - P.b * m["rho"]) - P.a * m["rho"] ** 2
        return m
    err = rel_err(fields(flat), fields(rows))
    assert max(err.values()) <= TOL[precision], err
