"""D2Q16 GPU path (libpond with lattice POND_D2Q16, through its C ABI) against the FP64
oracle on the same lattice.

Element by element on small grids (several 32 x 4 node patches plus ragged tails, and
the 128 x 1 strips of grids of fewer than four rows), the current-time non-local
variant, conservation sums, checkpoint/resume, and one-step checks at
sampled nodes of a full-size 1024 x 512 droplet (the oracle steps those nodes from the
GPU's own previous state).  Bars as on D2Q9: FP64 <= 1e-11, mixed <= 1e-5 relative
L-infinity per field (rho, uhat_x, uhat_y, T, p).
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2002_09217_gb300 import inputs

from parity_util import TOL, oracle_run, params_of, rel_linf, sample_nodes

pytestmark = pytest.mark.gpu
LAT = "d2q16"


@pytest.fixture(scope="module")
def pond():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2002_09217_gb300 import pond as mod
    mod.load()
    return mod


def gpu_run(pond, w, precision, steps=None, **kw):
    with pond.from_workload(w, precision=precision, lattice=LAT, **kw) as sim:
        sim.init_fields(*w.fields())
        sim.step(w.steps if steps is None else steps)
        return sim.moments(), sim.stats()


def small_cases():
    yield "slab40x6", inputs.slab(nx=40, ny=6, Tr=0.9, steps=25)
    yield "droplet24x20", inputs.droplet(n=24, ny=20, Tr=0.9, radius=5.0, steps=20)
    yield "droplet70x9", inputs.droplet(n=70, ny=9, Tr=0.9, radius=3.0, steps=10)
    yield "shock36x10_zerograd", inputs.shock_in_vapour(n=36, Tr=0.8, Mach=1.5, steps=15)
    yield "tube60x3_zerograd", inputs.shock_tube(nx=60, ny=3, width=2.0, steps=30)
    yield "column1x33", inputs.slab(nx=1, ny=33, Tr=0.9, steps=10)
    yield "single_node", inputs.slab(nx=1, ny=1, Tr=0.9, steps=5)
    yield "strong_shock_Tr0.7_Ma3", inputs.shock_in_vapour(n=20, Tr=0.7, Mach=3.0, steps=12)
    yield "sound_liquid_96x1", inputs.sound_pulse(0.9, "liquid", nx=96, width=4.0, steps=60)
    yield "dieterici_iso_48x3", inputs.dieterici_slab(0.8, nx=48, ny=3, steps=40)
    yield "anomalous_tube_64x2", dataclasses.replace(inputs.nonclassical_tube("fig4", nx=64, ny=2), steps=40)
    yield "double_well_slab_48x3", inputs.simplified_eos("slab", nx=48, ny=3, steps=40)
    yield "hot_bump24x20_wide_regions", wide_region_droplet()


def wide_region_droplet():
    """The 24 x 20 droplet's density field at 1.7 T_cr (a supercritical density bump) with
    dt = 1: sqrt(theta) dt up to 0.47, so that the departure floors of about two thirds of
    the nodes spread over three nodes (regions wider than 6), which take the per-pair
    stream, and the rest the region stream."""
    w = inputs.droplet(n=24, ny=20, Tr=0.9, radius=5.0, steps=8)
    return dataclasses.replace(w, name="hot_bump24x20_dt1", dt=1.0, T=w.T * (1.7 / 0.9))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", [c[0] for c in small_cases()])
def test_small_grids_match_oracle(pond, case, precision):
    w = dict(small_cases())[case]
    P, st, ostats = oracle_run(w, lattice=LAT)
    ref = oracle.moments(P, st)
    got, gstats = gpu_run(pond, w, precision)
    err = rel_linf(got, ref)
    assert max(err.values()) <= TOL[precision], err
    assert gstats["nonfinite"] == 0
    if precision == "fp64":
        assert abs(gstats["streams"] - ostats["streams"]) <= 0.01 * ostats["streams"] + 2


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_region_and_pair_streams_are_both_taken(pond, precision):
    """Every stream of a usual workload (|v| dt < 1) takes the region stream over at most
    6 x 6 nodes; the wide-region droplet sends streams down both paths."""
    w = inputs.droplet(n=24, ny=20, Tr=0.9, radius=5.0, steps=5)
    _, st = gpu_run(pond, w, precision)
    assert st["pair_streams"] == 0
    assert 15 * st["streams"] <= st["region_nodes"] <= 36 * st["streams"], st
    _, st = gpu_run(pond, wide_region_droplet(), precision)
    assert 0 < st["pair_streams"] < st["streams"], st
    assert st["region_nodes"] > 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_current_time_nonlocal_matches_oracle(pond, precision):
    w = inputs.slab(nx=40, ny=6, Tr=0.9, steps=15)
    P, st, _ = oracle_run(w, lattice=LAT, nonlocal_="current")
    got, _ = gpu_run(pond, w, precision, nonlocal_="current")
    err = rel_linf(got, oracle.moments(P, st))
    assert max(err.values()) <= TOL[precision], err


def test_full_state_and_conservation_sums_match_oracle(pond):
    w = inputs.droplet(n=32, ny=24, Tr=0.85, radius=6.0, steps=12)
    P, st, _ = oracle_run(w, lattice=LAT)
    with pond.from_workload(w, precision="fp64", lattice=LAT) as sim:
        sim.init_fields(*w.fields())
        sim.step(w.steps)
        got = sim.get_state()
        sums = sim.conservation()
    assert got.shape == st.shape == (39, 24, 32)
    scale = np.abs(st).reshape(39, -1).max(axis=1)
    scale[scale == 0] = 1.0
    err = (np.abs(got - st).reshape(39, -1).max(axis=1) / scale).max()
    assert err <= 1e-11, err
    L = oracle.core.plane_layout(LAT)
    rho = st[L["rho"]]
    want = [rho.sum(), (rho * st[L["uhx"]]).sum(), (rho * st[L["uhy"]]).sum(),
            0.5 * st[L["g"]:L["g"] + 16].sum()]
    np.testing.assert_allclose(sums, want, rtol=1e-11, atol=1e-11 * abs(want[0]))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_checkpoint_resume(pond, precision):
    """pond_get_state / pond_set_state round trip: FP64 resumes bit for bit; the mixed
    form exchanges its kept remainders folded into the FP64 populations and splits them
    again, which reproduces the run to rounding (1e-6 on the fields after 3 more steps)."""
    w = inputs.droplet(n=40, ny=20, Tr=0.9, radius=5.0, steps=6)
    with pond.from_workload(w, precision=precision, lattice=LAT) as a:
        a.init_fields(*w.fields())
        a.step(4)
        ck = a.get_state()
        a.step(3)
        ref, ref_m = a.get_state(), a.moments()
    with pond.from_workload(w, precision=precision, lattice=LAT) as b:
        b.set_state(ck)
        b.step(3)
        if precision == "fp64":
            np.testing.assert_array_equal(b.get_state(), ref)
        else:
            err = rel_linf(b.moments(), ref_m)
            assert max(err.values()) <= 1e-6, err


def _fields_q16(P, rows):
    L = oracle.core.plane_layout(LAT)
    m = {"rho": rows[:, L["rho"]], "ux": rows[:, L["uhx"]], "uy": rows[:, L["uhy"]], "T": rows[:, L["T"]]}
    m["p"] = m["rho"] * P.R * m["T"] / (1.0 - P.b * m["rho"]) - P.a * m["rho"] ** 2
    return m


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_droplet_sampled_nodes(pond, precision):
    """1024 x 512 droplet (the D2Q16 bench workload's grid): after 5 GPU steps, one more
    GPU step equals the oracle's step of sampled nodes from the GPU's state."""
    w = dataclasses.replace(inputs.droplet(n=1024, ny=512, Tr=0.85, radius=120.0), steps=5)
    P = params_of(w, lattice=LAT)
    with pond.from_workload(w, precision=precision, lattice=LAT) as sim:
        sim.init_fields(*w.fields())
        sim.step(w.steps)
        prev = sim.get_state()
        sim.step(1)
        now = sim.get_state()
    nodes = sample_nodes(w.nx, w.ny, 48)
    rows = oracle.step_nodes(P, prev, nodes)
    ref = _fields_q16(P, rows)
    got = _fields_q16(P, now.reshape(39, -1)[:, nodes].T)
    err = rel_linf(got, ref)
    assert max(err.values()) <= TOL[precision], err
