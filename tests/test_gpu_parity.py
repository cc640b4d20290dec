"""GPU time step (libpond through its C ABI) against the FP64 oracle.

Element-by-element parity on seeded inputs at sizes the oracle finishes in
seconds (several 128-node launch tiles plus a ragged tail), on the full
128x4 slab for its 2000 steps (the other workloads at their own step counts are in
test_gpu_full_length.py).  Bars: FP64 <= 1e-11, mixed FP32/FP64 <= 1e-5 relative
L-infinity per field (rho, uhat_x, uhat_y, T, p).
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2002_09217_gb300 import inputs

from parity_util import TOL, oracle_run, rel_linf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pond():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2002_09217_gb300 import pond as mod
    mod.load()
    return mod


def gpu_run(pond, w, precision, steps=None, **kw):
    with pond.from_workload(w, precision=precision, **kw) as sim:
        sim.init_fields(*w.fields())
        sim.step(w.steps if steps is None else steps)
        return sim.moments(), sim.stats()


def small_cases():
    yield "slab40x6", inputs.slab(nx=40, ny=6, Tr=0.9, steps=25)
    yield "droplet24x20", inputs.droplet(n=24, ny=20, Tr=0.9, radius=5.0, steps=20)
    yield "shock36x10_zerograd", inputs.shock_in_vapour(n=36, Tr=0.8, Mach=1.5, steps=15)
    yield "tube60x3_zerograd", inputs.shock_tube(nx=60, ny=3, width=2.0, steps=30)
    yield "column1x33", inputs.slab(nx=1, ny=33, Tr=0.9, steps=10)
    yield "single_node", inputs.slab(nx=1, ny=1, Tr=0.9, steps=5)
    yield "strong_shock_Tr0.7_Ma3", inputs.shock_in_vapour(n=20, Tr=0.7, Mach=3.0, steps=12)
    yield "sound_liquid_96x1", inputs.sound_pulse(0.9, "liquid", nx=96, width=4.0, steps=60)
    yield "sound_critical_64x2", inputs.sound_pulse(phase="critical", nx=64, ny=2, width=4.0, steps=40)
    yield "isothermal_sound_80x1", inputs.sound_pulse(0.9, "vapour", nx=80, width=4.0, steps=50,
                                                      isothermal=True)
    yield "dieterici_iso_48x3", inputs.dieterici_slab(0.8, nx=48, ny=3, steps=40)
    yield "anomalous_tube_64x2", dataclasses.replace(inputs.nonclassical_tube("fig4", nx=64, ny=2), steps=40)
    yield "double_well_slab_48x3", inputs.simplified_eos("slab", nx=48, ny=3, steps=40)
    yield "droplet_isothermal_40x36", dataclasses.replace(
        inputs.droplet(n=40, ny=36, Tr=0.9, radius=8.0, amp=0.0, steps=30), isothermal=True)
    yield "double_well_pulse_80x1", inputs.simplified_eos("pulse", "vapour", nx=80, pulse_width=4.0, steps=40)
    # near the critical point, where the EoS (float-float in the mixed form) is flattest:
    # a droplet and a slab at 0.95 T_cr (3.7 streams per node), a 1e-2 pulse at the
    # critical state, and a supercritical tube at 1.02 T_cr
    yield "droplet32x28_Tr0.95", inputs.droplet(n=32, ny=28, Tr=0.95, radius=7.0, steps=30)
    yield "slab48x3_Tr0.95", inputs.slab(nx=48, ny=3, Tr=0.95, steps=40)
    yield "sound_critical_amp1e-2_64x2", inputs.sound_pulse(phase="critical", nx=64, ny=2, amp=1e-2, width=4.0,
                                                            steps=40)
    yield "tube60x3_Tr1.02", inputs.shock_tube(nx=60, ny=3, Tr=1.02, width=2.0, steps=30)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", [c[0] for c in small_cases()])
def test_small_grids_match_oracle(pond, case, precision):
    w = dict(small_cases())[case]
    P, st, ostats = oracle_run(w)
    ref = oracle.moments(P, st)
    got, gstats = gpu_run(pond, w, precision)
    err = rel_linf(got, ref)
    assert max(err.values()) <= TOL[precision], err
    assert gstats["nonfinite"] == 0
    if precision == "fp64":
        # same frame-search work up to nodes sitting at the tolerance boundary
        assert abs(gstats["streams"] - ostats["streams"]) <= 0.01 * ostats["streams"] + 2


FLOWING = ("shock36x10_zerograd", "strong_shock_Tr0.7_Ma3", "tube60x3_zerograd", "tube60x3_Tr1.02")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", FLOWING)
def test_plain_relative_velocity_error_where_the_fluid_flows(pond, case, precision):
    """Where the flow speed is a sizeable part of the sound speed, the velocities also meet
    the bar as plain relative L-infinity errors, |got - ref|max / |ref|max (the other tests
    normalise by max(|uhat|, sqrt(max p/rho)))."""
    w = dict(small_cases())[case]
    P, st, _ = oracle_run(w)
    ref = oracle.moments(P, st)
    got, _ = gpu_run(pond, w, precision)
    cs = float(np.sqrt(np.max(np.abs(ref["p"] / ref["rho"]))))
    for k in ("ux", "uy"):
        umax = float(np.abs(ref[k]).max())
        if umax < 0.1 * cs:
            continue
        err = float(np.abs(np.asarray(got[k]) - ref[k]).max() / umax)
        print("%s %s %s: |u|max/cs %.3f, plain rel. err %.3e" % (case, precision, k, umax / cs, err))
        assert err <= TOL[precision], (k, umax / cs, err)


def test_ideal_gas_limit_matches_oracle(pond):
    nx = 64
    x = np.arange(nx) + 0.5
    sw = 0.5 * (1.0 - np.tanh((x - nx / 2) / 2.0))
    rho = np.tile(0.125 + 0.875 * sw, (2, 1))
    T = np.tile((0.01 + 0.09 * sw), (2, 1)) / rho
    w = inputs.Workload("sod64x2", nx, 2, 1, 0, 0.0, 0.0, 1.0, 0.5, 40, rho, 0 * rho, 0 * rho, T,
                        a=0.0, b=0.0, delta=0.4, p_floor=1e-6)
    P, st, _ = oracle_run(w)
    ref = oracle.moments(P, st)
    for prec in ("fp64", "mixed"):
        got, _ = gpu_run(pond, w, prec)
        err = rel_linf(got, ref)
        assert max(err.values()) <= TOL[prec], (prec, err)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_slab128x4_full_run(pond, precision):
    """The 128x4 quasi-1D slab at T = 0.9 T_cr with seeded noise, all 2000 steps."""
    w = inputs.slab()
    P, st, _ = oracle_run(w)
    ref = oracle.moments(P, st)
    got, gstats = gpu_run(pond, w, precision)
    err = rel_linf(got, ref)
    assert max(err.values()) <= TOL[precision], err
    assert gstats["nonfinite"] == 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_shocktube_reduced_full_run(pond, precision):
    """The supercritical tube recipe at 256x4 for 600 steps (waves reach the walls)."""
    w = inputs.shock_tube(nx=256, ny=4, steps=600)
    P, st, _ = oracle_run(w)
    ref = oracle.moments(P, st)
    got, _ = gpu_run(pond, w, precision)
    err = rel_linf(got, ref)
    assert max(err.values()) <= TOL[precision], err


def test_conservation_sums_match_oracle_state(pond):
    w = inputs.droplet(n=48, ny=40, Tr=0.9, radius=10.0, steps=30)
    P, st, _ = oracle_run(w)
    flat = st.reshape(25, -1)
    want = [flat[21].sum(), (flat[21] * flat[23]).sum(), (flat[21] * flat[24]).sum(),
            0.5 * flat[9:18].sum()]
    with pond.from_workload(w, precision="fp64") as sim:
        sim.init_fields(*w.fields())
        sim.step(w.steps)
        got = sim.conservation()
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-12)


def test_device_pointer_paths_equal_host_paths(pond):
    import torch
    w = inputs.slab(nx=40, ny=6, steps=5)
    dev = [torch.tensor(a, device="cuda", dtype=torch.float64) for a in w.fields()]
    with pond.from_workload(w, precision="mixed") as a, pond.from_workload(w, precision="mixed") as b:
        a.init_fields(*w.fields())
        b.init_fields(*dev)
        a.step(5)
        b.step(5)
        ha = a.moments()
        out = {k: torch.empty((w.ny, w.nx), device="cuda", dtype=torch.float64) for k in ha}
        b.moments_device(out)
        torch.cuda.synchronize()
        for k in ha:
            np.testing.assert_array_equal(ha[k], out[k].cpu().numpy())


def test_state_round_trip_and_invalid_init(pond):
    w = inputs.slab(nx=16, ny=4, steps=3)
    with pond.from_workload(w, precision="fp64") as sim:
        sim.init_fields(*w.fields())
        sim.step(3)
        s = sim.get_state()
        sim.set_state(s)
        np.testing.assert_array_equal(sim.get_state(), s)
        bad = w.rho.copy()
        bad[1, 2] = -1.0
        with pytest.raises(pond.PondError) as ei:
            sim.init_fields(bad, w.ux, w.uy, w.T)
        assert ei.value.status == 1


@pytest.mark.parametrize("lanes", [8, 16])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_lanes_per_node_variants_match_oracle(pond, lanes, precision):
    """Both work splits of the step kernel (8 or 16 lanes per node) meet the bar."""
    w = inputs.droplet(n=40, ny=28, Tr=0.9, radius=7.0, steps=20)
    P, st, _ = oracle_run(w)
    ref = oracle.moments(P, st)
    got, gstats = gpu_run(pond, w, precision, lanes_per_node=lanes)
    err = rel_linf(got, ref)
    assert max(err.values()) <= TOL[precision], err


@pytest.mark.parametrize("tile_x", [1, 2, 4, 8, 16])
def test_tile_shapes_match_oracle(pond, tile_x):
    """Every step-kernel tile shape (tile_x x 16/tile_x nodes, staged with a halo of 3)
    gives the oracle's result, including ragged tiles at the grid edge and departure
    points beyond the halo (a fast uniform flow, |v| dt > 1)."""
    w = inputs.droplet(n=37, ny=23, Tr=0.9, radius=6.0, steps=12)
    P, st, _ = oracle_run(w)
    ref = oracle.moments(P, st)
    got, _ = gpu_run(pond, w, "fp64", tile_x=tile_x)
    err = rel_linf(got, ref)
    assert max(err.values()) <= TOL["fp64"], err
    # fast flow: u = 2.6, dt = 0.5 -> departures up to ~1.6 nodes away plus the stencil
    fast = inputs.slab(nx=30, ny=9, Tr=0.95, steps=6)
    fast.ux = np.full_like(fast.rho, 2.6)
    P, st, _ = oracle_run(fast)
    ref = oracle.moments(P, st)
    got, _ = gpu_run(pond, fast, "fp64", tile_x=tile_x)
    err = rel_linf(got, ref)
    assert max(err.values()) <= TOL["fp64"], err


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_current_time_variant_matches_oracle(pond, precision):
    """The two-pass step with current-time non-local terms against the oracle's two-pass
    step (a moving slab and a droplet, where the terms change within a step)."""
    slab = inputs.slab(nx=40, ny=6, Tr=0.9, steps=20)
    slab.ux = np.full_like(slab.rho, 0.05)
    for w in (slab, inputs.droplet(n=24, ny=20, Tr=0.9, radius=5.0, steps=12)):
        P, st, _ = oracle_run(w, nonlocal_="current")
        ref = oracle.moments(P, st)
        got, gstats = gpu_run(pond, w, precision, nonlocal_="current")
        err = rel_linf(got, ref)
        assert max(err.values()) <= TOL[precision], (w.name, err)
        if precision == "fp64":
            lag, _ = gpu_run(pond, w, precision)
            assert max(rel_linf(lag, ref).values()) > 10 * TOL["fp64"]   # the variant matters


def test_current_time_context_is_stepped_alone(pond):
    w = inputs.slab(nx=16, ny=4, steps=2)
    with pond.from_workload(w, precision="mixed", nonlocal_="current") as sim:
        sim.init_fields(*w.fields())
        batch = pond.Batch()
        with pytest.raises(pond.PondError):
            batch.add(sim)
        batch.close()
        sim.step(2)


def test_fma_peak_microbenchmark_is_plausible(pond):
    """The measurement utility's FMA-chain peaks sit below the unit-count peaks of a
    152-SM, 2.07 GHz GPU (FP32 80.5 TFLOP/s, FP64 at 1/64) and above half of them."""
    import torch
    n32 = torch.cuda.get_device_properties(0).multi_processor_count * 128 * 2 * 2.07e9 / 1e12
    fp32 = pond.fma_peak("mixed", 100000)
    fp64 = pond.fma_peak("fp64", 10000)
    assert 0.5 * n32 < fp32 < 1.05 * n32, (fp32, n32)
    assert 0.3 * n32 / 64 < fp64 < 1.05 * n32 / 64, (fp64, n32 / 64)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_checkpoint_and_resume(pond, precision):
    """Stop after 20 steps, save the state (pond_get_state), restore it into a new context
    (pond_set_state) and run 15 more: the same fields as 35 steps straight, to rounding of
    what the exchanged state leaves out (the momentum's kept low part, below one ulp)."""
    w = inputs.droplet(n=40, ny=28, Tr=0.9, radius=7.0, steps=35)
    straight, _ = gpu_run(pond, w, precision)
    with pond.from_workload(w, precision=precision) as a:
        a.init_fields(*w.fields())
        a.step(20)
        saved = a.get_state()
    with pond.from_workload(w, precision=precision) as b:
        b.set_state(saved)
        b.step(15)
        resumed = b.moments()
    err = rel_linf(resumed, straight)
    assert max(err.values()) <= (1e-12 if precision == "fp64" else 1e-6), err


def test_oversized_grid_is_out_of_memory(pond):
    """A grid whose state cannot fit in device memory is refused with POND_ENOMEM."""
    with pytest.raises(pond.PondError) as ei:
        pond.Simulation(200000, 200000, precision="fp64")
    assert ei.value.status == 2
