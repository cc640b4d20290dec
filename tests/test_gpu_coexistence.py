"""Coexistence curves through the GPU path: a flat liquid slab in its vapour relaxes to
bulk densities on Maxwell's equal-area values, for the van der Waals fluid with
C_v = R/delta, delta = 1/3 and 2/3 (main text, Fig. 2: the saturated densities do not
depend on delta), and for the Dieterici fluid held isothermal (SM "Coexistence curve")."""
import math

import pytest

from oracle import thermo
from paper_2002_09217_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def experiments():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2002_09217_gb300 import experiments as mod
    from paper_2002_09217_gb300 import pond
    pond.load()
    return mod


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("delta", [1.0 / 3.0, 2.0 / 3.0])
@pytest.mark.parametrize("Tr", [0.85, 0.9, 0.95])
def test_bulk_densities_on_maxwell(experiments, Tr, delta, precision):
    probe = inputs.coexistence_slab(Tr, delta, nx=256)
    steps = int(math.ceil(1500.0 / probe.dt))          # the same relaxation time for every dt
    if precision == "fp64":
        steps = min(steps, 6000)
    w = inputs.coexistence_slab(Tr, delta, nx=256, steps=steps)
    res = experiments.coexistence(w, precision)
    rv, rl = thermo.maxwell(Tr)
    assert res["nonfinite"] == 0
    assert res["rho_v"] == pytest.approx(rv, rel=0.01), res
    assert res["rho_l"] == pytest.approx(rl, rel=0.01), res


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_sub_spinodal_interface_at_0_8_on_maxwell(experiments, precision):
    """At 0.8 T_cr the van der Waals pressure is negative inside the interface and the
    gauge uses the floored pressure (reading R11).  The vapour density then drifts upward
    at a rate that falls with the box size (measured at t = 1500: +2.8 % on 128 nodes,
    +0.7 % on 256, +0.1 % on 512; +0.9 % on 512 at t = 6000): on a 512-node box the flat
    interface holds Maxwell's densities within 1 % at the usual relaxation time."""
    probe = inputs.coexistence_slab(0.8, nx=512)
    w = inputs.coexistence_slab(0.8, nx=512, steps=int(math.ceil(1500.0 / probe.dt)))
    res = experiments.coexistence(w, precision)
    rv, rl = thermo.maxwell(0.8)
    assert res["nonfinite"] == 0 and res["clamped"] > 0
    assert res["rho_v"] == pytest.approx(rv, rel=0.01), res
    assert res["rho_l"] == pytest.approx(rl, rel=0.01), res


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_advected_slab_on_maxwell(experiments, precision):
    """The advected case of Fig. 2 (0.9 T_cr, the slab moving at U = 5 U_ch): the vapour
    density's error falls as the inverse box size at a fixed time (measured at t = 1900:
    -8.5 / -4.4 / -2.3 / -1.3 / -0.6 % on 128 / 256 / 512 / 1024 / 2048 nodes); on 2048
    nodes both densities are within 1 % of Maxwell's, and halving the box doubles the
    vapour error."""
    rv, rl = thermo.maxwell(0.9)
    err = {}
    for nx in (1024, 2048):
        probe = inputs.coexistence_slab(0.9, advected=True, nx=nx)
        w = inputs.coexistence_slab(0.9, advected=True, nx=nx, steps=int(math.ceil(1900.0 / probe.dt)))
        res = experiments.coexistence(w, precision)
        assert res["nonfinite"] == 0
        err[nx] = (res["rho_v"] / rv - 1.0, res["rho_l"] / rl - 1.0)
    assert abs(err[2048][0]) < 0.01 and abs(err[2048][1]) < 0.01, err
    assert 1.6 < err[1024][0] / err[2048][0] < 2.5, err


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("Tr", [0.7, 0.8, 0.9])
def test_isothermal_dieterici_on_maxwell(experiments, Tr, precision):
    w = inputs.dieterici_slab(Tr, nx=256, steps=3000)
    res = experiments.coexistence(w, precision)
    rv, rl = thermo.dieterici_maxwell(Tr)
    assert res["nonfinite"] == 0 and res["clamped"] == 0
    assert res["rho_v"] == pytest.approx(rv, rel=0.01), res
    assert res["rho_l"] == pytest.approx(rl, rel=0.01), res


def test_double_well_slab_near_its_saturated_densities(experiments):
    """The simplified EoS's slab oscillates slowly about its saturated densities; the
    average of the last quarter sits within 3 %."""
    sp = thermo.SIMP
    res = experiments.coexistence(inputs.simplified_eos("slab", nx=256), "mixed")
    assert res["nonfinite"] == 0
    assert res["rho_v"] == pytest.approx(sp["rho_v"], rel=0.03), res
    assert res["rho_l"] == pytest.approx(sp["rho_l"], rel=0.03), res


def _laplace_dpR(pond, R, n, steps=120000, every=500):
    """Pressure inside minus outside a droplet of radius R in an n x n periodic box at
    0.9 T_cr, averaged over the second half of the run (the droplet and the box ring with
    sound waves), times R."""
    import numpy as np
    w = inputs.droplet(n=n, Tr=0.9, radius=float(R), amp=0.0, steps=steps)
    dps = []
    with pond.from_workload(w, precision="mixed") as sim:
        sim.init_fields(*w.fields())
        sim.step(steps // 2)
        for _ in range(steps // 2 // every):
            sim.step(every)
            p = sim.moments()["p"]
            c = n // 2
            inside = p[c - 4:c + 4, c - 4:c + 4].mean()
            corners = np.concatenate([p[:6, :6].ravel(), p[-6:, -6:].ravel(), p[:6, -6:].ravel(),
                                      p[-6:, :6].ravel()])
            dps.append(inside - corners.mean())
    return float(np.mean(dps)) * R


def test_laplace_law_two_radii(experiments):
    """Delta p = sigma / R: Delta p R is the same for droplets of radius 32 and 64 (the
    interface is 4 nodes wide, so smaller droplets are not used).  The droplets and the
    box keep ringing with sound and the temperature relaxes slowly, so the time averages
    agree to ~12 % (measured 0.030 / 0.026); the bar, 20 %, still tells the 1/R law from
    any other (a pressure jump independent of R would be 100 % off)."""
    from paper_2002_09217_gb300 import pond
    s32 = _laplace_dpR(pond, 32, 128)
    s64 = _laplace_dpR(pond, 64, 256)
    assert s32 > 0 and s64 > 0
    assert s32 == pytest.approx(s64, rel=0.2), (s32, s64)
