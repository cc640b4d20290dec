"""The paper's benchmarks through the GPU path on the D2Q16 lattice: the speed of sound of
the van der Waals fluid (main text, Fig. 1) against its closed-form isentropic value, and
the saturated densities of a flat interface (main text, Fig. 2) against Maxwell's
equal-area rule.  The lattice changes the velocity set, not the hydrodynamics, so the
bars are those of the D2Q9 tests."""
import math

import pytest

from oracle import thermo
from paper_2002_09217_gb300 import inputs

pytestmark = pytest.mark.gpu
LAT = "d2q16"


@pytest.fixture(scope="module")
def experiments():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2002_09217_gb300 import experiments as mod
    from paper_2002_09217_gb300 import pond
    pond.load()
    return mod


@pytest.mark.parametrize("phase", ["vapour", "liquid"])
@pytest.mark.parametrize("precision,bar", [("fp64", 5e-4), ("mixed", 3e-3)])
def test_pulse_speed_matches_closed_form(experiments, phase, precision, bar):
    w = inputs.sound_pulse(0.85, phase, nx=2048, width=12.0)
    res = experiments.sound_speed(w, precision, lattice=LAT)
    rv, rl = thermo.maxwell(0.85)
    want = thermo.sound_speed(rv if phase == "vapour" else rl, 0.85 * thermo.critical()[1], 1.0 / 3.0)
    assert res["nonfinite"] == 0
    assert res["c"] == pytest.approx(want, rel=bar), res


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_bulk_densities_on_maxwell(experiments, precision):
    probe = inputs.coexistence_slab(0.9, 1.0 / 3.0, nx=256)
    steps = int(math.ceil(1500.0 / probe.dt))
    w = inputs.coexistence_slab(0.9, 1.0 / 3.0, nx=256, steps=steps)
    res = experiments.coexistence(w, precision, lattice=LAT)
    rv, rl = thermo.maxwell(0.9)
    assert res["nonfinite"] == 0
    assert res["rho_v"] == pytest.approx(rv, rel=0.01), res
    assert res["rho_l"] == pytest.approx(rl, rel=0.01), res
