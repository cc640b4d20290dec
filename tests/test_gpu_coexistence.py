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
