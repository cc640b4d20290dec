"""Non-classical gas dynamics through the GPU path (main text, Fig. 4; SM "Shock tube"):
in the anomalous tube (delta = 0.0125, Gamma < 0) the rarefaction travels as a shock,
keeping its steepness from t*/2 to t*; in the classical case I (delta = 0.329) it
spreads as a fan while the compression shock keeps its steepness."""
import pytest

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
def test_anomalous_tube_rarefaction_shock(experiments, precision):
    res = experiments.wave_steepness(inputs.nonclassical_tube("fig4", nx=1024), precision)
    h, e = res["half"], res["end"]
    assert res["nonfinite"] == 0
    assert e["left_at"] < h["left_at"]               # moves left
    assert e["left_outer"] > e["left_inner"]         # expands the fluid
    assert e["left_peak"] > 0.75 * h["left_peak"], res


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_classical_tube_rarefaction_fan(experiments, precision):
    res = experiments.wave_steepness(inputs.nonclassical_tube("I", nx=1024), precision)
    h, e = res["half"], res["end"]
    assert e["left_at"] < h["left_at"]
    assert e["left_peak"] < 0.65 * h["left_peak"], res
    assert e["right_peak"] > 0.85 * h["right_peak"], res
