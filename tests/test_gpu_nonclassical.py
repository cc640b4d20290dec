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


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("name,bar,fall", [("I", 2e-3, 0.8), ("fig4", 7e-3, 0.8), ("II", 8e-3, 0.9)])
def test_tubes_converge_to_the_exact_vdw_riemann_solution(experiments, precision, name, bar, fall):
    """The GPU's shock tubes at t* against the exact van der Waals Riemann solution
    (tests/vdw_riemann.py; case I: fan + shock, Fig. 4: rarefaction shock + compression
    fan, case II: composite waves on both sides): relative L1(rho) below the bar on 2048
    nodes and falling from 1024 nodes (measured, both forms: I 1.3e-3 -> 8.3e-4, Fig. 4
    4.8e-3 -> 3.1e-3, II 6.6e-3 -> 5.6e-3)."""
    import json
    import os
    import numpy as np
    from oracle import thermo
    from paper_2002_09217_gb300 import pond
    import vdw_riemann as vr
    tab = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "..",
                                      "paper_2002_09217_gb300", "workloads.json")))["nonclassical"]
    c = tab["cases"][name]
    L, R = c["left"], c["right"]
    rp = vr.Riemann(c["delta"], (L["rho"], 0.0, thermo.pressure(L["rho"], L["T"])),
                    (R["rho"], 0.0, thermo.pressure(R["rho"], R["T"])))
    l1 = []
    for nx in (1024, 2048):
        w = inputs.nonclassical_tube(name, nx=nx)
        with pond.from_workload(w, precision=precision) as sim:
            sim.init_fields(*w.fields())
            sim.step(w.steps)
            rho = sim.moments()["rho"][0]
        re, _, _ = rp.profile(np.arange(nx) + 0.5, w.steps * w.dt, nx / 2)
        l1.append(float(np.abs(rho - re).mean() / np.abs(re).mean()))
    print(name, precision, l1)
    assert l1[1] < bar and l1[1] < fall * l1[0], l1
