"""Sticky device flags returned as status by the synchronising calls, triggered through
data (no fault, no hang): a frame search capped at one stream (POND_ENONCONV) and a
sub-spinodal interface that meets the pressure floor (POND_ETHETA).  Each flag is
reported once and then cleared; the outputs are written either way.  Also the batch's
device-memory budget and its completion poll."""
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


def test_nonconverged_frame_search_is_reported_once(pond):
    w = inputs.slab(nx=64, ny=4, Tr=0.9)
    with pond.from_workload(w, precision="fp64", max_iter=1) as sim:
        sim.init_fields(*w.fields())
        sim.step(3)
        m = sim.moments()
        assert sim.last_flag == "POND_ENONCONV"
        assert np.isfinite(m["rho"]).all() and m["rho"].min() > 0
        assert sim.stats()["nonconverged"] > 0
        sim.moments()                      # nothing new since the report
        assert sim.last_flag is None
        sim.step(1)
        sim.conservation()
        assert sim.last_flag == "POND_ENONCONV"


def test_pressure_floor_is_reported_once(pond):
    # a flat interface at 0.75 T_cr: the van der Waals pressure is negative inside it
    w = inputs.coexistence_slab(0.75, nx=128, steps=50)
    with pond.from_workload(w, precision="mixed") as sim:
        sim.init_fields(*w.fields())
        sim.step(5)
        out = sim.conservation()
        assert sim.last_flag == "POND_ETHETA"
        assert np.isfinite(out).all()
        assert sim.stats()["clamped"] > 0 and sim.stats()["nonconverged"] == 0
        sim.conservation()
        assert sim.last_flag is None


def test_converged_run_reports_ok(pond):
    w = inputs.slab(nx=64, ny=4, Tr=0.9)
    with pond.from_workload(w, precision="fp64") as sim:
        sim.init_fields(*w.fields())
        sim.step(3)
        sim.moments()
        assert sim.last_flag is None and sim.flags == []


def test_batch_budget_refuses_and_poll_reports_completion(pond):
    import torch
    w = inputs.droplet(n=48, ny=40, Tr=0.9, radius=8.0)
    stream = torch.cuda.Stream()
    b = pond.Batch(stream)
    a = pond.from_workload(w, precision="mixed", stream=stream)
    c = pond.from_workload(w, precision="mixed", stream=stream)
    try:
        for s in (a, c):
            s.init_fields(*w.fields())
        assert b.poll()                                    # nothing enqueued yet
        b.set_budget(a.device_bytes() + c.device_bytes() // 2)
        b.add(a)
        assert b.device_bytes() == a.device_bytes()
        with pytest.raises(pond.PondError) as ei:
            b.add(c)
        assert ei.value.status == 2 and len(b) == 1
        with pytest.raises(pond.PondError):
            b.set_budget(a.device_bytes() - 1)             # below what the members hold
        b.step(40)
        b.synchronize()
        assert b.poll()
        b.remove(a)
        assert b.device_bytes() == 0
        b.add(c)                                           # fits once a has left
        b.step(2)
        b.synchronize()
        assert b.poll()
    finally:
        b.close()
        a.close()
        c.close()
