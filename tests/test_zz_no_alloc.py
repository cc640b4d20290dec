"""The allocation-free entry point, pond_conservation_noalloc: it serves callers that may
not allocate device memory, so it keeps its scratch in a static device array of the
library.  Its results must equal those of the regular entry point, pond_conservation,
on two calls in a row (the shared array keeps the previous call's contents).

This file is collected last on purpose, so that a run stopping at its first failure has
already run every other test; it also passes when run alone in a fresh process."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_conservation_matches_regular_entry_point_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2002_09217_gb300 import inputs, pond

    for precision in ("fp64", "mixed"):
        w = inputs.droplet(n=96, ny=80, Tr=0.9, radius=16.0, steps=25)
        with pond.from_workload(w, precision=precision) as sim:
            sim.init_fields(*w.fields())
            sim.step(w.steps)
            want = sim.conservation()
            planes = torch.tensor(sim.get_state().reshape(-1), device="cuda", dtype=torch.float64)
            torch.cuda.synchronize()
            first = pond.conservation_noalloc(planes, w.nodes)
            second = pond.conservation_noalloc(planes, w.nodes)
        np.testing.assert_allclose(first, want, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(second, want, rtol=1e-12, atol=1e-12)
        np.testing.assert_array_equal(first, second)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2002_09217_gb300 import pond

    planes = torch.zeros(25 * 8, device="cuda", dtype=torch.float64)
    # a raw address reaches the C entry point, which refuses the size before any launch
    with pytest.raises(pond.PondError) as ei:
        pond.conservation_noalloc(planes.data_ptr(), 8_388_609)
    assert ei.value.status == 1
    with pytest.raises(pond.PondError):
        pond.conservation_noalloc(planes.data_ptr(), 0)
    # a tensor is checked by the wrapper: 25 * n_nodes float64 values, contiguous, on the
    # current device
    for bad, n in ((planes, 8_388_609), (planes, 0), (planes, 9), (planes.float(), 8),
                   (planes.view(25, 8).t(), 8), (planes.cpu(), 8)):
        with pytest.raises(pond.PondError) as ei:
            pond.conservation_noalloc(bad, n)
        assert ei.value.status == 1
