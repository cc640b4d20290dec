"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/pond.h declares; the product path refuses to run without a
GPU instead of falling back to the CPU."""
import ctypes
import os
import re

import pytest

from paper_2002_09217_gb300 import build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if hdr.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", hdr)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(pond_\w+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    path = build_lib.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pond_create", "pond_init_fields", "pond_step", "pond_moments", "pond_destroy",
                     "pond_conservation", "pond_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_string(lib):
    lib.pond_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.pond_version()


def test_invalid_parameters_are_rejected_on_the_host(lib):
    """Parameter checks run before any device call, so they work without a GPU."""
    from paper_2002_09217_gb300 import pond
    L = pond.load()
    g = pond.Grid(0, 4, 0, 0)
    lat = pond.Lattice(0)
    eos = pond.Eos(0, 2 / 49, 2 / 21, 1.0, 1 / 3)
    opts = pond.Opts(1, 20, 1e-6, 0.5, -1.0, 1e-4, None, pond._ALLOC(), pond._FREE(), None, 0, 0)
    out = ctypes.c_void_p()
    assert L.pond_create(ctypes.byref(g), ctypes.byref(lat), ctypes.byref(eos), 0.0, 1.0,
                         ctypes.byref(opts), ctypes.byref(out)) == 1
    g = pond.Grid(8, 8, 0, 0)
    assert L.pond_create(ctypes.byref(g), ctypes.byref(lat), ctypes.byref(eos), 0.0, 0.5,
                         ctypes.byref(opts), ctypes.byref(out)) == 1      # tau must exceed 1/2
    bad = pond.Eos(0, 2 / 49, 2 / 21, 1.0, 0.9)                           # delta > 2/3
    assert L.pond_create(ctypes.byref(g), ctypes.byref(lat), ctypes.byref(bad), 0.0, 1.0,
                         ctypes.byref(opts), ctypes.byref(out)) == 1
    for bad in (pond.Eos(pond.POND_DIETERICI, 32 / 441, 1 / 7, 1.0, 1 / 3, 0, 0.0),   # not isothermal
                pond.Eos(0, 2 / 49, 2 / 21, 1.0, 1 / 3, 1, 0.0),                      # T_iso <= 0
                pond.Eos(5, 2 / 49, 2 / 21, 1.0, 1 / 3),                              # unknown kind
                pond.Eos(pond.POND_SIMPLIFIED, 0, 0, 1, 1 / 3, 0, 0.0, 1e-3, 5.0, 0.5, 0.1),  # not isothermal
                pond.Eos(pond.POND_SIMPLIFIED, 0, 0, 1, 1 / 3, 1, 0.1, 1e-3, 5.0, 0.5, 0.0)):  # p0 = 0
        assert L.pond_create(ctypes.byref(g), ctypes.byref(lat), ctypes.byref(bad), 0.0, 1.0,
                             ctypes.byref(opts), ctypes.byref(out)) == 1
    # the z extent: D3Q27 needs nz >= 1 and a valid bc_z; the 2-D lattices nz <= 1
    for gz, lk in ((pond.Grid(8, 8, 0, 0, 0, 0), pond.POND_D3Q27), (pond.Grid(8, 8, 0, 0, 4, 2), pond.POND_D3Q27),
                   (pond.Grid(8, 8, 0, 0, 2, 0), pond.POND_D2Q9), (pond.Grid(8, 8, 0, 0, 3, 0), pond.POND_D2Q16)):
        lz = pond.Lattice(lk)
        assert L.pond_create(ctypes.byref(gz), ctypes.byref(lz), ctypes.byref(eos), 0.0, 1.0,
                             ctypes.byref(opts), ctypes.byref(out)) == 1
    lat_bad = pond.Lattice(3)                                             # unknown lattice
    assert L.pond_create(ctypes.byref(g), ctypes.byref(lat_bad), ctypes.byref(eos), 0.0, 1.0,
                         ctypes.byref(opts), ctypes.byref(out)) == 1
    assert not out.value
    L.pond_destroy(None)


def test_no_cpu_fallback_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2002_09217_gb300 import pond
    with pytest.raises(pond.PondError):
        pond.Simulation(8, 8)


def test_header_states_the_sticky_status_semantics():
    """The synchronising calls return the device flags: the header documents that
    ENONCONV and ETHETA are warnings whose outputs are written, and declares the batch's
    budget and completion poll."""
    txt = open(os.path.join(ROOT, "include", "pond.h")).read()
    for needle in ("POND_ENONCONV = 4", "POND_ETHETA = 5", "sticky", "pond_batch_set_budget",
                   "pond_batch_poll", "pond_batch_bytes"):
        assert needle in txt, needle


def test_binding_keeps_warning_statuses_and_raises_on_errors():
    """Simulation._check_sync records POND_ENONCONV / POND_ETHETA (the call completed and
    wrote its outputs) and raises on every other non-zero status; checked with a stand-in
    for the library's last-error call, no GPU needed."""
    from paper_2002_09217_gb300 import pond

    class FakeLib:
        @staticmethod
        def pond_last_error(_ctx):
            return b"message"

    sim = pond.Simulation.__new__(pond.Simulation)
    sim._lib, sim._ctx, sim.flags, sim.last_flag = FakeLib(), None, [], None
    sim._check_sync(0)
    assert sim.flags == [] and sim.last_flag is None
    sim._check_sync(4)
    sim._check_sync(5)
    assert [f for f, _ in sim.flags] == ["POND_ENONCONV", "POND_ETHETA"] and sim.last_flag == "POND_ETHETA"
    for st in (1, 3, 6):
        with pytest.raises(pond.PondError) as ei:
            sim._check_sync(st)
        assert ei.value.status == st
    sim._ctx = None


def test_build_tracks_every_included_source():
    """Every header the CUDA translation unit includes is a build dependency, so an edit to
    any of them rebuilds the library."""
    src = open(os.path.join(ROOT, "paper_2002_09217_gb300", "csrc", "pond.cu")).read()
    included = re.findall(r'#include "([^"]+)"', src)
    deps = {os.path.basename(d) for d in build_lib.DEPS}
    assert included and all(os.path.basename(h) in deps for h in included), (included, deps)
