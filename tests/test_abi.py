"""The C-ABI library builds, loads without a GPU and exports every function
that include/chert.h declares; host-only entry points behave as documented."""
import ctypes
import math
import os
import re

import pytest

from paper_2609_26108_b300 import build, chert

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "chert.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(chert_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return chert.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["chert_build_cache", "chert_traveltime", "chert_raypath", "chert_edge_table",
                     "chert_thomsen_to_class", "chert_last_error", "chert_traveltime_workspace_bytes"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_thomsen_to_class_host_only(lib):
    c = chert.thomsen_to_class(3000.0, 1500.0, 0.2, 0.1, 0.1, 60.0, 30.0, tilt=0.3)
    assert list(c.aR)[2] == 9.0e6 and list(c.aR)[3] == 2.25e6
    assert c.aI[0] == pytest.approx(c.aR[0] / 60.0) and c.aI[4] == pytest.approx(c.aR[4] / 30.0)
    assert c.tilt == 0.3
    # Thomsen's delta recovered from the stored moduli
    a11, a13, a33, a44, a66 = list(c.aR)
    d = ((a13 + a44) ** 2 - (a33 - a44) ** 2) / (2 * a33 * (a33 - a44))
    assert d == pytest.approx(0.1, abs=1e-12)


def test_thomsen_to_class_rejects_bad_input(lib):
    with pytest.raises(chert.ChertError) as e:
        chert.thomsen_to_class(1000.0, 1500.0, 0.2, 0.1, 0.1, 60.0, 30.0)
    assert e.value.code == chert.EINVAL
    with pytest.raises(chert.ChertError):
        chert.thomsen_to_class(3000.0, 1500.0, 0.2, -0.9, 0.1, 60.0, 30.0)
    assert "delta" in lib.chert_last_error().decode()


def test_moduli_to_class_table2_layer1(lib):
    """Eq. 2 in the library for the paper's Table 2 layer 1 (moduli in
    (km/s)^2 and one Q per component): aI = aR / Q, an infinite Q elastic."""
    aR = [14.40e6, 4.50e6, 9.00e6, 2.25e6, 3.00e6]
    q = [30.0, 15.0, 20.0, 15.0, 12.0]
    c = chert.table_class(aR, q, tilt=0.25)
    assert list(c.aR) == aR
    assert list(c.aI) == [0.48e6, 0.3e6, 0.45e6, 0.15e6, 0.25e6]
    assert c.tilt == 0.25 and c.rho == 2200.0
    c = chert.table_class(aR, [math.inf] * 5)
    assert list(c.aI) == [0.0] * 5
    with pytest.raises(chert.ChertError) as e:
        chert.table_class(aR, [30.0, 15.0, 0.0, 15.0, 12.0])
    assert e.value.code == chert.EINVAL and "component 2" in lib.chert_last_error().decode()


def test_workspace_query(lib):
    a = chert.workspace_bytes(3, 8, 80, chert.FP32, 64)
    b = chert.workspace_bytes(3, 8, 80, chert.FP64, 64)
    assert 0 < a < b and a % 256 == 0
    assert chert.workspace_bytes(0, 8, 80, chert.FP32, 64) == 0


def test_workspace_grid_adds_per_node_area(lib):
    """The lattice-aware query adds the per-node weight area only where the
    class-pair table cannot hold the classes and the stencil is standard."""
    base = chert.workspace_bytes(3, 8, 80, chert.FP32, 64)
    assert chert.workspace_bytes(3, 8, 80, chert.FP32, 64, 401, 401) == base
    n = 100 * 60
    small = chert.workspace_bytes(3, n, 80, chert.FP32, 4)
    big = chert.workspace_bytes(3, n, 80, chert.FP32, 4, 100, 60)
    assert big - small >= 2 * (3 * 2 * 80 * n * 4)          # row and column layouts
    assert chert.workspace_bytes(3, n, 80, chert.FP64, 4, 100, 60) - chert.workspace_bytes(3, n, 80, chert.FP64, 4) \
        >= 2 * (3 * 2 * 80 * n * 8)
    assert chert.workspace_bytes(3, n, 84, chert.FP32, 4, 100, 60) == chert.workspace_bytes(3, n, 84, chert.FP32, 4)
    # 3D lattices have no per-node area: the class tables only
    assert lib.chert_traveltime_workspace_bytes_grid(3, n, 80, chert.FP32, 4, 100, 2, 60) == small
    assert lib.chert_traveltime_workspace_bytes_grid(3, n, 80, chert.FP32, 4, 100, 0, 60) == 0


def test_null_arguments_are_rejected_without_gpu(lib):
    assert lib.chert_build_cache(None, 1, None, 1, None, None, None) == chert.EINVAL
    assert lib.chert_raypath(None, 1, 10, None, None, 1, 4, None, None, None) == chert.EINVAL


def test_relax_scheduler_switch_host_only(lib):
    """The 2D scheduler switch is host state: the hybrid is the default, a
    negative argument queries, out-of-range values are refused, and every
    change returns the previous setting."""
    assert lib.chert_set_relax_scheduler(-1) == 2
    assert chert.relax_scheduler() == "hybrid"
    assert lib.chert_set_relax_scheduler(4) == chert.EINVAL
    assert lib.chert_set_relax_scheduler(-1) == 2                # unchanged by the refusal
    try:
        assert chert.set_relax_scheduler("block_heap") == "hybrid"
        assert lib.chert_set_relax_scheduler(0) == 1
        assert chert.relax_scheduler() == "sweeps"
        assert chert.set_relax_scheduler("frontier") == "sweeps"
        assert lib.chert_set_relax_scheduler(-1) == 3
        with pytest.raises(ValueError):
            chert.set_relax_scheduler("dijkstra")
    finally:
        chert.set_relax_scheduler("hybrid")
    assert chert.relax_scheduler() == "hybrid"


def test_relax_points_per_thread_switch_host_only(lib):
    assert lib.chert_set_relax_points_per_thread(3) == chert.EINVAL
    prev = lib.chert_set_relax_points_per_thread(2)
    assert lib.chert_set_relax_points_per_thread(prev) == 2


def test_tracer_counts_the_hybrid_continuation(lib):
    """The launch count a Tracer reports follows the scheduler: the hybrid
    adds its continuation only where the library launches it (stencil reach
    <= 8 and max_cycles > 6)."""
    import numpy as np
    from paper_2609_26108_b300 import inputs
    from paper_2609_26108_b300.pipeline import Tracer
    tr = Tracer.__new__(Tracer)                     # host state only, no device buffers
    tr.offsets = np.asarray(inputs.stencil_2d(5), np.int32).reshape(-1, 3)
    tr.max_cycles = 64
    tr.nx = tr.nz = 401
    tr.scan_half = 30000
    # main and finish pass of the cache build, lookup, class check, row-class
    # check, relaxation, 2 raypaths (+ the hybrid's continuation)
    try:
        chert.set_relax_scheduler("hybrid")
        assert tr.launches_per_run == 9
        tr.max_cycles = 6
        assert tr.launches_per_run == 8
        tr.max_cycles = 64
        chert.set_relax_scheduler("sweeps")
        assert tr.launches_per_run == 8
        chert.set_relax_scheduler("block_heap")                # no sweeps: no row-class check
        assert tr.launches_per_run == 7
        chert.set_relax_scheduler("sweeps")
        tr.scan_half = 2000                          # no finish pass
        assert tr.launches_per_run == 7
        tr.nx = 2049                                 # lines too long for the specialised kernel
        assert tr.launches_per_run == 6
    finally:
        chert.set_relax_scheduler("hybrid")


def test_new_switches_and_sizes_host_only(lib):
    """Process-wide launch-shape switches refuse values they do not know and
    return the previous setting; workspace queries refuse bad sizes; argument
    checks run before any device work."""
    import ctypes
    assert lib.chert_set_relax3d_tile(2) == chert.EINVAL
    prev = lib.chert_set_relax3d_tile(1)
    assert lib.chert_set_relax3d_tile(prev) == 1
    assert lib.chert_set_cache_finish_threads(128) == chert.EINVAL
    prev = lib.chert_set_cache_finish_threads(512)
    assert lib.chert_set_cache_finish_threads(prev) == 512
    # the surrogate cache with its device-side fallback list: the network's
    # scratch plus one int64 per solve and the counter
    s1 = lib.chert_surrogate_cache_workspace_bytes(10, 30)
    s2 = lib.chert_cache_surrogate_workspace_bytes(10, 3, 30)
    assert s1 > 0 and s2 >= s1 + 8 * 3 * 10 * 31 + 8
    assert lib.chert_cache_surrogate_workspace_bytes(10, 4, 30) == 0
    assert lib.chert_cache_surrogate_workspace_bytes(0, 3, 30) == 0
    # argument checks before any launch
    assert lib.chert_traveltime_batch(None, 1, 1, chert.FP64, None, 0, 8, None, None) == chert.EINVAL
    arr = (chert.chert_lattice * 49)()
    off = (ctypes.c_int32 * 3)(1, 0, 0)
    ctr = ctypes.c_void_p(8)                                   # never dereferenced: the count is refused first
    assert lib.chert_traveltime_batch(arr, 49, 1, chert.FP64, off, 1, 8, ctr, None) == chert.EINVAL
    assert "n_lattices" in lib.chert_last_error().decode()
    assert lib.chert_angular_coverage(None, 1, 1, 8, chert.FP32, None, 0, None, None, None, None, None) == chert.EINVAL
    assert lib.chert_mlp_set_wait_limit(-1) in (1 << 22, chert.ECUDA)


def test_autotuner_keeps_the_first_shape_on_a_tie():
    """The launch-shape choice of the autotuners: the smallest candidate unless
    another is faster by more than 3%, so timing noise does not flip it."""
    from paper_2609_26108_b300.pipeline import _pick
    assert _pick({1: 7.27, 2: 7.27, 4: 7.88}) == 1
    assert _pick({1: 7.27, 2: 7.10, 4: 7.88}) == 1            # 2.3% faster: a tie
    assert _pick({1: 8.00, 2: 7.50, 4: 7.90}) == 2
    assert _pick({0: 1490.0, 1: 1440.0}) == 1                  # 3.4% faster
