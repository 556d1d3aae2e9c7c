"""Block-heap marching (Eq. 32) and the hybrid scheduler (a few sweep cycles,
then block-heap marching for the fields not yet converged) against the sweeps
and the oracle.

Every scheduler stops only at the fixed point of Eq. 31, which is unique: a
node's value is the least rounded path sum, whatever order the edges are
relaxed in, and its parent the least-index argmin there.  So all must give
the same fields and parents bit for bit, in either precision; FP64 is also
checked against the oracle's Dijkstra."""
import math

import numpy as np
import pytest

from paper_2609_26108_b300 import chert, inputs

from test_gpu_relax import (_check_fields, _serpentine, _synthetic_cache, as_cache, oracle_fields, run_gpu,
                            small_oracle_cache)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    from paper_2609_26108_b300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def both(torch, cache, nx, nz, cls, off, src, max_cycles=256, dx=10.0):
    out = {}
    prev = chert.relax_scheduler()
    try:
        for name in ("sweeps", "block_heap", "hybrid"):
            chert.set_relax_scheduler(name)
            out[name] = run_gpu(torch, cache, nx, nz, dx, cls, off, src, max_cycles)
    finally:
        chert.set_relax_scheduler(prev)
    for other in ("block_heap", "hybrid"):
        for a, b in zip(out["sweeps"], out[other]):
            assert np.array_equal(a, b), other
    return out["block_heap"]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_layered_equals_sweeps(torch_dev, precision):
    """Five-class layered lattice of 5 x 4 blocks with ragged edges, R = 5
    stencil (class-pair table in shared memory), sources at a corner, inside
    and at the opposite corner."""
    nx, nz = 151, 97
    cls = inputs.layered_class_map_2d(nx, nz, 5).astype(np.int32)
    off = inputs.stencil_2d(5)
    cache = as_cache(torch_dev, small_oracle_cache(), precision)
    src = [0, 77 + nx * 40, nx * nz - 1]
    g = both(torch_dev, cache, nx, nz, cls, off, src)
    if precision == "fp64":
        ref = oracle_fields(small_oracle_cache(), precision, (nx, 1, nz), 10.0, cls, off, src)
        _check_fields(g, ref, src, 2, precision, (nx, 1, nz), 10.0, cls, off, small_oracle_cache())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_serpentine_many_block_passes(torch_dev, precision):
    """A fast channel with 12 bends across 9 x 4 blocks: blocks are taken
    many times each, in an order set by the keys; the oracle's field and
    parents all the same."""
    nx, nz = 280, 120
    cls = _serpentine(nx, nz, 12)
    cnp = _synthetic_cache([150.0, 6000.0], [1e-3, 1e-5])
    off = inputs.stencil_2d(3)
    src = [2 + nx * 1]
    g = both(torch_dev, as_cache(torch_dev, cnp, precision), nx, nz, cls, off, src)
    ref = oracle_fields(cnp, precision, (nx, 1, nz), 10.0, cls, off, src)
    _check_fields(g, ref, src, 1, precision, (nx, 1, nz), 10.0, cls, off, cnp)


def test_one_class_per_node_global_tables(torch_dev):
    """One class per node: the looked-up tables stay in global memory."""
    nx, nz = 150, 70
    n = nx * nz
    rng = np.random.default_rng(43)
    M = 6
    nd = 4 * M
    th = (math.pi / 2) * np.arange(nd) / M
    chan = _serpentine(nx, nz, 6).astype(bool)
    v0 = np.where(chan, 5200.0, 1400.0) * rng.uniform(0.97, 1.03, n)
    aniso = rng.uniform(-0.15, 0.15, n)
    V = v0[:, None] * (1 + aniso[:, None] * np.cos(2 * th)[None])
    a0 = np.where(chan, 1e-5, 3e-4) * rng.uniform(0.9, 1.1, n)
    cnp = {"V": V[None], "A": (a0[:, None] * np.ones(nd))[None],
           "rx": np.tile(np.sin(th), (1, n, 1)), "rz": np.tile(np.cos(th), (1, n, 1)),
           "theta": np.tile(th, (1, n, 1)), "vartheta": np.zeros((1, n, nd)),
           "flag": np.zeros((1, n, nd), np.uint8)}
    cnp["Q"] = np.full_like(cnp["V"], np.inf)
    off = inputs.stencil_2d(5)
    cls = np.arange(n, dtype=np.int32)
    src = [2 + nx * 1, 77 + nx * 40]
    for precision in ("fp64", "fp32"):
        g = both(torch_dev, as_cache(torch_dev, cnp, precision), nx, nz, cls, off, src)
        if precision == "fp64":
            ref = oracle_fields(cnp, precision, (nx, 1, nz), 10.0, cls, off, src)
            _check_fields(g, ref, src, 1, precision, (nx, 1, nz), 10.0, cls, off, cnp)


@pytest.mark.parametrize("shape", [(1, 1), (1, 40), (40, 1), (33, 2), (32, 32), (65, 33)])
def test_degenerate_and_ragged_lattices(torch_dev, shape):
    """Single node, single row or column, one block plus a one-node tail."""
    nx, nz = shape
    cls = (np.arange(nx * nz) % 2).astype(np.int32)
    cnp = _synthetic_cache([2000.0, 3000.0], [1e-4, 2e-4])
    off = inputs.stencil_2d(2)
    src = [0, nx * nz - 1]
    both(torch_dev, as_cache(torch_dev, cnp, "fp64"), nx, nz, cls, off, src)


def test_unreachable_nodes_keep_infinity(torch_dev):
    """Offsets that move two columns at a time never reach the odd columns:
    those stay +inf with parent -1 under both schedulers, across several
    blocks."""
    nx, nz = 90, 40
    off = np.array([(2, 0, 0), (-2, 0, 0), (0, 0, 1), (0, 0, -1)], np.int32)
    cls = np.zeros(nx * nz, np.int32)
    cnp = _synthetic_cache([3000.0], [2e-5])
    tR, _, pR, _, _, _ = both(torch_dev, as_cache(torch_dev, cnp, "fp64"), nx, nz, cls, off, [4])
    odd = (np.arange(nx * nz) % nx) % 2 == 1
    assert np.all(np.isinf(tR[0, 0, odd])) and np.all(pR[0, 0, odd] == -1)
    assert np.all(np.isfinite(tR[0, 0, ~odd]))


def test_scheduler_switch_rejects_unknown(torch_dev):
    with pytest.raises(ValueError):
        chert.set_relax_scheduler("heap")
    assert chert.lib().chert_set_relax_scheduler(4) == chert.EINVAL
    assert chert.relax_scheduler() == "hybrid"                 # the default
    assert chert.set_relax_scheduler("sweeps") == "hybrid"
    assert chert.relax_scheduler() == "sweeps"
    assert chert.set_relax_scheduler("hybrid") == "sweeps"


def test_block_scheduler_rejects_long_stencils(torch_dev):
    """A stencil that reaches beyond the staged halo (9 > 8 nodes) is refused
    with CHERT_EINVAL under the block scheduler, and runs under the sweeps."""
    nx, nz = 40, 30
    cls = np.zeros(nx * nz, np.int32)
    cache = as_cache(torch_dev, _synthetic_cache([3000.0], [2e-5]), "fp64")
    off = np.array([(9, 0, 1), (-9, 0, -1), (1, 0, 0), (-1, 0, 0), (0, 0, 1), (0, 0, -1)], np.int32)
    d_cls = torch_dev.as_tensor(cls, device="cuda")
    try:
        chert.set_relax_scheduler("block_heap")
        with pytest.raises(chert.ChertError) as e:
            chert.traveltime(cache, nx, nz, 10.0, d_cls, off, [0])
        assert e.value.code == chert.EINVAL
        chert.set_relax_scheduler("hybrid")          # sweeps only
        hy = [t.cpu() for t in chert.traveltime(cache, nx, nz, 10.0, d_cls, off, [0])]
        chert.set_relax_scheduler("sweeps")
        sw = [t.cpu() for t in chert.traveltime(cache, nx, nz, 10.0, d_cls, off, [0])]
    finally:
        chert.set_relax_scheduler("hybrid")
    for a, b in zip(sw, hy):
        assert torch_dev.equal(a, b)


def test_hybrid_continues_unconverged_fields(torch_dev):
    """A serpentine channel that needs more than 6 sweep cycles: under the
    hybrid scheduler with max_cycles = 7 (6 sweep cycles, then block-heap
    marching with a budget of 7) the continuation finishes it with the
    sweeps' fixed point and parents."""
    nx, nz = 280, 120
    cls = _serpentine(nx, nz, 12)
    cache = as_cache(torch_dev, _synthetic_cache([150.0, 6000.0], [1e-3, 1e-5]), "fp64")
    off = inputs.stencil_2d(3)
    src = [2 + nx * 1]
    d_cls = torch_dev.as_tensor(cls, device="cuda")
    try:
        chert.set_relax_scheduler("sweeps")
        with pytest.raises(chert.ChertError) as e:   # the sweeps alone need more than 6 cycles
            chert.traveltime(cache, nx, nz, 10.0, d_cls, off, src, max_cycles=6)
        assert e.value.code == chert.ETIMEOUT
        ref = run_gpu(torch_dev, cache, nx, nz, 10.0, cls, off, src, max_cycles=256)
    finally:
        chert.set_relax_scheduler("hybrid")
    g = [t.cpu().numpy() for t in chert.traveltime(cache, nx, nz, 10.0, d_cls, off, src, max_cycles=7)]
    for a, b in zip(ref, g):
        assert np.array_equal(a, b)


def test_hybrid_continuation_on_per_node_weights(torch_dev):
    """One class per node on the 12-bend serpentine: the sweeps use per-node
    weights and need more than 6 cycles, so the hybrid's continuation runs
    the standard-stencil block-heap kernel on those per-node weights; the
    fields and parents equal the sweeps'."""
    nx, nz = 280, 120
    n = nx * nz
    chan = _serpentine(nx, nz, 12).astype(bool)
    rng = np.random.default_rng(47)
    M = 6
    nd = 4 * M
    th = (math.pi / 2) * np.arange(nd) / M
    v0 = np.where(chan, 6000.0, 150.0) * rng.uniform(0.98, 1.02, n)
    a0 = np.where(chan, 1e-5, 1e-3) * rng.uniform(0.9, 1.1, n)
    cnp = {"V": np.repeat(v0[None, :, None], nd, 2), "A": np.repeat(a0[None, :, None], nd, 2),
           "rx": np.tile(np.sin(th), (1, n, 1)), "rz": np.tile(np.cos(th), (1, n, 1)),
           "theta": np.tile(th, (1, n, 1)), "vartheta": np.zeros((1, n, nd)),
           "flag": np.zeros((1, n, nd), np.uint8)}
    cnp["Q"] = np.full_like(cnp["V"], np.inf)
    off = inputs.stencil_2d(3)
    cls = np.arange(n, dtype=np.int32)
    src = [2 + nx * 1]
    d_cls = torch_dev.as_tensor(cls, device="cuda")
    for precision in ("fp64", "fp32"):
        cache = as_cache(torch_dev, cnp, precision)
        try:
            chert.set_relax_scheduler("sweeps")
            with pytest.raises(chert.ChertError) as e:
                chert.traveltime(cache, nx, nz, 10.0, d_cls, off, src, max_cycles=6)
            assert e.value.code == chert.ETIMEOUT
            ref = run_gpu(torch_dev, cache, nx, nz, 10.0, cls, off, src, max_cycles=256)
        finally:
            chert.set_relax_scheduler("hybrid")
        g = [t.cpu().numpy() for t in chert.traveltime(cache, nx, nz, 10.0, d_cls, off, src, max_cycles=7)]
        for a, b in zip(ref, g):
            assert np.array_equal(a, b)


def frontier_equals_sweeps(torch, cache, nx, nz, cls, off, src, max_cycles=256):
    out = {}
    prev = chert.relax_scheduler()
    try:
        for name in ("sweeps", "frontier"):
            chert.set_relax_scheduler(name)
            out[name] = run_gpu(torch, cache, nx, nz, 10.0, cls, off, src, max_cycles)
    finally:
        chert.set_relax_scheduler(prev)
    for a, b in zip(out["sweeps"], out["frontier"]):
        assert np.array_equal(a, b)
    return out["frontier"]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_frontier_label_correcting_equals_sweeps(torch_dev, precision):
    """The frontier label-correcting scheduler (atomicMin pushes on the
    traveltimes' bit patterns) against the sweeps, bit for bit: a layered
    lattice with ragged edges (FP64 also against the oracle), a 12-bend
    serpentine whose paths turn many times, and degenerate shapes."""
    nx, nz = 151, 97
    cls = inputs.layered_class_map_2d(nx, nz, 5).astype(np.int32)
    off = inputs.stencil_2d(5)
    cache = as_cache(torch_dev, small_oracle_cache(), precision)
    src = [0, 77 + nx * 40, nx * nz - 1]
    g = frontier_equals_sweeps(torch_dev, cache, nx, nz, cls, off, src)
    if precision == "fp64":
        ref = oracle_fields(small_oracle_cache(), precision, (nx, 1, nz), 10.0, cls, off, src)
        _check_fields(g, ref, src, 2, precision, (nx, 1, nz), 10.0, cls, off, small_oracle_cache())
    nx, nz = 280, 120
    frontier_equals_sweeps(torch_dev, as_cache(torch_dev, _synthetic_cache([150.0, 6000.0], [1e-3, 1e-5]), precision),
                           nx, nz, _serpentine(nx, nz, 12), inputs.stencil_2d(3), [2 + nx * 1])
    for nx, nz in ((1, 1), (1, 40), (40, 1), (33, 2)):
        frontier_equals_sweeps(torch_dev, as_cache(torch_dev, _synthetic_cache([2000.0, 3000.0], [1e-4, 2e-4]),
                                                   precision),
                               nx, nz, (np.arange(nx * nz) % 2).astype(np.int32), inputs.stencil_2d(2),
                               [0, nx * nz - 1])


def test_frontier_round_cap_reports_timeout(torch_dev):
    """The frontier scheduler runs at most max_cycles x max(nx, nz) rounds: on
    the 12-bend serpentine, whose shortest paths take far more than 280 hops,
    max_cycles = 1 stops it and the call reports CHERT_ETIMEOUT; the same
    context then relaxes the field to the sweeps' fixed point."""
    nx, nz = 280, 120
    cls = _serpentine(nx, nz, 12)
    cache = as_cache(torch_dev, _synthetic_cache([150.0, 6000.0], [1e-3, 1e-5]), "fp32")
    off = inputs.stencil_2d(3)
    src = [2 + nx * 1]
    d_cls = torch_dev.as_tensor(cls, device="cuda")
    prev = chert.set_relax_scheduler("frontier")
    try:
        with pytest.raises(chert.ChertError) as e:
            chert.traveltime(cache, nx, nz, 10.0, d_cls, off, src, max_cycles=1)
        assert e.value.code == chert.ETIMEOUT
    finally:
        chert.set_relax_scheduler(prev)
    frontier_equals_sweeps(torch_dev, cache, nx, nz, cls, off, src)
