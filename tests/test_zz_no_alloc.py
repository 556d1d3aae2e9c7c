"""chert_traveltime_static, the entry point for callers that cannot allocate
device memory (a host that owns all device memory through its own pool, a
runtime that forbids allocation after start-up): it must give what
chert_traveltime gives, bit for bit and call after call, while its scratch
lives in a fixed array inside libchert.  The kernels are the same, so the
fields and parents must be identical.  This file is collected last on
purpose, so that a run stopping at the first failure has run everything else."""
import numpy as np
import pytest

from paper_2609_26108_b300 import chert, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    from paper_2609_26108_b300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def _problem(torch, precision):
    model = inputs.layered_tti(nx=73, nz=59, n_layers=4, n_sources=5)
    d_classes = chert.classes_to_device(chert.classes_from_layers(model.layers))
    cache = chert.build_cache(d_classes, 4, ["qP", "qSV", "qSH"], 18, 0.02 * np.pi / 180, 1500,
                              "MEV", "mixed" if precision == "fp32" else "fp64")
    d_cls = torch.as_tensor(model.class_of_node.astype(np.int32), device="cuda")
    return model, cache, d_cls


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_static_scratch_matches_workspace_entry_point(torch_dev, precision):
    model, cache, d_cls = _problem(torch_dev, precision)
    off = inputs.stencil_2d(5)
    # two calls in a row with different sources: the shared scratch keeps the
    # first call's contents, which must not leak into the second
    for sources in ([0, 36, 72, 73 * 30 + 10], [5, 73 * 58]):
        ref = chert.traveltime(cache, model.nx, model.nz, model.dx, d_cls, off, sources)
        got = chert.traveltime_static(cache, model.nx, model.nz, model.dx, d_cls, off, sources)
        torch_dev.cuda.synchronize()
        for r, g in zip(ref, got):
            assert torch_dev.equal(r, g)


@pytest.mark.parametrize("side", [16, 20])
def test_static_scratch_one_class_per_node(torch_dev, side):
    """One class per node (per-cell media), so the class-pair table does not
    fit in shared memory: chert_traveltime gets a lattice-sized workspace and
    relaxes on precomputed per-node weights.  On 16 x 16 those weights also
    fit in the static array; on 20 x 20 they do not and the static entry
    point relaxes with the generic kernel.  Either way the fields and parents
    must equal chert_traveltime's, bit for bit."""
    n = side * side
    classes = inputs.random_tti_classes(n, seed=side)
    d_classes = chert.classes_to_device(chert.classes_from_layers(classes))
    cache = chert.build_cache(d_classes, n, ["qP"], 6, 0.02 * np.pi / 180, 1500, "MEV", "mixed")
    d_cls = torch_dev.arange(n, dtype=torch_dev.int32, device="cuda")
    off = inputs.stencil_2d(5)
    prec = chert.FP32
    need = chert.workspace_bytes(1, n, len(off), prec, 2, side, side)
    assert need > chert.workspace_bytes(1, n, len(off), prec, 2)          # the per-node area applies
    limit = chert.lib().chert_traveltime_static_limit()
    assert (need <= limit - 256) == (side == 16)
    for sources in ([0, n - 1], [side // 2 + side * 3, 7]):
        ref = chert.traveltime(cache, side, side, 10.0, d_cls, off, sources, max_cycles=256)
        got = chert.traveltime_static(cache, side, side, 10.0, d_cls, off, sources, max_cycles=256)
        torch_dev.cuda.synchronize()
        for r, g in zip(ref, got):
            assert torch_dev.equal(r, g)


def test_static_scratch_rejects_oversized_problems(torch_dev):
    """A problem whose tables exceed the static array is refused before any
    output is touched, so one-element placeholders stand in for the fields."""
    import ctypes
    model, cache, d_cls = _problem(torch_dev, "fp32")
    off = np.ascontiguousarray(inputs.stencil_2d(5), dtype=np.int32)
    limit = chert.lib().chert_traveltime_static_limit()
    need_per_source = 8 + 3 * 2 * 4
    n = int(limit // need_per_source) + 1000
    src = np.zeros(n, np.int64)
    tiny_f = torch_dev.zeros(1, dtype=torch_dev.float32, device="cuda")
    tiny_i = torch_dev.zeros(1, dtype=torch_dev.int32, device="cuda")
    st = cache.struct()
    P = ctypes.c_void_p
    rc = chert.lib().chert_traveltime_static(
        ctypes.byref(st), 3, 4, cache.n_dir, model.nx, 1, model.nz, float(model.dx), P(d_cls.data_ptr()),
        off.ctypes.data_as(P), len(off), src.ctypes.data_as(P), n, chert.MIXED, 64, P(tiny_f.data_ptr()),
        P(tiny_f.data_ptr()), P(tiny_i.data_ptr()), P(tiny_i.data_ptr()), None)
    assert rc == chert.EINVAL
    assert "scratch" in chert.lib().chert_last_error().decode()
