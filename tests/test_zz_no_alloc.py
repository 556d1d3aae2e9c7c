"""chert_traveltime_static, the entry point for callers that cannot allocate
device memory (allocator-free embeddings, code running under stream capture):
it must give what chert_traveltime gives, call after call, while its scratch
lives in a fixed array inside libchert.  This file is collected last on
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
    rtol = 1e-5 if precision == "fp32" else 1e-12
    # two calls in a row with different sources: the shared scratch keeps the
    # first call's contents, which must not leak into the second
    for sources in ([0, 36, 72, 73 * 30 + 10], [5, 73 * 58]):
        ref = chert.traveltime(cache, model.nx, model.nz, model.dx, d_cls, off, sources)
        got = chert.traveltime_static(cache, model.nx, model.nz, model.dx, d_cls, off, sources)
        torch_dev.cuda.synchronize()
        for r, g in zip(ref[:2], got[:2]):
            r, g = r.cpu().numpy(), g.cpu().numpy()
            assert np.array_equal(np.isfinite(r), np.isfinite(g))
            fin = np.isfinite(r)
            assert np.allclose(g[fin], r[fin], rtol=rtol, atol=0)
        for r, g in zip(ref[2:], got[2:]):
            assert np.array_equal(r.cpu().numpy(), g.cpu().numpy())


def test_static_scratch_rejects_oversized_problems(torch_dev):
    model, cache, d_cls = _problem(torch_dev, "fp32")
    off = inputs.stencil_2d(5)
    limit = chert.lib().chert_traveltime_static_limit()
    need_per_source = 8 + 3 * 2 * 4
    n = int(limit // need_per_source) + 1000
    with pytest.raises(chert.ChertError) as e:
        chert.traveltime_static(cache, model.nx, model.nz, model.dx, d_cls, off, np.zeros(n, np.int64))
    assert e.value.code == chert.EINVAL
    assert "scratch" in str(e.value)
