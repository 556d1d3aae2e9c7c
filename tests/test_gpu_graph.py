"""The capturable relaxation (chert_traveltime_enqueue) and the CUDA-graph
batch runner: the same fields, parents and raypaths as the eager calls, bit
for bit, on a batch that mixes a 2D layered problem, a 2D per-cell problem
and a 3D problem; the device status words report cycle caps."""
import math

import numpy as np
import pytest

from paper_2609_26108_b300 import chert, inputs
from paper_2609_26108_b300.pipeline import GraphBatch, Problem

pytestmark = pytest.mark.gpu
DEG = math.pi / 180


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    from paper_2609_26108_b300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def _layered(torch, n_sources=5):
    m = inputs.layered_tti(nx=61, nz=47, n_layers=4, n_sources=n_sources)
    d_classes = chert.classes_to_device(chert.classes_from_layers(m.layers))
    d_cls = torch.as_tensor(m.class_of_node.astype(np.int32), device="cuda")
    return m, d_classes, d_cls


def test_enqueue_matches_traveltime(torch_dev):
    m, d_classes, d_cls = _layered(torch_dev)
    cache = chert.build_cache(d_classes, len(m.layers), ["qP", "qSV"], 12, 0.02 * DEG, 1500, "MEV", "mixed")
    off = inputs.stencil_2d(5)
    ref = chert.traveltime(cache, m.nx, m.nz, m.dx, d_cls, off, m.sources)
    out = tuple(torch_dev.empty_like(t) for t in ref)
    ws = torch_dev.empty(chert.workspace_bytes(2, len(m.layers), len(off), cache.precision, len(m.sources),
                                               m.nx, m.nz), dtype=torch_dev.uint8, device="cuda")
    status = torch_dev.full((2,), 7, dtype=torch_dev.int32, device="cuda")
    d_src = torch_dev.as_tensor(m.sources, device="cuda")
    chert.traveltime_enqueue(cache, m.nx, m.nz, m.dx, d_cls, off, d_src, out, ws, status)
    torch_dev.cuda.synchronize()
    for a, b in zip(ref, out):
        assert torch_dev.equal(a, b)
    assert status.cpu().tolist() == [-1, 0]
    # a cap of one cycle: the attenuation fields need more, the status names one
    chert.traveltime_enqueue(cache, m.nx, m.nz, m.dx, d_cls, off, d_src, out, ws, status, max_cycles=1)
    torch_dev.cuda.synchronize()
    first, bad = status.cpu().tolist()
    assert bad == 0 and first >= 0


def test_graph_batch_replays_eager_results(torch_dev):
    probs = []
    m, d_classes, d_cls = _layered(torch_dev, 4)
    probs.append(Problem(d_classes, len(m.layers), ["qP", "qSV", "qSH"], m.nx, m.nz, m.dx, d_cls,
                         inputs.stencil_2d(5), m.sources, receivers=[0, 30, m.nx * m.nz - 1], M=12,
                         scan_step=0.02 * DEG, scan_half=1500))
    fm = inputs.folded_faulted(nx=71, nz=33, n_layers=4, n_sources=3, seed=7)
    n = fm.nx * fm.nz
    keys = ["vp0", "vs0", "eps", "delta", "gamma", "qp", "qs", "tilt"]
    d_cells = chert.classes_to_device(chert.classes_from_arrays(**{k: fm.params[k] for k in keys}))
    probs.append(Problem(d_cells, n, ["qP", "qSV"], fm.nx, fm.nz, fm.dx,
                         torch_dev.as_tensor(np.arange(n, dtype=np.int32), device="cuda"), inputs.stencil_2d(5),
                         fm.sources, M=12, scan_step=0.02 * DEG, scan_half=1500))
    m3 = inputs.layered_tti_3d(n=17, n_layers=3, n_sources=4)
    d3 = chert.classes_to_device(chert.classes_from_layers(m3.layers))
    probs.append(Problem(d3, len(m3.layers), ["qP", "qSV"], m3.nx, m3.nz, m3.dx,
                         torch_dev.as_tensor(m3.class_of_node, device="cuda"), inputs.stencil_3d(2), m3.sources,
                         receivers=[0, 17 ** 3 - 1], n_az=24, n_pol=12, ny=m3.ny, cache_precision="fp64",
                         scan_step=0.02 * DEG, scan_half=1500))
    batch = GraphBatch(probs)
    batch.run_eager()
    torch_dev.cuda.synchronize()
    batch.check()
    eager = [[t.clone() for t in batch.fields(i)] for i in range(len(probs))]
    eager_paths = [[t.clone() for t in st["paths"]] if "paths" in st else None for st in batch.state]
    batch.capture()
    for _ in range(2):
        for st in batch.state:                          # clobber the outputs between replays
            for t in st["tau"]:
                t.fill_(0)
        batch.replay()
        torch_dev.cuda.synchronize()
        batch.check()
        for i in range(len(probs)):
            for a, b in zip(eager[i], batch.fields(i)):
                assert torch_dev.equal(a, b)
            if eager_paths[i] is not None:
                for a, b in zip(eager_paths[i], batch.state[i]["paths"]):
                    assert torch_dev.equal(a, b)
    assert batch.n_fields == 4 * 3 + 3 * 2 + 4 * 2


def test_persistent_batch_with_surrogate_and_autotuner(torch_dev):
    """The batched form of many problems: a per-cell 2D problem whose cache
    comes from the surrogate with its exact fallback (chert_cache_surrogate)
    and a layered 2D problem, relaxed together by one batch call (persistent
    launches of the specialised kernel), and three 3D blocks of uneven size
    cut from one model (one shared cache build) relaxed in one persistent
    launch; launch shapes chosen by the batch's autotuner, then the whole
    batch captured in one CUDA graph.  Replays equal the eager pass bit for bit, and every
    problem's fields equal chert_traveltime on its own cache."""
    torch = torch_dev
    from test_gpu_surrogate import _decisive_nets
    params = _decisive_nets(torch)
    fm = inputs.folded_faulted(nx=71, nz=33, n_layers=4, n_sources=3, seed=7)
    n = fm.nx * fm.nz
    keys = ["vp0", "vs0", "eps", "delta", "gamma", "qp", "qs", "tilt"]
    d_cells = chert.classes_to_device(chert.classes_from_arrays(**{k: fm.params[k] for k in keys}))
    d_own = torch.as_tensor(np.arange(n, dtype=np.int32), device="cuda")
    probs = [Problem(d_cells, n, ["qP", "qSV", "qSH"], fm.nx, fm.nz, fm.dx, d_own, inputs.stencil_2d(5),
                     fm.sources, receivers=[0, 500, n - 1], M=30, scan_step=0.02 * DEG, scan_half=1500,
                     surrogate_params=params)]
    big = inputs.layered_tti_3d(n=41, n_layers=3, n_sources=4)
    d3 = chert.classes_to_device(chert.classes_from_layers(big.layers))
    for size, seed in ((21, 1), (15, 2), (27, 3)):
        sub = inputs.subvolume_3d(big, size, seed=seed, n_sources=4)
        probs.append(Problem(d3, len(big.layers), ["qP", "qSV"], sub.nx, sub.nz, sub.dx,
                             torch.as_tensor(sub.class_of_node, device="cuda"), inputs.stencil_3d(2), sub.sources,
                             receivers=[0, size ** 3 - 1], n_az=24, n_pol=12, ny=sub.ny, cache_precision="mixed",
                             relax_precision="fp32_acc64", scan_step=0.02 * DEG, scan_half=1500))
    m = inputs.layered_tti(nx=61, nz=47, n_layers=4, n_sources=3)
    probs.append(Problem(chert.classes_to_device(chert.classes_from_layers(m.layers)), len(m.layers),
                         ["qP", "qSV", "qSH"], m.nx, m.nz, m.dx,
                         torch.as_tensor(m.class_of_node.astype(np.int32), device="cuda"), inputs.stencil_2d(5),
                         m.sources, receivers=[0, 30, m.nx * m.nz - 1], M=30, scan_step=0.02 * DEG, scan_half=1500))
    batch = GraphBatch(probs, persistent_3d=True, persistent_2d=True)
    assert batch.cache_owner == [0, 1, 1, 1, 4]
    assert [sorted(g["members"]) for g in batch.groups] == [[1, 2, 3], [0, 4]]
    prev_tile = chert.set_relax3d_tile(0)
    prev_ppt = chert.lib().chert_set_relax_points_per_thread(0)
    try:
        batch.run_eager()
        torch.cuda.synchronize()
        batch.check()
        tuned = batch.autotune()
        assert set(tuned["tile3d"]) == {0, 1} and tuned["chosen"]["ppt2d"] in (1, 2, 4)
        batch.run_eager()
        torch.cuda.synchronize()
        eager = [[t.clone() for t in batch.fields(i)] for i in range(len(probs))]
        eager_paths = [[t.clone() for t in st["paths"]] for st in batch.state]
        # each problem alone, on the batch's caches
        for i, p in enumerate(probs):
            cache = batch.state[batch.cache_owner[i]]["cache"]
            ref = chert.traveltime(cache, p.nx, p.nz, p.dx, p.d_cls, p.offsets, p.sources, max_cycles=p.max_cycles,
                                   ny=p.ny, precision=p.relax_precision)
            torch.cuda.synchronize()
            for a, b in zip(ref, eager[i]):
                assert torch.equal(a, b), i
        assert int(batch.state[0]["cache"].n_fallback_dev.item()) > 0
        batch.capture(warm=False)
        for _ in range(2):
            for st in batch.state:
                for t in st["tau"]:
                    t.fill_(0)
            batch.replay()
            torch.cuda.synchronize()
            batch.check()
            for i in range(len(probs)):
                for a, b in zip(eager[i], batch.fields(i)):
                    assert torch.equal(a, b)
                for a, b in zip(eager_paths[i], batch.state[i]["paths"]):
                    assert torch.equal(a, b)
    finally:
        chert.set_relax3d_tile(prev_tile)
        chert.lib().chert_set_relax_points_per_thread(prev_ppt)
