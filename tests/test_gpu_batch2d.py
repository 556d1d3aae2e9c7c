"""chert_traveltime_batch on 2D lattices: lattices of uneven size and launch
shape (the row-class path, the class-pair table, per-node weights, one, two
and four nodes a thread) grouped into persistent launches (a group of more
than 24 lattices of one shape split over launches), against
chert_traveltime on each lattice alone under the sweeps scheduler: fields and
parents bit for bit, status [-1, 0] for each; also captured in a CUDA graph.
A stencil other than radius 5 is relaxed lattice by lattice, with the same
results."""
import numpy as np
import pytest

from paper_2609_26108_b300 import chert, inputs

from test_gpu_relax import as_cache, small_oracle_cache

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    from paper_2609_26108_b300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def _cache(torch, precision, n_classes):
    """The oracle's small cache (5 classes, qP and qSV), its classes repeated
    to n_classes (many classes: the class-pair table no longer fits, so the
    kernel takes per-node weights)."""
    c = small_oracle_cache()
    if n_classes != 5:
        reps = np.arange(n_classes) % 5
        c = {k: v[:, reps] for k, v in c.items()}
    return as_cache(torch, c, precision)


def _item(torch, precision, nx, nz, cls, sources, n_classes, off):
    cache = _cache(torch, precision, n_classes)
    nm, n = len(cache.modes), nx * nz
    fd = torch.float64 if precision == "fp64" else torch.float32
    ns = len(sources)
    out = (torch.full((ns, nm, n), -3.0, dtype=fd, device="cuda"), torch.full((ns, nm, n), -3.0, dtype=fd, device="cuda"),
           torch.full((ns, nm, n), -7, dtype=torch.int32, device="cuda"),
           torch.full((ns, nm, n), -7, dtype=torch.int32, device="cuda"))
    ws = torch.empty(chert.workspace_bytes(nm, n_classes, len(off), cache.precision, ns, nx, nz), dtype=torch.uint8,
                     device="cuda")
    return {"cache": cache, "nx": nx, "ny": 1, "nz": nz, "dx": 10.0,
            "d_cls": torch.as_tensor(np.asarray(cls, np.int32), device="cuda"),
            "d_sources": torch.as_tensor(np.asarray(sources, np.int64), device="cuda"), "out": out, "workspace": ws,
            "d_status": torch.full((2,), 5, dtype=torch.int32, device="cuda")}


def _cases(torch, precision, off):
    rng = np.random.default_rng(3)
    return [
        _item(torch, precision, 151, 97, inputs.layered_class_map_2d(151, 97, 5), [0, 77 + 151 * 40, 151 * 97 - 1], 5,
              off),                                                         # row-class path
        _item(torch, precision, 90, 60, rng.integers(0, 5, 90 * 60), [5, 2000], 5, off),     # class-pair table
        _item(torch, precision, 70, 50, rng.integers(0, 400, 70 * 50), [10, 3000], 400, off),  # per-node weights
        _item(torch, precision, 600, 40, inputs.layered_class_map_2d(600, 40, 5), [3, 599], 5, off),  # 2 nodes a thread
        _item(torch, precision, 64, 33, inputs.layered_class_map_2d(64, 33, 5), [0], 5, off),
        _item(torch, precision, 1100, 24, inputs.layered_class_map_2d(1100, 24, 5), [7, 1100 * 12 + 1099], 5,
              off),                                                         # 4 nodes a thread
    ]


def _check(torch, items, off):
    prev = chert.set_relax_scheduler("sweeps")
    try:
        for it in items:
            assert it["d_status"].cpu().tolist() == [-1, 0]
            ref = chert.traveltime(it["cache"], it["nx"], it["nz"], 10.0, it["d_cls"], off, it["d_sources"].cpu().numpy())
            torch.cuda.synchronize()
            for a, b in zip(ref, it["out"]):
                assert torch.equal(a, b), (it["nx"], it["nz"])
    finally:
        chert.set_relax_scheduler(prev)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_of_uneven_2d_lattices_equals_single_calls(torch_dev, precision):
    torch = torch_dev
    off = inputs.stencil_2d(5)
    items = _cases(torch, precision, off)
    counter = torch.zeros(1, dtype=torch.int64, device="cuda")
    chert.traveltime_batch(items, off, counter)
    torch.cuda.synchronize()
    _check(torch, items, off)
    # captured in a graph: the same results on two replays
    for it in items:
        for o in it["out"]:
            o.fill_(-1)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        chert.traveltime_batch(items, off, counter, stream=s)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        _check(torch, items, off)


def test_batch_2d_more_lattices_than_one_launch_takes(torch_dev):
    """26 lattices of one launch shape (one launch takes 24): two launches on
    the one counter, each lattice as chert_traveltime relaxes it alone."""
    torch = torch_dev
    off = inputs.stencil_2d(5)
    items = [_item(torch, "fp32", 40 + 3 * i, 21 + i % 5, inputs.layered_class_map_2d(40 + 3 * i, 21 + i % 5, 5),
                   [i, 20 + 3 * i], 5, off) for i in range(26)]
    counter = torch.zeros(1, dtype=torch.int64, device="cuda")
    chert.traveltime_batch(items, off, counter)
    torch.cuda.synchronize()
    _check(torch, items, off)


def test_batch_2d_other_stencil_and_mix_refused(torch_dev):
    """Radius 3: no persistent launch, each lattice on its own (the default
    scheduler), same results as chert_traveltime; a 2D lattice with a 3D one
    is refused."""
    torch = torch_dev
    off = inputs.stencil_2d(3)
    items = _cases(torch, "fp32", off)[:2]
    counter = torch.zeros(1, dtype=torch.int64, device="cuda")
    chert.traveltime_batch(items, off, counter)
    torch.cuda.synchronize()
    for it in items:
        assert it["d_status"].cpu().tolist() == [-1, 0]
        ref = chert.traveltime(it["cache"], it["nx"], it["nz"], 10.0, it["d_cls"], off, it["d_sources"].cpu().numpy())
        torch.cuda.synchronize()
        for a, b in zip(ref, it["out"]):
            assert torch.equal(a, b)
    three = dict(items[0])
    three["ny"], three["nz"] = 3, 97 // 3
    with pytest.raises(chert.ChertError) as e:
        chert.traveltime_batch([items[1], three], off, counter)
    assert e.value.code == chert.EINVAL
