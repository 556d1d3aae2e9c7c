"""chert_angular_coverage against the coverage oracle: identical counts
(covered directions, branch mismatches, missing angles) per (mode, class),
on the oracle's own caches cast to each precision and on the GPU's MIXED
cache of the benchmark's layered model.  The counts are integer decisions
taken from the same stored entries in the same precision on both sides, so
they must agree exactly."""
import numpy as np
import pytest

from oracle import coverage_oracle as cov
from paper_2609_26108_b300 import chert, inputs

from helpers import DEG, cache_to_torch, golden_cache, load_cache_golden
from test_oracle_coverage import FOLD_PSI, synthetic

pytestmark = pytest.mark.gpu

MODES = ["qP", "qSV", "qSH"]


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    from paper_2609_26108_b300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def as_cache(torch, cnp, precision):
    prec = chert.PRECISION_IDS[precision]
    dt = torch.float64 if prec == chert.FP64 else torch.float32
    arr = cache_to_torch(cnp, dt, "cuda")
    nm, nk, nd = cnp["V"].shape
    return chert.Cache(arr, list(range(nm)), nk, nd // 4, prec)


def gpu_counts(torch, cache, off, truth=None):
    t = None if truth is None else torch.as_tensor(truth, device="cuda").contiguous()
    out = chert.angular_coverage(cache, off, truth_flag=t)
    torch.cuda.synchronize()
    return tuple(o.cpu().numpy().astype(np.int64) for o in out)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("golden,n", [("layered_tti_cache_M90.txt", 8), ("folded_cells_cache_M90.txt", 48)])
def test_coverage_matches_oracle_on_oracle_caches(torch_dev, precision, golden, n):
    g = load_cache_golden(golden)
    tilts = g["tilts"] if g["tilts"] is not None else [p["tilt"] for _, p in g["cells"]]
    cnp = golden_cache(g, MODES, n, tilts)
    dt = np.float64 if precision == "fp64" else np.float32
    cast = {k: (v.astype(dt) if k != "flag" else v) for k, v in cnp.items()}
    off = inputs.stencil_2d(5)
    truth = cnp["flag"].copy()
    truth[:, :, ::7] = 0                       # a reference with more valid entries: some go missing
    ref = cov.coverage_counts(cast, off, dtype=dt, truth_flag=truth)
    got = gpu_counts(torch_dev, as_cache(torch_dev, cnp, precision), off, truth)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    assert np.all(ref[0] <= len(off)) and ref[0].min() > 0


def test_coverage_of_gpu_mixed_cache(torch_dev):
    """The benchmark's MIXED cache (layered 401x401 classes, 1 deg, full
    0.001 deg scan): counts from its own stored entries equal the oracle's
    on the same entries, its flags lose no direction against the FP64
    oracle's (missing = 0), and qP and qSH are fully covered with no
    mismatch."""
    torch = torch_dev
    model = inputs.layered_tti()
    d_classes = chert.classes_to_device(chert.classes_from_layers(model.layers))
    c = chert.build_cache(d_classes, 8, MODES, 90, 0.001 * DEG, 30000, "MEV", "mixed")
    torch.cuda.synchronize()
    g = load_cache_golden("layered_tti_cache_M90.txt")
    truth = golden_cache(g, MODES, 8, g["tilts"])["flag"]
    off = inputs.stencil_2d(5)
    got = gpu_counts(torch, c, off, truth)
    host = {k: v.cpu().numpy() for k, v in c.arrays.items()}
    ref = cov.coverage_counts(host, off, dtype=np.float32, truth_flag=truth)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    assert np.all(got[2] == 0)
    assert np.all(got[0][[0, 2]] == len(off)) and np.all(got[1][[0, 2]] == 0)


def test_coverage_fold_and_errors(torch_dev):
    torch = torch_dev
    V = [1.0] * len(FOLD_PSI)
    V[9] = V[10] = 1.2
    cnp = synthetic(FOLD_PSI, V)
    cnp["Q"] = cnp["theta"] = cnp["vartheta"] = np.zeros_like(cnp["V"])
    arr = {k: torch.as_tensor(v, dtype=torch.float64 if k != "flag" else torch.uint8, device="cuda")
           for k, v in cnp.items()}
    cache = chert.Cache(arr, [0], 1, len(FOLD_PSI) // 4, chert.FP64)       # 20 entries: n_dir = 4M
    off = np.array([[3, 0, 4], [1, 0, 0], [0, 0, 1]], np.int32)
    ref = cov.coverage_counts(cnp, off)
    out = chert.angular_coverage(cache, off)
    torch.cuda.synchronize()
    got = tuple(o.cpu().numpy().astype(np.int64) for o in out)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)
    assert got[0][0, 0] == 3 and got[1][0, 0] == 1
    with pytest.raises(chert.ChertError) as e:
        chert.angular_coverage(cache, np.array([[1, 1, 0]], np.int32))
    assert e.value.code == chert.EINVAL
