"""The small configuration end to end in FP64 against the oracle: the 2D
homogeneous visco-VTI case (one class: Vp0 3000, Vs0 1500, eps 0.2, delta
0.1, gamma 0.1, Qp 60, Qs 30), 1 deg cache (360 directions) at the full
0.001 deg x 30,000 scan, 101 x 101 lattice at dx = 10 m, one centre source,
radius-5 stencil.

* Cache (Eq. 4-14, 26): every solve of qP, qSV and qSH against the oracle's
  stored solves (tests/golden/homogeneous_vti_cache_M90.txt, written by
  tests/golden/make_cache_golden.py from the oracle alone): 1e-9, flags
  identical.
* Traveltimes and parents (Eq. 27-33), qP as the configuration states: the
  GPU's FP64 relaxation on its own cache against the oracle's binary-heap
  Dijkstra on the oracle's cache, through the GPU's lookup choice (a lookup
  that differs must tie with the oracle's to 1e-6 in the dot product).
  Traveltimes to 1e-9 relative: the two caches agree to 1e-9 and every field
  value is a sum of weights taken from them.  Parents identical except at
  nodes where the oracle's two best candidates lie within 1e-9 of each other
  (the cache-level difference can reorder those).
* Raypaths (Eq. 34) to the corners and edge midpoints: identical to the
  oracle's outside those near-ties, and valid shortest-path steps there.
"""
import numpy as np
import pytest

from oracle import graph_oracle as go
from paper_2609_26108_b300 import chert, inputs

from helpers import DEG, golden_cache, load_cache_golden
from test_gpu_fullsize import compare_cache, oracle_lookup

pytestmark = pytest.mark.gpu

MODES = ["qP", "qSV", "qSH"]
M, H, K = 90, 0.001 * DEG, 30000
NEAR = 1e-9


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    from paper_2609_26108_b300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def test_homogeneous_config_fp64_end_to_end(torch_dev):
    torch = torch_dev
    g = load_cache_golden("homogeneous_vti_cache_M90.txt")
    model = inputs.homogeneous_vti()
    assert (model.nx, model.nz, model.dx) == (101, 101, 10.0)
    d_classes = chert.classes_to_device(chert.classes_from_layers(model.layers))
    # the cache of all three modes against the oracle's solves
    c3 = chert.build_cache(d_classes, 1, MODES, M, H, K, "MEV", "fp64")
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in c3.arrays.items()}
    compare_cache(got, golden_cache(g, MODES, 1, g["tilts"]), 1e-9)
    # the configuration: qP only
    ref = golden_cache(g, ["qP"], 1, g["tilts"])
    cache = chert.build_cache(d_classes, 1, ["qP"], M, H, K, "MEV", "fp64")
    off = inputs.stencil_2d(5)
    cls = model.class_of_node.astype(np.int32)
    d_cls = torch.as_tensor(cls, device="cuda")
    src = int(model.sources[0])
    assert src == 50 + 101 * 50
    tR, tI, pR, pI = chert.traveltime(cache, model.nx, model.nz, model.dx, d_cls, off, [src])
    rcv = np.array([0, 50, 100, 101 * 50, 101 * 50 + 100, 101 * 100, 101 * 100 + 50, 101 * 101 - 1], np.int64)
    paths, lens = chert.raypath(pR.reshape(1, -1), [src], rcv, cap=512)
    pathsI, lensI = chert.raypath(pI.reshape(1, -1), [src], rcv, cap=512)
    idx = chert.edge_table(cache, off)[0].cpu().numpy()
    torch.cuda.synchronize()
    Vs, As, _ = oracle_lookup(ref, 0, off, idx[0])
    shape = (model.nx, 1, model.nz)
    for comp, (t, p, sel, pa, ln) in enumerate([(tR, pR, Vs, paths, lens), (tI, pI, As, pathsI, lensI)]):
        rt, rp = go.dijkstra(shape, model.dx, cls, off, sel, comp, src)
        gt, gp = t[0, 0].cpu().numpy(), p[0, 0].cpu().numpy()
        assert np.all(np.isfinite(rt)) and np.all(np.isfinite(gt))
        assert gt[src] == 0.0 and gp[src] == src
        pos = rt > 0
        assert np.max(np.abs(gt[pos] - rt[pos]) / rt[pos]) <= 1e-9
        near = go.parent_ties(shape, model.dx, cls, off, sel, comp, rt, src, NEAR)
        assert np.array_equal(gp[~near], rp[~near]), int(np.sum((gp != rp) & ~near))
        cand, pred = go.in_candidates(shape, model.dx, cls, off, sel, comp, rt)
        pa, ln = pa.cpu().numpy(), ln.cpu().numpy()
        for r, node in enumerate(rcv):
            want = go.raypath(rp, src, int(node))
            path = [int(v) for v in pa[0, r, :ln[0, r]]]
            assert path[0] == src and path[-1] == node
            if path == want:
                continue
            for i, j in zip(path[:-1], path[1:]):
                if rp[j] == i:
                    continue
                assert near[j], (comp, r, j)
                hit = pred[:, j] == i
                assert hit.any() and cand[hit, j][0] <= rt[j] * (1 + NEAR), (comp, r, j)
