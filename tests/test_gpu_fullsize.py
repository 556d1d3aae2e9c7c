"""Full-size parity of the benchmark's own precision against the FP64 oracle.

Cache (Eq. 4-14, 26): the MIXED build (float scan, float-float root polish
and ray quantities, float storage) at the benchmark's grid -- 0.001 deg scan
step over [-30, 30] deg (K = 30000), 1 deg cache (M = 90), MEV -- against the
oracle's solves stored by tests/golden/make_cache_golden.py: every solve of
the layered 401x401 model's 8 classes in qP, qSV and qSH (8,640 entries), and
every solve of 48 per-cell media of the folded and faulted model.  Flags must
agree exactly; V, A and r to 1e-6 relative (A: of its own size), Q to 1e-5,
the imaginary angle to 1e-6 rad.  FP64 builds to 1e-9.

End to end (Eq. 27-34): the benchmark's launch (Tracer: MIXED cache, lookup,
FP32 relaxation with parents under the default scheduler, raypaths) against
the oracle's FP64 cache, FP64 lookup and binary-heap Dijkstra.  Two discrete
decisions may legitimately differ and are compared for what is unique:
  * the lookup (Eq. 27): where the GPU's float argmax picks another entry than
    the oracle's double one, the two entries' oracle dot products must lie
    within 1e-6 (a lookup tie); the oracle's fields are then computed with
    the GPU's choice, from the oracle's FP64 entries;
  * the parents (Eq. 33): identical outside the nodes that chert_parent_ties
    logs at 1e-5 (test_gpu_relax.check_parents_fp32), and raypaths identical
    until they reach such a node, valid shortest-path steps after it.
Traveltimes to 1e-5 relative at every reachable node.
"""

import numpy as np
import pytest

from oracle import graph_oracle as go
from paper_2609_26108_b300 import chert, inputs

from helpers import DEG, THOMSEN_KEYS, golden_cache, load_cache_golden
from test_gpu_relax import TIE_FP32, check_parents_fp32

pytestmark = pytest.mark.gpu

MODES = ["qP", "qSV", "qSH"]
M = 90
H = 0.001 * DEG
K = 30000
LOOKUP_TIE = 1e-6


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    from paper_2609_26108_b300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


_golden = {}


def layered():
    if "layered" not in _golden:
        g = load_cache_golden("layered_tti_cache_M90.txt")
        model = inputs.layered_tti()
        _golden["layered"] = (model, golden_cache(g, MODES, 8, g["tilts"]))
    return _golden["layered"]


def cells():
    if "cells" not in _golden:
        g = load_cache_golden("folded_cells_cache_M90.txt")
        params = {key: np.array([p[key] for _, p in g["cells"]]) for key in THOMSEN_KEYS}
        nodes = np.array([node for node, _ in g["cells"]])
        _golden["cells"] = (nodes, params, golden_cache(g, MODES, len(nodes), params["tilt"]))
    return _golden["cells"]


def compare_cache(got, ref, tol):
    assert np.array_equal(got["flag"], ref["flag"]), int(np.sum(got["flag"] != ref["flag"]))
    ok = ref["flag"] == 0
    assert np.all(np.isnan(got["V"][~ok]))
    V, A = ref["V"][ok], ref["A"][ok]
    assert np.max(np.abs(got["V"][ok] - V) / V) <= tol
    assert np.all(np.abs(got["A"][ok] - A) <= tol * A + 1e-15 / V)
    for key in ("rx", "rz"):
        assert np.max(np.abs(got[key][ok] - ref[key][ok])) <= tol
    fin = ok & np.isfinite(ref["Q"])
    assert np.max(np.abs(got["Q"][fin] - ref["Q"][fin]) / np.abs(ref["Q"][fin])) <= 10 * tol
    assert np.max(np.abs(got["vartheta"][ok] - ref["vartheta"][ok])) <= tol
    assert np.max(np.abs(got["theta"] - ref["theta"])) <= tol


def gpu_cache(torch, d_classes, n, precision):
    c = chert.build_cache(d_classes, n, MODES, M, H, K, "MEV", precision)
    torch.cuda.synchronize()
    return c, {k: v.cpu().numpy().astype(np.float64) if v.dtype != torch.uint8 else v.cpu().numpy()
               for k, v in c.arrays.items()}


@pytest.mark.parametrize("precision,tol", [("mixed", 1e-6), ("fp64", 1e-9)])
def test_layered_cache_every_solve(torch_dev, precision, tol):
    model, ref = layered()
    d = chert.classes_to_device(chert.classes_from_layers(model.layers))
    _, got = gpu_cache(torch_dev, d, 8, precision)
    compare_cache(got, ref, tol)


@pytest.mark.parametrize("precision,tol", [("mixed", 1e-6), ("fp64", 1e-9)])
def test_per_cell_cache_every_solve(torch_dev, precision, tol):
    nodes, params, ref = cells()
    d = chert.classes_to_device(chert.classes_from_arrays(**params))
    _, got = gpu_cache(torch_dev, d, len(nodes), precision)
    compare_cache(got, ref, tol)


def oracle_lookup(ref, m, off, gpu_idx):
    """Oracle lookup of mode m in FP64 against the GPU's choice: the GPU index
    must be the oracle's or tie with it (dot products within LOOKUP_TIE);
    returns the oracle's FP64 (V, A) tables at the GPU's choice and the number
    of lookup ties."""
    o_idx, _, _ = go.lookup_tables(ref, m, off)
    d = off[:, [0, 2]] / np.linalg.norm(off[:, [0, 2]], axis=1)[:, None]
    rx, rz = ref["rx"][m], ref["rz"][m]
    g = np.asarray(gpu_idx, dtype=np.int64)
    assert np.array_equal(g < 0, o_idx < 0)
    diff = (g != o_idx) & (g >= 0)
    k, o = np.nonzero(diff)
    if len(k):
        dot_g = d[o, 0] * rx[k, g[k, o]] + d[o, 1] * rz[k, g[k, o]]
        dot_o = d[o, 0] * rx[k, o_idx[k, o]] + d[o, 1] * rz[k, o_idx[k, o]]
        assert np.all(ref["flag"][m][k, g[k, o]] == 0)
        assert np.all(dot_o - dot_g <= LOOKUP_TIE), float(np.max(dot_o - dot_g))
    safe = np.maximum(g, 0)
    Vs = np.where(g >= 0, np.take_along_axis(ref["V"][m], safe, axis=1), np.nan)
    As = np.where(g >= 0, np.take_along_axis(ref["A"][m], safe, axis=1), np.nan)
    return Vs, As, int(diff.sum())


def check_paths(paths, lens, rcv, src, rt, rp, gpar, gtie, cand_pred):
    """Raypaths (Eq. 33-34): identical to the oracle's except where they pass
    a node whose parent the GPU logs as a tie; there the GPU's step must be a
    near-optimal oracle step (candidate within TIE_FP32 of the oracle's
    traveltime)."""
    cand, pred = cand_pred
    for r, node in enumerate(rcv):
        want = go.raypath(rp, src, node)
        got = [int(v) for v in paths[r, :lens[r]]]
        assert len(got) > 0 and got[0] == src and got[-1] == node
        if got == want:
            continue
        for i, j in zip(got[:-1], got[1:]):           # step i -> j, j's parent i
            if rp[j] == i:
                continue
            assert gtie[j], (r, j)
            hit = pred[:, j] == i
            assert hit.any() and cand[hit, j][0] <= rt[j] * (1 + TIE_FP32), (r, j)


def run_end_to_end(torch, tracer, ref, off, cls, shape, dx, pick, d_cls):
    tracer.run()
    torch.cuda.synchronize()
    cache = tracer.cache
    idx, _, _ = chert.edge_table(cache, off)
    idx = idx.cpu().numpy()
    tR, tI, pR, pI = (t.cpu().numpy() for t in tracer.tau)
    kR, kI, _ = chert.parent_ties(cache, shape[0], shape[2], dx, d_cls, off, tracer.sources, tracer.tau[0],
                                  tracer.tau[1], TIE_FP32)
    kR, kI = kR.cpu().numpy(), kI.cpu().numpy()
    nf = tracer.n_sources * len(MODES)
    paths, lens = tracer.paths[0].cpu().numpy(), tracer.paths[1].cpu().numpy()
    n_lookup_ties, worst = 0, 0.0
    for m in range(len(MODES)):
        Vs, As, nt = oracle_lookup(ref, m, off, idx[m])
        n_lookup_ties += nt
        for si in pick:
            s = int(tracer.sources[si])
            for comp, (t, p, k, sel) in enumerate([(tR, pR, kR, Vs), (tI, pI, kI, As)]):
                rt, rp = go.dijkstra(shape, dx, cls, off, sel, comp, s)
                gt, gp, gk = t[si, m], p[si, m], k[si, m]
                fin = np.isfinite(rt)
                assert np.array_equal(np.isfinite(gt), fin)
                pos = fin & (rt > 0)
                err = np.abs(gt[pos] - rt[pos]) / rt[pos]
                assert np.all(err <= 1e-5), (si, m, comp, float(err.max()))
                worst = max(worst, float(err.max()))
                check_parents_fp32(gp, gk, rt, rp, sel, comp, s, shape, dx, cls, off)
                f = comp * nf + si * len(MODES) + m
                check_paths(paths[f], lens[f], tracer.receivers, s, rt, rp, gp, gk.astype(bool),
                            go.in_candidates(shape, dx, cls, off, sel, comp, rt))
    return n_lookup_ties, worst


def test_layered_end_to_end_bench_launch(torch_dev):
    """The 401x401, 64-source, 3-mode launch that bench.py times (MIXED cache,
    FP32 relaxation), sources 0, 31 and 63 in every mode against the oracle."""
    from paper_2609_26108_b300.pipeline import Tracer
    model, ref = layered()
    off = inputs.stencil_2d(5)
    rcv = np.round(np.linspace(0, model.nx - 1, 41)).astype(np.int64)
    tr = Tracer(8, MODES, M, model.nx, model.nz, model.dx, off, len(model.sources), rcv, scan_step=H,
                scan_half=K)
    d_classes = chert.classes_to_device(chert.classes_from_layers(model.layers))
    cls = model.class_of_node.astype(np.int32)
    d_cls = torch_dev.as_tensor(cls, device="cuda")
    tr.set_inputs(d_classes, d_cls, model.sources)
    run_end_to_end(torch_dev, tr, ref, off, cls, (model.nx, 1, model.nz), model.dx, [0, 31, 63], d_cls)


def cell_slice():
    """A 241 x 101 slice of the folded and faulted model (x 730..970, z 120..220,
    across the fault) whose nodes take the medium of the nearest of the 48
    stored cells of their own layer (nearest overall if the layer has none)."""
    nodes, params, ref = cells()
    fm = inputs.folded_faulted(n_sources=1)
    x0, x1, z0, z1 = 730, 971, 120, 221
    xs, zs = np.arange(x0, x1), np.arange(z0, z1)
    X, Z = np.meshgrid(xs, zs)
    layer = fm.layer_of_node.reshape(fm.nz, fm.nx)[z0:z1, x0:x1]
    cx, cz = nodes % fm.nx, nodes // fm.nx
    clayer = fm.layer_of_node[nodes]
    d2 = (X[..., None] - cx) ** 2 + (Z[..., None] - cz) ** 2
    same = layer[..., None] == clayer
    d2 = np.where(same | ~same.any(axis=-1, keepdims=True), d2, np.inf)
    cls = np.argmin(d2, axis=-1).astype(np.int32).reshape(-1)
    return x1 - x0, z1 - z0, cls, params, ref


def test_cell_slice_end_to_end(torch_dev):
    """The per-cell media of the folded model (meandering qSV attenuation
    paths) on a 241 x 101 slice, 3 surface sources x 3 modes, MIXED cache and
    FP32 relaxation against the oracle."""
    from paper_2609_26108_b300.pipeline import Tracer
    nx, nz, cls, params, ref = cell_slice()
    off = inputs.stencil_2d(5)
    src = np.array([10, 120, 230], np.int64)
    rcv = np.arange(0, nx * nz, 997).astype(np.int64)
    tr = Tracer(48, MODES, M, nx, nz, 10.0, off, len(src), rcv, scan_step=H, scan_half=K, max_cycles=512)
    d_classes = chert.classes_to_device(chert.classes_from_arrays(**params))
    d_cls = torch_dev.as_tensor(cls, device="cuda")
    tr.set_inputs(d_classes, d_cls, src)
    run_end_to_end(torch_dev, tr, ref, off, cls, (nx, 1, nz), 10.0, [0, 1, 2], d_cls)
