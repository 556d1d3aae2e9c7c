"""Parity of the 3D cache build (chert_build_cache_3d, Eq. 35) and of the
3D direction lookup with the FP64 oracle.

Classes with tilted and azimuthally rotated symmetry axes; tolerances as for
the 2D cache (FP64 1e-9; MIXED 1e-6; FP32 V and r to 2e-6, A within
8 eps32 (A + 1/V)), the ray's y component included; flags exact."""
import math
from dataclasses import replace

import numpy as np
import pytest

from oracle import cache_oracle as co
from oracle import graph_oracle as go
from paper_2609_26108_b300 import chert, inputs

from helpers import DEG, cache_to_torch, mixed_layers, oracle_moduli, rel_err

pytestmark = pytest.mark.gpu

H = 0.02 * DEG
K = 1500
N_AZ, N_POL = 12, 7
MODES = ["qP", "qSV", "qSH"]


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    from paper_2609_26108_b300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def layers3d():
    ls = mixed_layers()[:4]
    return [replace(L, azim=a) for L, a in zip(ls, [0.0, 0.6, 2.0, -1.1])]


_oracle = {}


def oracle3d():
    if "c" not in _oracle:
        ls = layers3d()
        mods, tilts = oracle_moduli(ls)
        _oracle["c"] = co.build_cache_3d(mods, tilts, [L.azim for L in ls], MODES, N_AZ, N_POL, "MEV", H, K)
    return _oracle["c"]


def gpu3d(torch, precision):
    ls = layers3d()
    d_cls = chert.classes_to_device(chert.classes_from_layers(ls))
    c = chert.build_cache_3d(d_cls, len(ls), MODES, N_AZ, N_POL, H, K, "MEV", precision)
    torch.cuda.synchronize()
    return c, {k: v.cpu().numpy() for k, v in c.arrays.items()}


@pytest.mark.parametrize("precision", ["fp64", "mixed", "fp32"])
def test_cache3d_matches_oracle(torch_dev, precision):
    _, g = gpu3d(torch_dev, precision)
    o = oracle3d()
    assert np.array_equal(g["flag"], o["flag"])
    ok = o["flag"] == 0
    assert ok.sum() > 0.5 * ok.size
    tang = 1e-12 if precision == "fp64" else 1e-6
    assert np.max(np.abs(g["theta"] - o["theta"])) < tang and np.max(np.abs(g["phi"] - o["phi"])) < tang
    V_o, A_o = o["V"][ok], o["A"][ok]
    if precision == "fp64":
        tV, tr = 1e-9, 1e-9
        A_tol = 1e-9 * np.maximum(np.abs(A_o), 1e-9 / V_o)
    elif precision == "mixed":
        tV, tr = 1e-6, 1e-6
        A_tol = 1e-6 * np.maximum(np.abs(A_o), 1e-9 / V_o)
    else:
        tV, tr = 2e-6, 2e-6
        A_tol = 8 * 2.0 ** -24 * (np.abs(A_o) + 1.0 / V_o)
    assert np.max(rel_err(g["V"][ok], V_o)) < tV
    assert np.all(np.abs(g["A"][ok] - A_o) <= A_tol)
    for key in ("rx", "ry", "rz"):
        assert np.max(np.abs(g[key][ok] - o[key][ok])) < tr, key


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_lookup3d_matches_oracle(torch_dev, precision):
    """3D stencil (radius 2, 98 offsets): the selected entries, with the y term
    of the dot product, agree exactly when both sides read the same cache."""
    o = oracle3d()
    dt = torch_dev.float64 if precision == "fp64" else torch_dev.float32
    arr = cache_to_torch(o, dt, "cuda")
    prec = chert.PRECISION_IDS[precision]
    cache = chert.Cache(arr, list(range(len(MODES))), 4, 0, prec, N_AZ, N_POL)
    off = inputs.stencil_3d(2)
    assert len(off) == 98
    idx, Vs, As = chert.edge_table(cache, off)
    torch_dev.cuda.synchronize()
    idx = idx.cpu().numpy()
    npdt = np.float64 if precision == "fp64" else np.float32
    cast = {k: (o[k].astype(npdt).astype(np.float64) if k != "flag" else o[k]) for k in o}
    for m in range(len(MODES)):
        ref, _, _ = go.lookup_tables(cast, m, off, dtype=npdt)
        assert np.array_equal(idx[m], ref)
