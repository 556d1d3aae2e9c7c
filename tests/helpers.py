"""Shared helpers of the test suite: inputs for both sides and comparisons."""
import math

import numpy as np

from oracle import cache_oracle as co
from paper_2609_26108_b300 import inputs

DEG = math.pi / 180.0


def oracle_moduli(layers):
    """Complex moduli and tilts of layer descriptions, by the oracle's conversion."""
    mods, tilts = [], []
    for L in layers:
        if hasattr(L, "vp0"):
            mods.append(co.moduli_from_thomsen(L.vp0, L.vs0, L.eps, L.delta, L.gamma, L.qp, L.qs))
        else:
            mods.append(co.moduli_from_table(L.aR, L.q))
        tilts.append(L.tilt)
    return np.array(mods), np.array(tilts)


def mixed_layers():
    """A spread of classes: Table 2 layers 1 and 3 (one tilted) and seeded TTI layers."""
    t2 = inputs.table2_layers()
    seeded = inputs.seeded_tti_layers(3, seed=77)
    from dataclasses import replace
    return [t2[0], replace(t2[2], tilt=0.35)] + seeded


def cache_to_torch(cache_np, precision_dtype, device):
    """Oracle cache dict (numpy) -> dict of device tensors in the given dtype."""
    import torch
    out = {}
    for k in ("V", "A", "Q", "rx", "rz", "theta", "vartheta", "ry", "phi"):
        if k not in cache_np:
            continue
        out[k] = torch.as_tensor(np.ascontiguousarray(cache_np[k]), dtype=precision_dtype, device=device)
    out["flag"] = torch.as_tensor(np.ascontiguousarray(cache_np["flag"]), dtype=torch.uint8, device=device)
    return out


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__import__("os").path.abspath(__file__)), "golden")
THOMSEN_KEYS = ("vp0", "vs0", "eps", "delta", "gamma", "qp", "qs", "tilt")


def load_cache_golden(name):
    """A cache golden written by tests/golden/make_cache_golden.py: returns
    {"folded": {(mode, class): [solve dict] * (M+1)}, "tilts": [...] or None,
     "cells": [(node, {thomsen key: value})] or []} with solve dicts holding
    flag, vartheta, V, A, Q and r = (r_x, 0, r_z) as the oracle returns them."""
    import os
    folded, tilts, cells = {}, None, []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("# tilts:"):
                tilts = [float(v) for v in line.split(":", 1)[1].split()]
                continue
            if line.startswith("# cell "):
                parts = line.split()
                cells.append((int(parts[3]), dict(zip(THOMSEN_KEYS, map(float, parts[4:])))))
                continue
            if line.startswith("#") or not line.strip():
                continue
            mode, k, j, flag, vt, V, A, Q, rx, rz = line.split()
            folded.setdefault((mode, int(k)), []).append(
                {"flag": int(flag), "vartheta": float(vt), "V": float(V), "A": float(A), "Q": float(Q),
                 "r": np.array([float(rx), 0.0, float(rz)])})
            assert len(folded[(mode, int(k))]) == int(j) + 1
    return {"folded": folded, "tilts": tilts, "cells": cells}


def golden_cache(g, modes, n_classes, tilts, M=90):
    """The oracle's cache arrays [n_modes, n_classes, 4M] from a loaded golden."""
    folded = [[g["folded"][(m, k)] for k in range(n_classes)] for m in modes]
    return co.assemble_cache(folded, tilts, M)
