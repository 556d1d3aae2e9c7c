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
