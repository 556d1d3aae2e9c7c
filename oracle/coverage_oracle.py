"""Oracle of the nodewise angular-coverage checks -- TEST INFRASTRUCTURE ONLY.

Only tests, the smoke check and the benchmark's CPU-baseline leg may call this.

The paper validates the cache at selected nodes by an angular-coverage test
(section "Nodewise local-truth and angular-coverage validation"): whether the
sampled ray directions of the cache leave any acceptable local direction
uncovered, and whether the path search could pick a wrong branch.  It names
three figures -- coverage ratio, missing-angle ratio, branch mismatch -- and
gives no formula for them.  This module states one reading, for a 2D cache
(entries e = 0..4M-1 in slowness-angle order) and the node's stencil, whose
candidate path directions d = o/|o| are the nodal angular coverage of the
paper's "Traveltime and Raypath Algorithm" (the directions the lookup of
Eq. 27 must match):

* bracket: two cyclically adjacent valid entries e, e+1 whose ray directions
  r_e, r_e+1 are less than 90 degrees apart and hold d on the closed short
  arc between them (signs of the 2D cross products);
* covered: d has at least one bracket -- the sampled ray-direction manifold
  passes through d;
* first-arrival branch: of the brackets of d, the one with the largest ray
  velocity interpolated at d, V_e + t (V_e+1 - V_e) with
  t = cross(r_e, d) / cross(r_e, r_e+1) (t = 0 for coincident r_e, r_e+1);
  ties to the lower e.  Where the manifold folds (qSV cusps) d has several
  brackets, one per branch, and the first arrival takes the fastest;
* branch mismatch: d is covered and the entry the lookup picks (largest
  d . r, Eq. 27, in the cache's precision: ``graph_oracle.select_direction``)
  is neither end of the first-arrival bracket;
* missing angle: an entry that is valid in a reference ("local truth") cache
  of the same sampling but flagged invalid in the cache under test.

Per (mode, class): covered and mismatched counts over the n_off stencil
directions, missing count over the 4M entries; the ratios divide by those.
Every product, sum and quotient is a separate IEEE double operation, in the
order written here.

Parity status: pinned by the isotropic closed form (ray = slowness
direction: every direction covered, no mismatch), hand-built caches with
planted holes and a planted fold (tests/test_oracle_coverage.py), and the
oracle's Table-2 layer-1 qP cache (no cusps: full coverage, no mismatch).
"""
from __future__ import annotations

import numpy as np

from . import graph_oracle as go


def _cross(ax, az, bx, bz):
    """2D cross product a x b = ax*bz - az*bx (sign: b counter-clockwise of a
    in the (x, z) plane)."""
    return ax * bz - az * bx


def brackets(rx, rz, V, valid, dx, dz):
    """List of (e, V_at_d) for the brackets of direction (dx, dz) in one
    class's entries (1D arrays of length n_dir; float64 values)."""
    n = len(rx)
    out = []
    for e in range(n):
        f = (e + 1) % n
        if not (valid[e] and valid[f]):
            continue
        if rx[e] * rx[f] + rz[e] * rz[f] <= 0.0:
            continue
        c_ef = _cross(rx[e], rz[e], rx[f], rz[f])
        c_ed = _cross(rx[e], rz[e], dx, dz)
        c_df = _cross(dx, dz, rx[f], rz[f])
        if c_ef > 0.0:
            inside = c_ed >= 0.0 and c_df >= 0.0
        elif c_ef < 0.0:
            inside = c_ed <= 0.0 and c_df <= 0.0
        else:
            inside = c_ed == 0.0 and rx[e] * dx + rz[e] * dz > 0.0
        if not inside:
            continue
        t = c_ed / c_ef if c_ef != 0.0 else 0.0
        out.append((e, V[e] + t * (V[f] - V[e])))
    return out


def coverage_counts(cache, offsets, dtype=np.float64, truth_flag=None):
    """(covered, mismatched, missing): int arrays [n_modes, n_classes] for a 2D
    cache dict (arrays [n_modes, n_classes, 4M]); offsets int [n_off, 3] with
    y = 0; dtype: the cache's precision (the lookup's arithmetic);
    truth_flag: flags of the reference cache, or None (missing = 0)."""
    off = np.asarray(offsets, dtype=np.int64).reshape(-1, 3)
    if np.any(off[:, 1] != 0):
        raise ValueError("coverage_counts: 2D stencils only")
    nm, nk, nd = cache["V"].shape
    # unit stencil directions, rounded like the lookup's: d = o/|o| in dtype
    norm = np.sqrt((off.astype(np.float64) ** 2).sum(axis=1)).astype(dtype)
    d = (off.astype(dtype) / norm[:, None]).astype(dtype).astype(np.float64)
    covered = np.zeros((nm, nk), np.int64)
    mismatched = np.zeros((nm, nk), np.int64)
    missing = np.zeros((nm, nk), np.int64)
    for m in range(nm):
        idx = go.select_direction(cache["rx"][m], None, cache["rz"][m], cache["flag"][m], off, dtype)
        for k in range(nk):
            rx = np.asarray(cache["rx"][m, k], np.float64)
            rz = np.asarray(cache["rz"][m, k], np.float64)
            V = np.asarray(cache["V"][m, k], np.float64)
            valid = np.asarray(cache["flag"][m, k]) == 0
            for o in range(len(off)):
                br = brackets(rx, rz, V, valid, d[o, 0], d[o, 2])
                if not br:
                    continue
                covered[m, k] += 1
                best_e, best_v = br[0]
                for e, v in br[1:]:
                    if v > best_v:
                        best_e, best_v = e, v
                pick = idx[k, o]
                if pick != best_e and pick != (best_e + 1) % nd:
                    mismatched[m, k] += 1
            if truth_flag is not None:
                missing[m, k] = int(np.sum((np.asarray(truth_flag[m, k]) == 0) & ~valid))
    return covered, mismatched, missing
