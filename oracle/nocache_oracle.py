"""Oracle of the no-cache (MSPM-style) traveltime -- TEST INFRASTRUCTURE ONLY.

Only tests, the smoke check and the benchmark's CPU-baseline leg may call this.

The paper's Algorithm 1 (the conventional modified shortest-path method it
compares against) evaluates the ray quantities of the kernel afresh at the
nodes of every cell that becomes active, for every source and wave mode,
instead of reading a directional cache built once per class (Algorithm 2).
This module restates that for the lattice form used here, in plain FP64:

* for each node, its own directional table: the homogeneity solve (Eq. 9-11)
  of the node's medium at the sampled slowness angles (Eq. 26), built with
  ``cache_oracle.build_cache`` for that one medium -- nothing is shared
  between nodes, even where two nodes have the same medium;
* for each node and stencil offset, the entry of the node's own table whose
  ray best matches the offset direction (Eq. 27), as ``graph_oracle`` does;
* the fixed point of Eq. 31 by ``graph_oracle.dijkstra`` with those per-node
  values (Eq. 28-30).

Parity status: where nodes share a medium the per-node tables equal the
class tables entry for entry, so the fields equal those of the cached path
(``graph_oracle`` on the class cache); the tests check exactly that.
"""
from __future__ import annotations

import numpy as np

from . import cache_oracle as co
from . import graph_oracle as go


def node_tables(moduli, tilts, class_of_node, mode, M, kernel="MEV", h=0.001 * co.DEG, K=30000):
    """Each node's own cache of one mode: dict of arrays [1, n_nodes, 4M], the
    solves repeated for every node from its medium (moduli[class_of_node[j]],
    tilts[class_of_node[j]])."""
    moduli = np.asarray(moduli, dtype=np.complex128).reshape(-1, 5)
    tilts = np.asarray(tilts, dtype=np.float64).reshape(-1)
    cls = np.asarray(class_of_node).reshape(-1)
    per_node = [co.build_cache(moduli[k:k + 1], tilts[k:k + 1], [mode], M, kernel, h, K) for k in cls]
    return {key: np.concatenate([t[key] for t in per_node], axis=1) for key in per_node[0]}


def no_cache_fields(moduli, tilts, class_of_node, shape, dx, offsets, mode, M, source, kernel="MEV",
                    h=0.001 * co.DEG, K=30000):
    """(tauR, parR, tauI, parI) of one (source, mode) field with every node's
    ray quantities evaluated from its own table (module docstring)."""
    tables = node_tables(moduli, tilts, class_of_node, mode, M, kernel, h, K)
    n = int(np.prod(shape))
    own = np.arange(n, dtype=np.int32)                 # node j reads its own table
    _, Vs, As = go.lookup_tables(tables, 0, offsets)
    tR, pR = go.dijkstra(shape, dx, own, offsets, Vs, 0, source)
    tI, pI = go.dijkstra(shape, dx, own, offsets, As, 1, source)
    return tR, pR, tI, pI
