"""Oracle of the lookup, relaxation and backtracking stages -- TEST INFRASTRUCTURE ONLY.

Only tests, the smoke check and the benchmark's CPU-baseline leg may call this.

* ``select_direction``  the lookup of the paper's "Traveltime and Raypath
  Algorithm": for every (mode, class, offset o) the cached entry whose ray
  direction r has the largest normalised dot product with d = o/|o| (Eq. 27);
  ties go to the lowest entry index, flagged entries never match.
* ``dijkstra``          FP64 binary-heap Dijkstra in plain C (graph_oracle.c) for
  the fixed point of Eq. 31 with the segment-averaged increments of Eq. 28-30,
  and the deterministic parent rule.
* ``parent_ties``       the nodes where the parent rule's two best candidates lie
  within a relative tolerance of each other (where rounding can change the
  parent, Eq. 33).
* ``floyd_warshall``    all-pairs check for tiny grids.
* ``raypath``           backtracking of Eq. 33 from a receiver to the source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graph_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libgraph_oracle.so")
_lib = None


def build() -> str:
    """Compile graph_oracle.c with gcc (-O2, plain C99) if it is out of date."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not os.path.exists(_LIB_PATH)
            or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.oracle_dijkstra.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_double, P, P, ctypes.c_int, P,
                                        ctypes.c_int, ctypes.c_int64, P, P]
        lib.oracle_dijkstra.restype = ctypes.c_int
        _lib = lib
    return _lib


def select_direction(rx, ry, rz, flag, offsets, dtype=np.float64):
    """Best-matching cache entry per (class, offset).

    rx, ry, rz, flag: [n_classes, n_dir] (ry may be None in 2D).
    offsets: int [n_off, 3].  Returns idx [n_classes, n_off] (-1 when a class
    has no valid entry).  The dot product is evaluated in ``dtype`` as
    ((dx*rx) + (dy*ry)) + (dz*rz) with each product rounded, d = o/|o|."""
    off = np.asarray(offsets, dtype=np.float64)
    t = np.dtype(dtype).type
    norm = np.sqrt((off * off).sum(axis=1)).astype(dtype)
    d = (off.astype(dtype) / norm[:, None]).astype(dtype)
    rx = np.asarray(rx).astype(dtype)
    rz = np.asarray(rz).astype(dtype)
    dots = (d[:, None, None, 0] * rx[None]).astype(dtype)
    if ry is not None:
        dots = (dots + (d[:, None, None, 1] * np.asarray(ry).astype(dtype)[None])).astype(dtype)
    dots = (dots + (d[:, None, None, 2] * rz[None])).astype(dtype)   # [n_off, n_classes, n_dir]
    dots = np.where(np.asarray(flag)[None] != 0, t(-np.inf), dots)
    dots = np.where(np.isnan(dots), t(-np.inf), dots)
    idx = np.argmax(dots, axis=2).T.astype(np.int64)                  # first max = lowest index
    none = np.all(np.asarray(flag) != 0, axis=1)
    idx[none, :] = -1
    return idx


def lookup_tables(cache, mode_index, offsets, dtype=np.float64):
    """(idx, Vsel, Asel) for one mode of a cache dict from ``build_cache``."""
    ry = cache.get("ry")
    idx = select_direction(cache["rx"][mode_index], None if ry is None else ry[mode_index],
                           cache["rz"][mode_index], cache["flag"][mode_index], offsets, dtype)
    V = cache["V"][mode_index]
    A = cache["A"][mode_index]
    safe = np.maximum(idx, 0)
    Vsel = np.where(idx >= 0, np.take_along_axis(V, safe, axis=1), np.nan)
    Asel = np.where(idx >= 0, np.take_along_axis(A, safe, axis=1), np.nan)
    return idx, Vsel, Asel


def dijkstra(shape, dx, cls, offsets, sel, component, src):
    """Shortest-path field and parents for one source and one component.

    shape = (nx, ny, nz); cls int [n_nodes]; sel float64 [n_classes, n_off]
    (V for component 0, A for component 1)."""
    nx, ny, nz = shape
    n = nx * ny * nz
    cls = np.ascontiguousarray(cls, dtype=np.int32)
    off = np.ascontiguousarray(offsets, dtype=np.int32)
    sel = np.ascontiguousarray(sel, dtype=np.float64)
    tau = np.empty(n, dtype=np.float64)
    par = np.empty(n, dtype=np.int32)
    rc = _load().oracle_dijkstra(nx, ny, nz, float(dx), cls.ctypes.data, off.ctypes.data,
                                 off.shape[0], sel.ctypes.data, int(component), int(src),
                                 tau.ctypes.data, par.ctypes.data)
    if rc != 0:
        raise RuntimeError("oracle_dijkstra failed")
    return tau, par


def in_candidates(shape, dx, cls, offsets, sel, component, tau):
    """Candidates of the parent rule for every node of a field ``tau``.

    Returns (cand, pred), both [n_off, n_nodes]: pred[o, j] = j - o (the
    in-neighbour through offset o, -1 outside the lattice) and cand[o, j] =
    tau_i + w_ij with the weights of ``dijkstra`` (Eq. 28-30, float64; +inf
    outside the lattice)."""
    nx, ny, nz = shape
    n = nx * ny * nz
    cls = np.asarray(cls).reshape(-1)
    tau = np.asarray(tau, dtype=np.float64).reshape(-1)
    sel = np.asarray(sel, dtype=np.float64)
    j = np.arange(n)
    x, y, z = j % nx, (j // nx) % ny, j // (nx * ny)
    cand = np.full((len(offsets), n), np.inf)
    pred = np.full((len(offsets), n), -1, dtype=np.int64)
    for o, (ox, oy, oz) in enumerate(np.asarray(offsets, dtype=np.int64)):
        X, Y, Z = x - ox, y - oy, z - oz
        ok = (X >= 0) & (X < nx) & (Y >= 0) & (Y < ny) & (Z >= 0) & (Z < nz)
        i = np.where(ok, X + nx * (Y + ny * Z), 0)
        L = dx * np.sqrt(float(ox * ox + oy * oy + oz * oz))
        a, b = sel[cls[i], o], sel[cls[j], o]
        w = L / (0.5 * (a + b)) if component == 0 else L * (0.5 * (a + b))
        cand[o] = np.where(ok, tau[i] + w, np.inf)
        pred[o] = np.where(ok, i, -1)
    return cand, pred


def parent_ties(shape, dx, cls, offsets, sel, component, tau, src, rel_tol):
    """Tie flags of the parent rule for a converged field ``tau`` (Eq. 33).

    Node j is a tie when the second smallest of its candidates
    (``in_candidates``) exceeds the smallest by at most rel_tol times the
    smallest.  The source and the unreachable nodes are never ties.  Returns a
    bool array [n_nodes]."""
    cand, _ = in_candidates(shape, dx, cls, offsets, sel, component, tau)
    n = cand.shape[1]
    if cand.shape[0] < 2:
        return np.zeros(n, dtype=bool)
    two = np.partition(cand, 1, axis=0)[:2]
    best, second = two[0], two[1]
    tau = np.asarray(tau, dtype=np.float64).reshape(-1)
    tie = np.isfinite(second) & (second - best <= rel_tol * best)
    return tie & np.isfinite(tau) & (np.arange(n) != src)


def edge_list(shape, dx, cls, offsets, sel, component):
    """All directed edges (i, j, w) of the stencil graph, for small checks."""
    nx, ny, nz = shape
    I, J, W = [], [], []
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                i = x + nx * (y + ny * z)
                for o, (ox, oy, oz) in enumerate(np.asarray(offsets)):
                    X, Y, Z = x + ox, y + oy, z + oz
                    if 0 <= X < nx and 0 <= Y < ny and 0 <= Z < nz:
                        j = X + nx * (Y + ny * Z)
                        L = dx * np.sqrt(float(ox * ox + oy * oy + oz * oz))
                        a, b = sel[cls[i], o], sel[cls[j], o]
                        w = L / (0.5 * (a + b)) if component == 0 else L * (0.5 * (a + b))
                        I.append(i); J.append(j); W.append(w)
    return np.array(I), np.array(J), np.array(W)


def floyd_warshall(n, I, J, W):
    """All-pairs shortest paths by Floyd-Warshall (dense, O(n^3))."""
    D = np.full((n, n), np.inf)
    np.fill_diagonal(D, 0.0)
    for i, j, w in zip(I, J, W):
        if w < D[i, j]:
            D[i, j] = w
    for k in range(n):
        D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
    return D


def raypath(par, src, rcv, cap=None):
    """Node sequence source -> receiver by following parents from the receiver
    (Eq. 33).  Returns [] if the receiver is unreachable or a cycle appears."""
    par = np.asarray(par)
    cap = len(par) if cap is None else cap
    path = [int(rcv)]
    node = int(rcv)
    if par[node] < 0:
        return []
    while node != src:
        node = int(par[node])
        if node < 0 or len(path) > cap:
            return []
        path.append(node)
    return path[::-1]
