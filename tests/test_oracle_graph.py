"""Pins of the graph oracle (lookup, Dijkstra, parents, raypath) against
Floyd-Warshall, scipy's independent Dijkstra, straight-ray closed forms and
reciprocity.  CPU only."""
import math

import numpy as np
import pytest
import scipy.sparse
import scipy.sparse.csgraph

from oracle import graph_oracle as go
from paper_2609_26108_b300 import inputs


def _random_sel(n_classes, offsets, seed, lo=1500.0, hi=4500.0):
    """Per-(class, offset) values that are centrosymmetric (sel[k][o] = sel[k][-o]),
    as a lookup on a centrosymmetric ray surface is."""
    rng = np.random.default_rng(seed)
    off = [tuple(o) for o in offsets]
    sel = np.zeros((n_classes, len(off)))
    for o_i, o in enumerate(off):
        m = off.index(tuple(-x for x in o))
        if m < o_i:
            sel[:, o_i] = sel[:, m]
        else:
            sel[:, o_i] = rng.uniform(lo, hi, n_classes)
    return sel


def test_stencil_counts():
    assert len(inputs.stencil_2d(1)) == 8
    assert len(inputs.stencil_2d(5)) == 80
    assert len(inputs.stencil_3d(1)) == 26
    assert len(inputs.stencil_3d(2)) == 98


@pytest.mark.parametrize("component", [0, 1])
def test_dijkstra_equals_floyd_warshall(component):
    nx, nz = 7, 6
    off = inputs.stencil_2d(3)
    cls = inputs.random_class_map_2d(nx, nz, 3, seed=5).astype(np.int32)
    sel = _random_sel(3, off, 11, 1e-4, 1e-3) if component else _random_sel(3, off, 11)
    I, J, W = go.edge_list((nx, 1, nz), 10.0, cls, off, sel, component)
    D = go.floyd_warshall(nx * nz, I, J, W)
    for src in [0, 17, nx * nz - 1]:
        tau, par = go.dijkstra((nx, 1, nz), 10.0, cls, off, sel, component, src)
        assert np.allclose(tau, D[src], rtol=1e-14, atol=0)


def test_dijkstra_equals_scipy_on_r5_stencil():
    nx, nz = 31, 27
    off = inputs.stencil_2d(5)
    cls = inputs.layered_class_map_2d(nx, nz, 4).astype(np.int32)
    sel = _random_sel(4, off, 3)
    I, J, W = go.edge_list((nx, 1, nz), 10.0, cls, off, sel, 0)
    G = scipy.sparse.csr_matrix((W, (I, J)), shape=(nx * nz, nx * nz))
    ref = scipy.sparse.csgraph.dijkstra(G, directed=True, indices=[0, 400])
    for r, src in enumerate([0, 400]):
        tau, _ = go.dijkstra((nx, 1, nz), 10.0, cls, off, sel, 0, src)
        assert np.allclose(tau, ref[r], rtol=1e-13, atol=0)


def test_dijkstra_3d_equals_scipy():
    nx, ny, nz = 6, 5, 7
    off = inputs.stencil_3d(2)
    rng = np.random.default_rng(2)
    cls = rng.integers(0, 2, nx * ny * nz).astype(np.int32)
    sel = _random_sel(2, off, 9)
    I, J, W = go.edge_list((nx, ny, nz), 10.0, cls, off, sel, 0)
    G = scipy.sparse.csr_matrix((W, (I, J)), shape=(nx * ny * nz,) * 2)
    ref = scipy.sparse.csgraph.dijkstra(G, directed=True, indices=[37])
    tau, _ = go.dijkstra((nx, ny, nz), 10.0, cls, off, sel, 0, 37)
    assert np.allclose(tau, ref[0], rtol=1e-13, atol=0)


def test_homogeneous_isotropic_straight_rays():
    """One class, V and A independent of direction: on nodes reached by a
    straight run of one stencil offset, tau^R = r/V and tau^I = A r exactly;
    elsewhere r/V <= tau^R <= r/(V cos(gap/2)), gap the largest angular gap."""
    nx = nz = 41
    off = inputs.stencil_2d(5)
    V, Aatt = 3000.0, 2e-5
    cls = np.zeros(nx * nz, dtype=np.int32)
    src = 20 + nx * 20
    tR, _ = go.dijkstra((nx, 1, nz), 10.0, cls, off, np.full((1, len(off)), V), 0, src)
    tI, _ = go.dijkstra((nx, 1, nz), 10.0, cls, off, np.full((1, len(off)), Aatt), 1, src)
    x = np.arange(nx * nz) % nx - 20
    z = np.arange(nx * nz) // nx - 20
    r = 10.0 * np.hypot(x, z)
    ang = np.sort(np.arctan2(off[:, 0], off[:, 2]))
    gap = np.max(np.diff(np.concatenate([ang, ang[:1] + 2 * np.pi])))
    m = r > 0
    assert np.all(tR[m] >= r[m] / V * (1 - 1e-14))
    assert np.all(tR[m] <= r[m] / (V * math.cos(gap / 2)) * (1 + 1e-14))
    for (ox, _, oz) in off:
        for s in range(1, 4):
            X, Z = 20 + s * ox, 20 + s * oz
            if 0 <= X < nx and 0 <= Z < nz:
                j = X + nx * Z
                assert tR[j] == pytest.approx(r[j] / V, rel=1e-14)
                assert tI[j] == pytest.approx(Aatt * r[j], rel=1e-14)


def test_reciprocity_and_parent_chains():
    nx, nz = 25, 21
    off = inputs.stencil_2d(4)
    cls = inputs.layered_class_map_2d(nx, nz, 3).astype(np.int32)
    sel = _random_sel(3, off, 21)
    a, b = 3, 18 + nx * 19
    ta, pa = go.dijkstra((nx, 1, nz), 10.0, cls, off, sel, 0, a)
    tb, _ = go.dijkstra((nx, 1, nz), 10.0, cls, off, sel, 0, b)
    assert ta[b] == pytest.approx(tb[a], rel=1e-13)
    # every parent chain reaches the source, tau decreases along it, and each
    # step is an edge whose increment reproduces tau exactly
    offs = {tuple(o): i for i, o in enumerate(off)}
    for rcv in [b, 100, nx * nz - 1]:
        path = go.raypath(pa, a, rcv)
        assert path[0] == a and path[-1] == rcv
        for i, j in zip(path[:-1], path[1:]):
            o = (j % nx - i % nx, 0, j // nx - i // nx)
            oi = offs[o]
            L = 10.0 * math.sqrt(o[0] ** 2 + o[2] ** 2)
            w = L / (0.5 * (sel[cls[i], oi] + sel[cls[j], oi]))
            assert ta[i] + w == ta[j]


def test_parent_tie_rule_smallest_index():
    # 3x3 grid, 4-neighbour stencil, equal weights: the centre-right node (5)
    # from source 0 has two equal-cost parents 2 and 4; the rule keeps 2.
    off = np.array([(1, 0, 0), (-1, 0, 0), (0, 0, 1), (0, 0, -1)], dtype=np.int32)
    sel = np.full((1, 4), 10.0)
    tau, par = go.dijkstra((3, 1, 3), 10.0, np.zeros(9, np.int32), off, sel, 0, 0)
    assert tau[4] == pytest.approx(2.0)
    assert par[4] == 1          # parents 1 and 3 tie; 1 is smaller
    assert par[8] == 5          # 5 and 7 tie
    assert par[0] == 0


def test_unreachable_nodes():
    off = np.array([(1, 0, 0), (-1, 0, 0)], dtype=np.int32)   # rows never connect
    tau, par = go.dijkstra((4, 1, 3), 10.0, np.zeros(12, np.int32), off, np.full((1, 2), 5.0), 0, 1)
    assert np.all(np.isinf(tau[4:])) and np.all(par[4:] == -1)
    assert tau[3] == pytest.approx(4.0)
    assert go.raypath(par, 1, 7) == []


def test_select_direction_brute_force_and_ties():
    rng = np.random.default_rng(4)
    ang = rng.uniform(0, 2 * np.pi, (2, 50))
    rx, rz = np.sin(ang), np.cos(ang)
    flag = (rng.uniform(size=(2, 50)) < 0.2).astype(np.uint8)
    off = inputs.stencil_2d(3)
    idx = go.select_direction(rx, None, rz, flag, off)
    for k in range(2):
        for o_i, (ox, _, oz) in enumerate(off):
            d = np.array([ox, oz]) / math.hypot(ox, oz)
            best, bi = -np.inf, -1
            for e in range(50):
                if flag[k, e]:
                    continue
                dot = d[0] * rx[k, e] + d[1] * rz[k, e]
                if dot > best:
                    best, bi = dot, e
            assert idx[k, o_i] == bi
    # exact tie: two identical directions -> lower index
    rx2 = np.array([[0.0, 1.0, 1.0]]); rz2 = np.array([[1.0, 0.0, 0.0]])
    idx2 = go.select_direction(rx2, None, rz2, np.zeros((1, 3), np.uint8), np.array([(1, 0, 0)]))
    assert idx2[0, 0] == 1
    idx3 = go.select_direction(rx2, None, rz2, np.ones((1, 3), np.uint8), np.array([(1, 0, 0)]))
    assert idx3[0, 0] == -1


def test_parent_ties_manhattan_closed_form():
    """Homogeneous medium, 4-neighbour stencil, source in a corner: every node
    off the two axes through the source is reached by two equally short
    paths (from its left and from its upper neighbour), so it is an exact tie;
    nodes on the axes have one shortest predecessor."""
    nx, nz = 9, 7
    off = np.array([(1, 0, 0), (-1, 0, 0), (0, 0, 1), (0, 0, -1)], np.int32)
    cls = np.zeros(nx * nz, np.int32)
    sel = np.full((1, 4), 2500.0)
    tau, par = go.dijkstra((nx, 1, nz), 10.0, cls, off, sel, 0, 0)
    tie = go.parent_ties((nx, 1, nz), 10.0, cls, off, sel, 0, tau, 0, 0.0)
    x, z = np.arange(nx * nz) % nx, np.arange(nx * nz) // nx
    assert np.array_equal(tie, (x > 0) & (z > 0))
    # with anisotropic speeds the two Manhattan orders still cost the same
    sel2 = np.array([[2000.0, 2000.0, 3100.0, 3100.0]])
    tau2, _ = go.dijkstra((nx, 1, nz), 10.0, cls, off, sel2, 0, 0)
    tie2 = go.parent_ties((nx, 1, nz), 10.0, cls, off, sel2, 0, tau2, 0, 1e-12)
    assert np.array_equal(tie2, (x > 0) & (z > 0))


def test_parent_ties_against_brute_force():
    """Tiny random lattices: the tie flags equal a brute-force enumeration over
    the edge list with Floyd-Warshall distances, at several tolerances."""
    rng = np.random.default_rng(5)
    for trial in range(4):
        nx, nz = 6, 5
        off = inputs.stencil_2d(2)
        cls = rng.integers(0, 3, nx * nz).astype(np.int32)
        sel = rng.uniform(1500, 1600, (3, len(off)))
        src = int(rng.integers(0, nx * nz))
        comp = trial % 2
        if comp:
            sel = sel * 1e-8
        tau, _ = go.dijkstra((nx, 1, nz), 10.0, cls, off, sel, comp, src)
        I, J, W = go.edge_list((nx, 1, nz), 10.0, cls, off, sel, comp)
        D = go.floyd_warshall(nx * nz, I, J, W)
        assert np.allclose(D[src], tau, rtol=1e-12)
        for tol in (0.0, 1e-4, 3e-3, 3e-2):
            want = np.zeros(nx * nz, bool)
            for j in range(nx * nz):
                if j == src:
                    continue
                c = np.sort(D[src, I[J == j]] + W[J == j])
                want[j] = len(c) >= 2 and c[1] - c[0] <= tol * c[0]
            got = go.parent_ties((nx, 1, nz), 10.0, cls, off, sel, comp, tau, src, tol)
            assert np.array_equal(got, want), (trial, tol)


def test_no_cache_fields_equal_the_cached_path():
    """Algorithm 1's per-node evaluation against Algorithm 2's class cache on
    a small two-layer lattice: each node's own table equals its class's table
    entry for entry, so the fields and parents are identical (the paper's
    qP difference below 1e-13 ms between the two methods)."""
    import math
    from oracle import cache_oracle as co
    from oracle import nocache_oracle as nc
    layers = inputs.seeded_tti_layers(2, seed=4)
    mods = np.array([co.moduli_from_thomsen(L.vp0, L.vs0, L.eps, L.delta, L.gamma, L.qp, L.qs) for L in layers])
    tilts = np.array([L.tilt for L in layers])
    nx, nz = 5, 4
    cls = inputs.layered_class_map_2d(nx, nz, 2).astype(np.int32)
    off = inputs.stencil_2d(2)
    h, K, M = 0.05 * math.pi / 180, 600, 6
    for mode in ("qP", "qSV"):
        tables = nc.node_tables(mods, tilts, cls, mode, M, "MEV", h, K)
        cache = co.build_cache(mods, tilts, [mode], M, "MEV", h, K)
        for key in ("V", "A", "rx", "rz", "flag"):
            assert np.array_equal(tables[key][0], cache[key][0][cls], equal_nan=True)
        _, Vs, As = go.lookup_tables(cache, 0, off)
        got = nc.no_cache_fields(mods, tilts, cls, (nx, 1, nz), 10.0, off, mode, M, 3, "MEV", h, K)
        tR, pR = go.dijkstra((nx, 1, nz), 10.0, cls, off, Vs, 0, 3)
        tI, pI = go.dijkstra((nx, 1, nz), 10.0, cls, off, As, 1, 3)
        for a, b in zip(got, (tR, pR, tI, pI)):
            assert np.array_equal(a, b)
