"""Parity of the 3D relaxation (plane sweeps) and parents with the oracle's
binary-heap Dijkstra on the same cache, and of the 3D pipeline (GPU 3D cache,
lookup, traveltime, raypaths) with the oracle end to end.

Tolerances as in 2D: FP64 tau to 1e-12 relative with identical parents; FP32
tau per node within max(1e-5, 2 (hops + 2) 2^-24)."""
import math

import numpy as np
import pytest

from oracle import graph_oracle as go
from paper_2609_26108_b300 import chert, inputs

from helpers import cache_to_torch
from test_gpu_relax import TIE_FP32, TIE_FP64, _check_fields, check_parents_fp32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    from paper_2609_26108_b300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def synthetic_cache3d(n_classes, n_az=16, n_pol=9, seed=0):
    """Lookup-only 3D cache: rays along the slowness directions of the global
    grid, V and A varying with the polar angle per class."""
    rng = np.random.default_rng(seed)
    nd = n_az * n_pol
    th = (np.arange(n_pol) + 0.5) * math.pi / n_pol
    ph = np.arange(n_az) * 2 * math.pi / n_az
    T, P = np.meshgrid(th, ph, indexing="ij")
    T, P = T.reshape(-1), P.reshape(-1)
    v0 = rng.uniform(1500, 4500, n_classes)
    an = rng.uniform(-0.2, 0.2, n_classes)
    V = v0[:, None] * (1 + an[:, None] * np.cos(2 * T)[None])
    A = rng.uniform(1e-5, 1e-4, n_classes)[:, None] * (1 + 0.3 * np.sin(T)[None] ** 2)
    c = {"V": V[None], "A": A[None],
         "rx": np.tile(np.sin(T) * np.cos(P), (1, n_classes, 1)),
         "ry": np.tile(np.sin(T) * np.sin(P), (1, n_classes, 1)),
         "rz": np.tile(np.cos(T), (1, n_classes, 1)),
         "theta": np.tile(T, (1, n_classes, 1)), "phi": np.tile(P, (1, n_classes, 1)),
         "vartheta": np.zeros((1, n_classes, nd)), "flag": np.zeros((1, n_classes, nd), np.uint8)}
    c["Q"] = np.full_like(c["V"], np.inf)
    return c, n_az, n_pol


def run3d(torch, cnp, n_az, n_pol, precision, shape, cls, off, sources):
    prec = chert.PRECISION_IDS[precision]
    dt = torch.float64 if prec == chert.FP64 else torch.float32
    nm, nk, _ = cnp["V"].shape
    cache = chert.Cache(cache_to_torch(cnp, dt, "cuda"), list(range(nm)), nk, 0, prec, n_az, n_pol)
    nx, ny, nz = shape
    d_cls = torch.as_tensor(np.asarray(cls, np.int32), device="cuda")
    tR, tI, pR, pI = chert.traveltime(cache, nx, nz, 10.0, d_cls, off, sources, max_cycles=64, ny=ny)
    kR, kI, _ = chert.parent_ties(cache, nx, nz, 10.0, d_cls, off, sources, tR, tI,
                                  TIE_FP64 if prec == chert.FP64 else TIE_FP32, ny=ny)
    torch.cuda.synchronize()
    return tuple(t.cpu().numpy() for t in (tR, tI, pR, pI, kR, kI))


def oracle3d_fields(cnp, precision, shape, cls, off, sources):
    dt = np.float64 if precision == "fp64" else np.float32
    cast = {k: (cnp[k].astype(dt).astype(np.float64) if k != "flag" else cnp[k]) for k in cnp}
    out = {}
    for m in range(cnp["V"].shape[0]):
        _, Vs, As = go.lookup_tables(cast, m, off, dtype=dt)
        for s in sources:
            out[(s, m, 0)] = go.dijkstra(shape, 10.0, cls, off, Vs, 0, s) + (Vs,)
            out[(s, m, 1)] = go.dijkstra(shape, 10.0, cls, off, As, 1, s) + (As,)
    return out


@pytest.mark.parametrize("n_classes", [4, 30, 400])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_relax3d_matches_oracle(torch_dev, precision, n_classes):
    """4 layers (class-pair table in shared memory), 30 random classes (raw
    tables in shared memory) and 400 random classes (tables in global
    memory); a lattice of several planes in each direction, ragged sizes."""
    shape = (19, 14, 11)
    nx, ny, nz = shape
    n = nx * ny * nz
    if n_classes == 4:
        z = np.arange(n) // (nx * ny)
        cls = np.minimum(z * 4 // nz, 3).astype(np.int32)
    else:
        cls = np.random.default_rng(n_classes).integers(0, n_classes, n).astype(np.int32)
    cnp, n_az, n_pol = synthetic_cache3d(n_classes, seed=n_classes)
    off = inputs.stencil_3d(2)
    sources = [0, nx // 2 + nx * (ny // 2 + ny * (nz // 2))]
    g = run3d(torch_dev, cnp, n_az, n_pol, precision, shape, cls, off, sources)
    ref = oracle3d_fields(cnp, precision, shape, cls, off, sources)
    _check_fields(g, ref, sources, 1, precision, shape, 10.0, cls, off, cnp)


def test_pipeline3d_gpu_cache_to_traveltime_fp64(torch_dev):
    """GPU 3D cache (tilted, azimuthally rotated TTI classes) -> lookup ->
    traveltime against the oracle's 3D cache -> Dijkstra, and raypaths that
    follow the oracle's parents."""
    from test_gpu_cache3d import H, K, MODES, N_AZ, N_POL, layers3d, oracle3d
    ls = layers3d()
    d_cls = chert.classes_to_device(chert.classes_from_layers(ls))
    cache = chert.build_cache_3d(d_cls, len(ls), MODES, N_AZ, N_POL, H, K, "MEV", "fp64")
    shape = (13, 11, 9)
    nx, ny, nz = shape
    n = nx * ny * nz
    cls = np.minimum((np.arange(n) // (nx * ny)) * 4 // nz, 3).astype(np.int32)
    off = inputs.stencil_3d(2)
    src = [nx // 2 + nx * (ny // 2)]
    tR, tI, pR, pI = chert.traveltime(cache, nx, nz, 10.0, torch_dev.as_tensor(cls, device="cuda"), off, src,
                                      ny=ny)
    torch_dev.cuda.synchronize()
    o = oracle3d()
    for m in range(len(MODES)):
        _, Vs, As = go.lookup_tables(o, m, off)
        for comp, (t, p, sel) in enumerate([(tR, pR, Vs), (tI, pI, As)]):
            rt, rp = go.dijkstra(shape, 10.0, cls, off, sel, comp, src[0])
            gt = t[0, m].cpu().numpy()
            fin = np.isfinite(rt)
            assert np.array_equal(np.isfinite(gt), fin)
            assert np.allclose(gt[fin], rt[fin], rtol=1e-9, atol=0)
    rcv = [0, n - 1, nx * ny * (nz - 1) + 3]
    paths, lens = chert.raypath(pR[0, 0], src, rcv, cap=256)
    paths, lens = paths.cpu().numpy()[0], lens.cpu().numpy()[0]
    par = pR[0, 0].cpu().numpy()
    for r, node in enumerate(rcv):
        want = go.raypath(par, src[0], node)
        assert lens[r] == len(want) and list(paths[r, :lens[r]]) == want


def test_full_size_3d_sampled(torch_dev):
    """The 201^3 layered TTI model in the benchmark's launch configuration
    (1 deg x 1 deg FP64 cache, 98 offsets): sampled cache entries against
    single oracle solves at the full 0.001 deg scan, and the qP propagation
    and qSV attenuation fields of one source against the oracle's Dijkstra on
    the GPU cache's own lookup (FP64 tau to 1e-12, identical parents)."""
    import math as _m
    from oracle import cache_oracle as co
    from helpers import oracle_moduli
    m = inputs.layered_tti_3d(n_sources=1)
    modes = ["qP", "qSV"]
    nk = len(m.layers)
    d_classes = chert.classes_to_device(chert.classes_from_layers(m.layers))
    cache = chert.build_cache_3d(d_classes, nk, modes, 360, 180, precision="fp64")
    torch_dev.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in cache.arrays.items()}
    mods, tilts = oracle_moduli(m.layers)
    rng = np.random.default_rng(5)
    for _ in range(6):
        mi, k, i, j = rng.integers(0, 2), rng.integers(0, nk), rng.integers(0, 180), rng.integers(0, 360)
        d = i * 360 + j
        s, r, _sz = co.solve_direction_3d(co.stiffness_tensor(mods[k]), tilts[k], m.layers[k].azim,
                                          (i + 0.5) * _m.pi / 180, j * 2 * _m.pi / 360, modes[mi], "MEV")
        assert g["flag"][mi, k, d] == s["flag"]
        if s["flag"]:
            continue
        assert g["V"][mi, k, d] == pytest.approx(s["V"], rel=1e-9)
        assert g["A"][mi, k, d] == pytest.approx(s["A"], rel=1e-9)
        for q, key in enumerate(("rx", "ry", "rz")):
            assert g[key][mi, k, d] == pytest.approx(r[q], abs=1e-9)
    cls = m.class_of_node
    off = inputs.stencil_3d(2)
    src = int(m.sources[0])
    tR, tI, pR, pI = chert.traveltime(cache, m.nx, m.nz, m.dx, torch_dev.as_tensor(cls, device="cuda"), off,
                                      [src], ny=m.ny)
    torch_dev.cuda.synchronize()
    shape = (m.nx, m.ny, m.nz)
    for mi, comp, t, p in ((0, 0, tR, pR), (1, 1, tI, pI)):
        _, Vs, As = go.lookup_tables(g, mi, off)
        rt, rp = go.dijkstra(shape, m.dx, cls, off, Vs if comp == 0 else As, comp, src)
        gt, gp = t[0, mi].cpu().numpy(), p[0, mi].cpu().numpy()
        fin = np.isfinite(rt)
        assert np.array_equal(np.isfinite(gt), fin)
        assert np.allclose(gt[fin], rt[fin], rtol=1e-12, atol=0)
        assert np.array_equal(gp, rp)


@pytest.mark.parametrize("n_classes", [4, 400])
def test_relax3d_float_weights_wide_accumulation(torch_dev, n_classes):
    """CHERT_FP32_ACC64: float cache and weights, float-float accumulation,
    double output.  Against the oracle's double Dijkstra on the float lookup:
    each weight carries about two float roundings and the accumulation about
    2^-47 per hop, so tau is within 4e-7 relative however long the path (FP32
    accumulation drifts with the hop count); the source and unreachable nodes
    are exact."""
    shape = (23, 12, 15)
    nx, ny, nz = shape
    n = nx * ny * nz
    if n_classes == 4:
        cls = np.minimum((np.arange(n) // (nx * ny)) * 4 // nz, 3).astype(np.int32)
    else:
        cls = np.random.default_rng(n_classes + 1).integers(0, n_classes, n).astype(np.int32)
    cnp, n_az, n_pol = synthetic_cache3d(n_classes, seed=n_classes + 2)
    nm, nk, _ = cnp["V"].shape
    cache = chert.Cache(cache_to_torch(cnp, torch_dev.float32, "cuda"), list(range(nm)), nk, 0, chert.FP32,
                        n_az, n_pol)
    off = inputs.stencil_3d(2)
    sources = [3, nx * ny * nz - 5]
    d_cls = torch_dev.as_tensor(cls, device="cuda")
    tR, tI, pR, pI = chert.traveltime(cache, nx, nz, 10.0, d_cls, off, sources, ny=ny, precision="fp32_acc64")
    kR, kI, _ = chert.parent_ties(cache, nx, nz, 10.0, d_cls, off, sources, tR, tI, TIE_FP32, ny=ny,
                                  precision="fp32_acc64")
    torch_dev.cuda.synchronize()
    assert tR.dtype == torch_dev.float64
    ref = oracle3d_fields(cnp, "fp32", shape, cls, off, sources)
    for si, s in enumerate(sources):
        for comp, (t, p, k) in enumerate([(tR, pR, kR), (tI, pI, kI)]):
            rt, rp, sel = ref[(s, 0, comp)]
            gt, gp = t[si, 0].cpu().numpy(), p[si, 0].cpu().numpy()
            fin = np.isfinite(rt)
            assert np.array_equal(np.isfinite(gt), fin)
            pos = fin & (rt > 0)
            assert np.max(np.abs(gt[pos] - rt[pos]) / rt[pos]) < 4e-7
            assert gt[s] == 0.0 and gp[s] == s
            assert np.all(gp[~fin] == -1)
            check_parents_fp32(gp, k[si, 0].cpu().numpy(), rt, rp, sel, comp, s, shape, 10.0, cls, off)


@pytest.mark.parametrize("precision", ["fp64", "fp32_acc64"])
def test_relax3d_split_across_ctas_equals_one_cta(torch_dev, precision):
    """A lattice of several tiles per plane with few field components: the
    eager launch shares each plane's tiles among several CTAs per field
    component (cooperative launch), the same call captured in a CUDA graph
    runs one CTA per field component; fields and parents must be identical,
    bit for bit (the fixed point and its parents do not depend on the order
    the tiles are relaxed in)."""
    torch = torch_dev
    shape = (70, 41, 33)
    nx, ny, nz = shape
    n = nx * ny * nz
    cls = np.minimum((np.arange(n) // (nx * ny)) * 4 // nz, 3).astype(np.int32)
    cnp, n_az, n_pol = synthetic_cache3d(4, seed=9)
    nm, nk, _ = cnp["V"].shape
    cache_prec = chert.FP64 if precision == "fp64" else chert.FP32
    dt = torch.float64 if precision == "fp64" else torch.float32
    cache = chert.Cache(cache_to_torch(cnp, dt, "cuda"), list(range(nm)), nk, 0, cache_prec, n_az, n_pol)
    off = inputs.stencil_3d(2)
    d_cls = torch.as_tensor(cls, device="cuda")
    src = torch.as_tensor(np.array([3, n // 2 + 17], np.int64), device="cuda")
    prec = chert.PRECISION_IDS[precision]
    ws = torch.empty(chert.workspace_bytes(1, nk, len(off), prec, 2), dtype=torch.uint8, device="cuda")
    fd = torch.float64
    outs = []
    for captured in (False, True):
        out = (torch.empty((2, 1, n), dtype=fd, device="cuda"), torch.empty((2, 1, n), dtype=fd, device="cuda"),
               torch.empty((2, 1, n), dtype=torch.int32, device="cuda"),
               torch.empty((2, 1, n), dtype=torch.int32, device="cuda"))
        status = torch.zeros(2, dtype=torch.int32, device="cuda")
        run = lambda: chert.lib().chert_traveltime_enqueue(
            __import__("ctypes").byref(cache.struct()), 1, nk, cache.n_dir, nx, ny, nz, 10.0,
            chert._dev_ptr(d_cls), *chert._offsets_arr(off)[1:], len(off), chert._dev_ptr(src), 2, prec, 64,
            chert._dev_ptr(out[0]), chert._dev_ptr(out[1]), chert._dev_ptr(out[2]), chert._dev_ptr(out[3]),
            chert._dev_ptr(ws), ws.numel(), chert._dev_ptr(status), chert._stream_ptr(None))
        if captured:
            g = torch.cuda.CUDAGraph()
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                with torch.cuda.graph(g, stream=s):
                    assert run() == 0
            g.replay()
        else:
            assert run() == 0
        torch.cuda.synchronize()
        assert status.cpu().tolist() == [-1, 0]
        outs.append(out)
    for a, b in zip(*outs):
        assert torch.equal(a, b)


def _lattice_case(torch, shape, n_classes, seed, precision, sources):
    nx, ny, nz = shape
    n = nx * ny * nz
    rng = np.random.default_rng(seed)
    if n_classes <= 6:
        cls = np.minimum((np.arange(n) // (nx * ny)) * n_classes // nz, n_classes - 1).astype(np.int32)
    else:
        cls = rng.integers(0, n_classes, n).astype(np.int32)
    cnp, n_az, n_pol = synthetic_cache3d(n_classes, seed=seed)
    nm, nk, _ = cnp["V"].shape
    cache_prec = chert.FP64 if precision == "fp64" else chert.FP32
    dt = torch.float64 if precision == "fp64" else torch.float32
    cache = chert.Cache(cache_to_torch(cnp, dt, "cuda"), list(range(nm)), nk, 0, cache_prec, n_az, n_pol)
    fd = torch.float64 if precision in ("fp64", "fp32_acc64") else torch.float32
    ns = len(sources)
    out = (torch.full((ns, nm, n), -3.0, dtype=fd, device="cuda"), torch.full((ns, nm, n), -3.0, dtype=fd, device="cuda"),
           torch.full((ns, nm, n), -7, dtype=torch.int32, device="cuda"),
           torch.full((ns, nm, n), -7, dtype=torch.int32, device="cuda"))
    prec = chert.PRECISION_IDS[precision]
    ws = torch.empty(chert.workspace_bytes(nm, nk, 98, prec, ns), dtype=torch.uint8, device="cuda")
    return {"cache": cache, "nx": nx, "ny": ny, "nz": nz, "dx": 10.0,
            "d_cls": torch.as_tensor(cls, device="cuda"),
            "d_sources": torch.as_tensor(np.asarray(sources, np.int64), device="cuda"), "out": out,
            "workspace": ws, "d_status": torch.full((2,), 5, dtype=torch.int32, device="cuda")}


@pytest.mark.parametrize("precision", ["fp64", "fp32_acc64", "fp32"])
def test_batch_of_uneven_lattices_equals_single_calls(torch_dev, precision):
    """chert_traveltime_batch (one persistent launch over the field components
    of several 3D lattices of uneven size and class count) against
    chert_traveltime on each lattice alone: fields and parents bit for bit,
    status [-1, 0] for each.  Under both 3D tile shapes, and captured in a
    CUDA graph (two replays)."""
    torch = torch_dev
    off = inputs.stencil_3d(2)
    cases = [((19, 14, 11), 4, 1, [0, 19 * 14 * 11 - 1, 700]), ((33, 9, 21), 30, 2, [5, 2000]),
             ((12, 12, 12), 6, 3, [100]), ((41, 17, 8), 400, 4, [3, 4000, 5000])]
    prev = chert.set_relax3d_tile(0)
    try:
        for tile in (0, 1):
            chert.set_relax3d_tile(tile)
            items = [_lattice_case(torch, sh, nk, sd, precision, src) for sh, nk, sd, src in cases]
            counter = torch.zeros(1, dtype=torch.int64, device="cuda")
            chert.traveltime_batch(items, off, counter, precision=precision)
            torch.cuda.synchronize()
            for it in items:
                assert it["d_status"].cpu().tolist() == [-1, 0]
                ref = chert.traveltime(it["cache"], it["nx"], it["nz"], 10.0, it["d_cls"], off,
                                       it["d_sources"].cpu().numpy(), ny=it["ny"], precision=precision)
                torch.cuda.synchronize()
                for a, b in zip(ref, it["out"]):
                    assert torch.equal(a, b), tile
            # the same batch recorded in a graph
            for it in items:
                for o in it["out"]:
                    o.fill_(-1)
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                chert.traveltime_batch(items, off, counter, precision=precision, stream=s)
            for _ in range(2):
                g.replay()
                torch.cuda.synchronize()
                for it in items:
                    ref = chert.traveltime(it["cache"], it["nx"], it["nz"], 10.0, it["d_cls"], off,
                                           it["d_sources"].cpu().numpy(), ny=it["ny"], precision=precision)
                    torch.cuda.synchronize()
                    for a, b in zip(ref, it["out"]):
                        assert torch.equal(a, b)
    finally:
        chert.set_relax3d_tile(prev)


def test_batch_rejects_2d_lattices(torch_dev):
    torch = torch_dev
    it = _lattice_case(torch, (19, 14, 11), 4, 1, "fp64", [0])
    it["ny"], it["nz"] = 1, 14 * 11
    with pytest.raises(chert.ChertError) as e:
        chert.traveltime_batch([it], inputs.stencil_3d(2), torch.zeros(1, dtype=torch.int64, device="cuda"))
    assert e.value.code == chert.EINVAL


@pytest.mark.parametrize("elastic", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_acc64"])
def test_unrolled_stencil_equals_general_form(torch_dev, precision, elastic):
    """The reach-2 stencil in its standard order runs the unrolled sweeps
    (class-pair table); the same 98 offsets in reverse order run the general
    form.  The fixed point and the parent rule (smallest node index among
    equal candidates) do not depend on the order of the offsets, so fields
    and parents must be identical, bit for bit, on a ragged lattice of
    several tiles per plane.  elastic: A = 0 everywhere, so the attenuation
    field is 0 and every parent is decided by the tie rule alone."""
    torch = torch_dev
    shape = (45, 23, 19)
    nx, ny, nz = shape
    n = nx * ny * nz
    cls = np.minimum((np.arange(n) // (nx * ny)) * 5 // nz, 4).astype(np.int32)
    cnp, n_az, n_pol = synthetic_cache3d(5, seed=4)
    if elastic:
        cnp["A"] = np.zeros_like(cnp["A"])
    nm, nk, _ = cnp["V"].shape
    cache_prec = chert.FP64 if precision == "fp64" else chert.FP32
    dt = torch.float64 if precision == "fp64" else torch.float32
    cache = chert.Cache(cache_to_torch(cnp, dt, "cuda"), list(range(nm)), nk, 0, cache_prec, n_az, n_pol)
    d_cls = torch.as_tensor(cls, device="cuda")
    sources = [0, 21 + nx * (11 + ny * 9), n - 1]
    off = inputs.stencil_3d(2)
    res = []
    for o in (off, np.ascontiguousarray(off[::-1])):
        r = chert.traveltime(cache, nx, nz, 10.0, d_cls, o, sources, max_cycles=64, ny=ny, precision=precision)
        torch.cuda.synchronize()
        res.append(r)
    for a, b in zip(*res):
        assert torch.equal(a, b)
    assert np.all(np.isfinite(res[0][0].cpu().numpy()))
    if elastic:
        assert not res[0][1].any()
