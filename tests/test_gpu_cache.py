"""Parity of the CUDA cache build (chert_build_cache) with the FP64 oracle.

Tolerances (relative unless noted), written here and derived in the design notes:
  FP64   every quantity 1e-9; ray direction and angles 1e-9 absolute.
  MIXED  float scan, double polish: V, A, Q and r to 1e-6 (float storage).
  FP32   V and r to 2e-6; A to 8 eps32 (1 + 1/(A V)): the attenuation is the
         small imaginary part of quantities whose real parts are 1/(A V)
         times larger, so its float error scales with that ratio.
Flags (no acceptable root) must agree exactly.
"""
import math

import numpy as np
import pytest

from oracle import cache_oracle as co
from paper_2609_26108_b300 import chert, inputs

from helpers import DEG, mixed_layers, oracle_moduli, rel_err

pytestmark = pytest.mark.gpu

H = 0.01 * DEG
K = 3000
M = 6
MODES = ["qP", "qSV", "qSH"]


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    from paper_2609_26108_b300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


_oracle = {}


def oracle_cache(kernel):
    if kernel not in _oracle:
        mods, tilts = oracle_moduli(mixed_layers())
        _oracle[kernel] = co.build_cache(mods, tilts, MODES, M, kernel, H, K)
    return _oracle[kernel]


def gpu_cache(torch, kernel, precision, layers=None, modes=MODES, m=M, h=H, k=K):
    layers = mixed_layers() if layers is None else layers
    d_cls = chert.classes_to_device(chert.classes_from_layers(layers))
    c = chert.build_cache(d_cls, len(layers), modes, m, h, k, kernel, precision)
    torch.cuda.synchronize()
    return {key: v.cpu().numpy() for key, v in c.arrays.items()}


def compare(g, o, precision):
    assert np.array_equal(g["flag"], o["flag"]), "flag sets differ"
    ok = o["flag"] == 0
    assert ok.sum() > 0
    assert np.all(np.isnan(g["V"][~ok]))
    theta_tol = 1e-12 if precision == "fp64" else 1e-6
    assert np.max(np.abs(g["theta"] - o["theta"])) < theta_tol
    V_o, A_o = o["V"][ok], o["A"][ok]
    if precision == "fp64":
        tV, tA, tr, tQ = 1e-9, 1e-9, 1e-9, 1e-8
        A_tol = tA * np.maximum(np.abs(A_o), 1e-9 / V_o)
    elif precision == "mixed":
        tV, tA, tr, tQ = 1e-6, 1e-6, 1e-6, 1e-5
        A_tol = tA * np.maximum(np.abs(A_o), 1e-9 / V_o)
    else:
        tV, tr, tQ = 2e-6, 2e-6, None
        eps32 = 2.0 ** -24
        A_tol = 8 * eps32 * (np.abs(A_o) + 1.0 / V_o)
    assert np.max(rel_err(g["V"][ok], V_o)) < tV
    assert np.all(np.abs(g["A"][ok] - A_o) <= A_tol)
    assert np.max(np.abs(g["rx"][ok] - o["rx"][ok])) < tr
    assert np.max(np.abs(g["rz"][ok] - o["rz"][ok])) < tr
    if tQ is not None:
        fin = ok & np.isfinite(o["Q"])
        assert np.max(rel_err(g["Q"][fin], o["Q"][fin])) < tQ
    if precision == "fp64":
        assert np.max(np.abs(g["vartheta"][ok] - o["vartheta"][ok])) < 1e-9


@pytest.mark.parametrize("precision", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("kernel", ["MEV", "OEV"])
def test_cache_matches_oracle(torch_dev, kernel, precision):
    compare(gpu_cache(torch_dev, kernel, precision), oracle_cache(kernel), precision)


def test_cache_isotropic_closed_form(torch_dev):
    """Independent of the oracle: isotropic visco-elastic V = 1/Re(1/c), A = Im(1/c)."""
    from paper_2609_26108_b300.inputs import TableLayer
    M_, mu = 9.0e6, 2.25e6
    a11, a44 = M_ * (1 - 1j / 60), mu * (1 - 1j / 30)
    a13 = a11 - 2 * a44
    aR = [a11.real, a13.real, a11.real, a44.real, a44.real]
    q13 = math.inf if a13.imag == 0 else a13.real / -a13.imag
    q = [60.0, q13, 60.0, 30.0, 30.0]
    layer = TableLayer(aR=tuple(aR), q=tuple(q))
    g = gpu_cache(torch_dev, "OEV", "fp64", [layer], ["qP", "qSH"], 9, H, K)
    for mi, a in enumerate([a11, a44]):
        c = np.sqrt(a)
        assert np.allclose(g["V"][mi], 1 / (1 / c).real, rtol=1e-12)
        assert np.allclose(g["A"][mi], (1 / c).imag, rtol=1e-9)
        th = g["theta"][mi, 0]
        assert np.allclose(g["rx"][mi, 0], np.sin(th), atol=1e-12)
        assert np.allclose(g["rz"][mi, 0], np.cos(th), atol=1e-12)
        assert np.max(np.abs(g["vartheta"][mi])) < 1e-10


def test_full_scan_grid_layered_model_sampled(torch_dev):
    """The layered TTI model at the default grid (0.001 deg over [-30, 30] deg)
    and 1 deg cache: sampled entries against one-by-one oracle solves."""
    model = inputs.layered_tti()
    layers = model.layers
    g = gpu_cache(torch_dev, "MEV", "fp64", layers, MODES, 90, 0.001 * DEG, 30000)
    mods, tilts = oracle_moduli(layers)
    rng = np.random.default_rng(3)
    for _ in range(10):
        mi, k, j = rng.integers(0, 3), rng.integers(0, len(layers)), rng.integers(0, 91)
        A = co.stiffness_tensor(mods[k])
        s = co.solve_direction(A, (math.pi / 2) * j / 90, MODES[mi], "MEV", 0.001 * DEG, 30000)
        d = j                          # first quadrant: no mirroring
        assert g["flag"][mi, k, d] == s["flag"]
        if s["flag"]:
            continue
        ct, st = math.cos(tilts[k]), math.sin(tilts[k])
        rx, rz = s["r"][0] * ct + s["r"][2] * st, -s["r"][0] * st + s["r"][2] * ct
        assert g["V"][mi, k, d] == pytest.approx(s["V"], rel=1e-9)
        assert g["A"][mi, k, d] == pytest.approx(s["A"], rel=1e-9)
        assert g["rx"][mi, k, d] == pytest.approx(rx, abs=1e-9)
        assert g["rz"][mi, k, d] == pytest.approx(rz, abs=1e-9)
    # VTI mirror symmetry of every entry (holds at any size)
    for d in range(1, 90):
        for q in (2 * 90 - d, 2 * 90 + d, 4 * 90 - d):
            assert np.array_equal(g["V"][:, :, d], g["V"][:, :, q], equal_nan=True)


def test_cache_rejects_bad_arguments(torch_dev):
    d_cls = chert.classes_to_device(chert.classes_from_layers(mixed_layers()))
    with pytest.raises(chert.ChertError):
        chert.build_cache(d_cls, 5, ["qP", "qP"], 4)
    with pytest.raises(chert.ChertError):
        chert.build_cache(d_cls, 5, ["qP"], 0)
    with pytest.raises(chert.ChertError):
        chert.build_cache(d_cls, 5, ["qP"], 4, scan_step=-1.0)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_finish_pass_thread_counts_give_the_same_cache(torch_dev, precision):
    """The finish pass with 1024, 512 and 256 threads a CTA (rounds of 2,048,
    1,024 and 512 grid points per side; the nearest 64-point slice with a
    decaying root wins in each) picks the same roots -- the layered model's 8
    classes x 3 modes at the full 0.001 deg x 30,000 grid, whose pending qSV
    solves include ones with no decaying root.  Flags identical; MIXED
    entries bit for bit (float storage); FP64 entries within 8 units in the
    last place, since each instantiation compiles the double ray-quantity
    arithmetic on its own and may contract its multiply-adds differently."""
    torch = torch_dev
    model = inputs.layered_tti()
    d_classes = chert.classes_to_device(chert.classes_from_layers(model.layers))
    lib = chert.lib()
    prev = lib.chert_set_cache_finish_threads(0)
    try:
        out = {}
        for nt in (1024, 512, 256):
            lib.chert_set_cache_finish_threads(nt)
            c = chert.build_cache(d_classes, 8, MODES, 90, 0.001 * DEG, 30000, "MEV", precision)
            torch.cuda.synchronize()
            out[nt] = {k: v.clone() for k, v in c.arrays.items()}
        assert int((out[1024]["flag"] == 1).sum()) > 0
        for nt in (512, 256):
            assert torch.equal(out[1024]["flag"], out[nt]["flag"]), nt
            ok = out[1024]["flag"] == 0
            for k in out[nt]:
                if k == "flag":
                    continue
                a, b = out[1024][k], out[nt][k]
                if precision == "mixed":
                    assert torch.equal(torch.nan_to_num(a, nan=-7.0), torch.nan_to_num(b, nan=-7.0)), (nt, k)
                else:
                    d = (a[ok] - b[ok]).abs()
                    assert bool((d <= 8 * 2.0 ** -52 * a[ok].abs() + 1e-300).all()), (nt, k, float(d.max()))
        assert lib.chert_set_cache_finish_threads(128) == chert.EINVAL
    finally:
        lib.chert_set_cache_finish_threads(prev)
