"""The cache surrogate on the GPU: BF16 forward and gradient against the FP64
oracle network with the same BF16 rounding points, the training pairs against
the oracle's own exact cache, and what a trained network gains.

Tolerances: with the operands rounded to bfloat16 at the same points on both
sides, the remaining difference is FP32 against FP64 accumulation, plus an
occasional activation that rounds to the neighbouring bfloat16 value (2^-8
relative) because the two accumulations straddle a rounding boundary; one
such flip moves an output by about 2^-8 * |w| * |h| / sqrt(256).  Outputs and
gradients are compared to 1e-2 of their scale and must agree to 1e-3 in the
median."""
import math

import numpy as np
import pytest

from oracle import cache_oracle as co
from oracle import mlp_oracle as mo
from paper_2609_26108_b300 import chert, inputs, surrogate

from helpers import DEG, cache_to_torch, oracle_moduli

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    from paper_2609_26108_b300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def _net(seed):
    layers = inputs.mlp_init(seed)
    rng = np.random.default_rng(seed + 1)
    layers = [(W, rng.normal(0, 0.05, b.shape)) for W, b in layers]
    mean = rng.normal(0, 0.1, 5)
    std = rng.uniform(0.5, 2.0, 5)
    mean[3], std[3] = 0.0, 1.0
    return layers, mean, std


def _x(n, seed):
    x = np.random.default_rng(seed).uniform(-1, 1, (n, 8))
    x[:, 7] = 0.0
    return x


def test_forward_matches_oracle_bf16(torch_dev):
    layers, mean, std = _net(3)
    params = torch_dev.as_tensor(surrogate.pack_params(layers, mean, std), device="cuda")
    x = _x(1000, 4)
    y = chert.mlp_forward(params, torch_dev.as_tensor(x, dtype=torch_dev.float32, device="cuda"))
    torch_dev.cuda.synchronize()
    W = [l[0].astype(np.float32).astype(np.float64) for l in layers]
    b = [l[1].astype(np.float32).astype(np.float64) for l in layers]
    ref, _ = mo.forward(W, b, x[:, :7].astype(np.float32).astype(np.float64), quantize=True)
    err = np.abs(y.cpu().numpy() - ref)
    scale = np.abs(ref).mean(0)
    assert np.all(err <= 1e-2 * scale + 1e-4)
    assert np.median(err / scale) < 1e-3


def test_gradient_matches_oracle_bf16(torch_dev):
    layers, mean, std = _net(5)
    params = torch_dev.as_tensor(surrogate.pack_params(layers, mean, std), device="cuda")
    n = 512
    x = _x(n, 6)
    rng = np.random.default_rng(7)
    t = rng.normal(0, 1, (n, 5)) * std + mean
    t[:, 3] = (rng.uniform(size=n) > 0.2).astype(float)
    t[::7, 1] = np.nan                        # left out of the fit of output 1
    t[3::11, 0:3] = np.nan
    zeros = torch_dev.zeros_like(params)
    loss, grad = chert.mlp_train_step(params, zeros.clone(), zeros.clone(), 1, 0.0,
                                      torch_dev.as_tensor(x, dtype=torch_dev.float32, device="cuda"),
                                      torch_dev.as_tensor(t, dtype=torch_dev.float32, device="cuda"),
                                      want_grad=True)
    torch_dev.cuda.synchronize()
    W = [l[0].astype(np.float32).astype(np.float64) for l in layers]
    b = [l[1].astype(np.float32).astype(np.float64) for l in layers]
    rl, dW, db = mo.loss_and_grad(W, b, x[:, :7].astype(np.float32).astype(np.float64),
                                  t.astype(np.float32).astype(np.float64),
                                  mean.astype(np.float32), std.astype(np.float32), quantize=True)
    assert float(loss.item()) == pytest.approx(rl, rel=1e-3)
    g_layers, _, _ = surrogate.unpack_params(grad.cpu().numpy())
    for l in range(5):
        for got, ref in [(g_layers[l][0], dW[l]), (g_layers[l][1], db[l])]:
            scale = np.abs(ref).mean() + 1e-12
            err = np.abs(got - ref)
            assert np.all(err <= 1e-2 * scale + 1e-2 * np.abs(ref)), (l, err.max() / scale)
            assert np.median(err / scale) < 1e-3


def test_tensor_core_gemm_matches_cuda_core_gemm(torch_dev):
    """The tcgen05 GEMMs (256-wide layers) against the CUDA-core kernel on the
    same bf16 operands: forward outputs and gradients, to accumulation order."""
    layers, mean, std = _net(8)
    params = torch_dev.as_tensor(surrogate.pack_params(layers, mean, std), device="cuda")
    n = 3000                                   # ragged: 23 full 128-row tiles and a tail
    x = torch_dev.as_tensor(_x(n, 9), dtype=torch_dev.float32, device="cuda")
    rng = np.random.default_rng(10)
    t = rng.normal(0, 1, (n, 5)) * std + mean
    t[:, 3] = (rng.uniform(size=n) > 0.2).astype(float)
    t = torch_dev.as_tensor(t, dtype=torch_dev.float32, device="cuda")
    out = {}
    lib = chert.lib()
    try:
        for tc in (1, 0):
            lib.chert_mlp_set_tensor_cores(tc)
            y = chert.mlp_forward(params, x)
            z = torch_dev.zeros_like(params)
            _, g = chert.mlp_train_step(params, z.clone(), z.clone(), 1, 0.0, x, t, want_grad=True)
            torch_dev.cuda.synchronize()
            out[tc] = (y.cpu().numpy(), g.cpu().numpy())
    finally:
        lib.chert_mlp_set_tensor_cores(1)
    for a, b in zip(out[1], out[0]):
        scale = np.abs(b).mean()
        assert np.all(np.abs(a - b) <= 1e-2 * scale + 1e-2 * np.abs(b))
        assert np.median(np.abs(a - b)) < 1e-4 * scale


@pytest.mark.parametrize("mode", ["qP", "qSV", "qSH"])
def test_training_pairs_match_oracle(torch_dev, mode):
    """Features, elastic baseline and targets from the oracle's exact cache."""
    classes = inputs.random_tti_classes(4, seed=11)
    M = 6
    mods, tilts = oracle_moduli(classes)
    cnp = co.build_cache(mods, tilts, [mode], M, "MEV", 0.02 * DEG, 1500)
    cache = chert.Cache(cache_to_torch(cnp, torch_dev.float64, "cuda"), [0], 4, M, chert.FP64)
    d_cls = chert.classes_to_device(chert.classes_from_layers(classes))
    x, t = chert.surrogate_dataset(d_cls, 4, M, mode, 0, cache)
    torch_dev.cuda.synchronize()
    x, t = x.cpu().numpy(), t.cpu().numpy()
    for k, L in enumerate(classes):
        aR = mods[k].real
        A = co.stiffness_tensor(mods[k])
        th = (math.pi / 2) * np.arange(M + 1) / M
        u, out = mo.features(th, np.full(M + 1, L.vs0 / L.vp0), np.full(M + 1, L.eps),
                             np.full(M + 1, L.delta), np.full(M + 1, L.gamma), np.full(M + 1, 1 / L.qp),
                             np.full(M + 1, 1 / L.qs))
        rows = slice(k * (M + 1), (k + 1) * (M + 1))
        assert np.allclose(x[rows, :7], u, atol=2e-6)
        Vg, psi_el = mo.elastic_baseline(aR, th, mode)
        A0 = mo.attenuation_baseline(mods[k], th, mode, psi_el)
        for j in range(M + 1):
            s = co.solve_direction(A, th[j], mode, "MEV", 0.02 * DEG, 1500)
            ref = mo.encode_targets(s["V"], s["A"], math.atan2(s["r"][0], s["r"][2]), s["flag"],
                                    s["vartheta"], Vg[j], psi_el[j], A0[j],
                                    vt_max=2 * DEG if mode == "qSV" else None)
            # A0 is evaluated in float on the device: log(A/A0) to 1e-5
            assert np.allclose(t[k * (M + 1) + j], ref, atol=[3e-6, 1e-5, 3e-6, 0, 3e-6], rtol=1e-5,
                               equal_nan=True), (k, j)


def test_trained_surrogate_beats_elastic_baseline(torch_dev):
    """Trained on exact entries of 512 seeded media, evaluated on 48 others:
    errors against the exact cache of the surrogate and of the elastic
    baseline alone (elastic group velocity and ray angle of the real moduli,
    homogeneous-wave attenuation A0: the network predicting no correction,
    computed by the oracle).  The network must cut the median ray-velocity
    error at least 3-fold in every mode and the median qP attenuation error.
    For qSH the decode uses A0 itself (exact for that mode), so its
    attenuation equals the baseline's; for qSV, where A0 is already within
    about 1e-5 of the exact value at the median, the network's attenuation
    is held to 2e-4 at the median."""
    from oracle import mlp_oracle as mo
    modes = ["qP", "qSV", "qSH"]
    M = 30
    train_sets = surrogate.exact_training_set(inputs.random_tti_classes(512, seed=21), modes, M)
    test_cls = inputs.random_tti_classes(48, seed=99)
    d_test = chert.classes_to_device(chert.classes_from_layers(test_cls))
    exact = chert.build_cache(d_test, 48, modes, M, kernel="MEV", precision="mixed")
    params = []
    for m in modes:
        x, t = train_sets[m]
        p, hist = surrogate.train(x, t, steps=1500, batch=2048, lr=2e-3, seed=1, log_every=500)
        params.append(p)
    surr = chert.surrogate_cache(params, d_test, 48, modes, M)
    torch_dev.cuda.synchronize()
    ex = {k: v.cpu().numpy()[:, :, :M + 1] for k, v in exact.arrays.items()}
    su = {k: v.cpu().numpy()[:, :, :M + 1] for k, v in surr.arrays.items()}
    decided = su["flag"] != 2                 # 2: handed to the exact solver
    agree = np.mean(((ex["flag"] == 0) == (su["flag"] == 0))[decided])
    assert agree > 0.99
    assert np.mean(decided[0]) > 0.9 and np.mean(decided[2]) > 0.9        # qP, qSH mostly decided
    mods, _ = oracle_moduli(test_cls)
    th = (math.pi / 2) * np.arange(M + 1) / M
    for mi, m in enumerate(modes):
        bV, bA = np.zeros((48, M + 1)), np.zeros((48, M + 1))
        for k in range(48):
            Vg, psi = mo.elastic_baseline(mods[k].real, th, m)
            bV[k], bA[k] = Vg, mo.attenuation_baseline(mods[k], th, m, psi)
        ok = (ex["flag"][mi] == 0) & (su["flag"][mi] == 0)

        def rel(a, key):
            return np.median(np.abs(a[ok] / ex[key][mi][ok] - 1))

        assert rel(su["V"][mi], "V") < rel(bV, "V") / 3, (m, rel(su["V"][mi], "V"), rel(bV, "V"))
        if m == "qP":
            assert rel(su["A"][mi], "A") < rel(bA, "A"), (m, rel(su["A"][mi], "A"), rel(bA, "A"))
        elif m == "qSH":
            assert np.allclose(su["A"][mi][ok], bA[ok], rtol=1e-6)
        else:
            assert rel(su["A"][mi], "A") < 2e-4, (m, rel(su["A"][mi], "A"))


def _decisive_nets(torch):
    """Untrained networks of the three modes whose validity logit (output 3)
    is scaled up, so that they call some solves valid, some invalid and leave
    some to the exact solver."""
    params = []
    for i in range(3):
        layers, mean, std = _net(40 + i)
        W, b = layers[-1]
        W = W.copy()
        W[3] *= 400.0
        layers = layers[:-1] + [(W, b)]
        params.append(torch.as_tensor(surrogate.pack_params(layers, mean, std), device="cuda"))
    return params


def test_cache_surrogate_one_call_equals_composed_flow(torch_dev):
    """chert_cache_surrogate (networks, then the flag-2 solves compacted on the
    device and recomputed exactly, with no host read) against the same steps
    composed on the host (chert_surrogate_cache, the list of flag-2 solves,
    chert_build_cache_items), bit for bit, with the same count of exact
    solves; no entry is left with flag 2; a CUDA-graph capture of the call
    replays the same cache."""
    torch = torch_dev
    modes, M, n = ["qP", "qSV", "qSH"], 30, 40
    params = _decisive_nets(torch)
    d_cls = chert.classes_to_device(chert.classes_from_layers(inputs.random_tti_classes(n, seed=7)))
    ref = chert.surrogate_cache(params, d_cls, n, modes, M, precision="fp32")
    items = torch.nonzero(ref["flag"][:, :, :M + 1].reshape(-1) == 2).flatten().to(torch.int64).contiguous()
    assert 0 < items.numel() < 3 * n * (M + 1)
    chert.build_cache_items(ref, d_cls, items, precision="mixed")
    got = chert.cache_surrogate(params, d_cls, n, modes, M, precision="mixed")
    torch.cuda.synchronize()
    assert got.n_fallback == items.numel()
    for k in ref.arrays:
        assert torch.equal(torch.nan_to_num(ref[k].float(), nan=-7.0), torch.nan_to_num(got[k].float(), nan=-7.0)), k
    assert not bool((got["flag"] == 2).any())
    # captured into a graph: the same cache on replay
    out = {k: torch.full_like(v, 0) for k, v in got.arrays.items()}
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        cap = chert.cache_surrogate(params, d_cls, n, modes, M, precision="mixed", out=out,
                                    stream=torch.cuda.current_stream())
    for _ in range(2):
        for v in out.values():
            v.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert int(cap.n_fallback_dev.item()) == items.numel()
        for k in ref.arrays:
            assert torch.equal(torch.nan_to_num(out[k].float(), nan=-7.0), torch.nan_to_num(got[k].float(), nan=-7.0)), k


def test_tensor_core_wait_that_runs_out_is_reported(torch_dev):
    """The bounded mbarrier waits of the tcgen05 GEMM: with the main-loop poll
    limit set to 0 every wait runs out at once (the TMA loads are still in
    flight), the kernel drains its loads, frees its tensor memory and returns,
    and chert_mlp_forward reports CHERT_ETIMEOUT.  chert_cache_surrogate then
    hands every solve to the exact solver, so its cache equals the exact
    build, and chert_mlp_check reports the time-out once.  With the limit
    restored the same context gives the same outputs as before."""
    torch = torch_dev
    modes, M, n = ["qP", "qSV", "qSH"], 30, 40
    params = _decisive_nets(torch)
    x = torch.as_tensor(_x(1000, 4), dtype=torch.float32, device="cuda")
    y0 = chert.mlp_forward(params[0], x)
    d_cls = chert.classes_to_device(chert.classes_from_layers(inputs.random_tti_classes(n, seed=7)))
    exact = chert.build_cache(d_cls, n, modes, M, kernel="MEV", precision="mixed")
    torch.cuda.synchronize()
    prev = chert.mlp_set_wait_limit(0)
    try:
        assert prev == 1 << 22
        with pytest.raises(chert.ChertError) as e:
            chert.mlp_forward(params[0], x)
        assert e.value.code == chert.ETIMEOUT
        c = chert.cache_surrogate(params, d_cls, n, modes, M, precision="mixed")
        torch.cuda.synchronize()
        assert c.n_fallback == len(modes) * n * (M + 1)
        with pytest.raises(chert.ChertError) as e:
            chert.mlp_check()
        assert e.value.code == chert.ETIMEOUT
    finally:
        chert.mlp_set_wait_limit(prev)
    chert.mlp_check()
    for k in exact.arrays:
        assert torch.equal(torch.nan_to_num(exact[k].float(), nan=-7.0), torch.nan_to_num(c[k].float(), nan=-7.0)), k
    y1 = chert.mlp_forward(params[0], x)
    torch.cuda.synchronize()
    assert torch.equal(y0, y1)
