"""Pins of the surrogate oracle: gradient by finite differences, forward by
explicit loops, Adam by hand, the elastic baseline by the exact cache oracle."""
import math

import numpy as np
import pytest

from oracle import cache_oracle as co
from oracle import mlp_oracle as mo


def _tiny(seed=0):
    rng = np.random.default_rng(seed)
    sizes = [7, 6, 5, 5]
    W = [rng.normal(0, 0.7, (o, i)) for i, o in zip(sizes[:-1], sizes[1:])]
    b = [rng.normal(0, 0.1, o) for o in sizes[1:]]
    return W, b


def test_forward_matches_explicit_loops():
    W, b = _tiny()
    x = np.random.default_rng(1).uniform(-1, 1, (3, 7))
    y, _ = mo.forward(W, b, x)
    for n in range(3):
        h = list(x[n])
        for l in range(len(W)):
            z = [sum(W[l][o][i] * h[i] for i in range(len(h))) + b[l][o] for o in range(len(b[l]))]
            h = [v / (1 + math.exp(-v)) for v in z] if l < len(W) - 1 else z
        assert np.allclose(y[n], h, rtol=1e-13)


def test_gradient_matches_finite_differences():
    W, b = _tiny(2)
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, (9, 7))
    t = rng.normal(0, 1, (9, 5))
    t[:, 3] = (rng.uniform(size=9) > 0.3).astype(float)
    mean, std = rng.normal(0, 0.1, 5), rng.uniform(0.5, 2, 5)
    mean[3], std[3] = 0.0, 1.0
    loss, dW, db = mo.loss_and_grad(W, b, x, t, mean, std)
    h = 1e-6
    for l in range(len(W)):
        for (o, i) in [(0, 0), (1, 2), (W[l].shape[0] - 1, W[l].shape[1] - 1)]:
            W[l][o, i] += h
            lp, _, _ = mo.loss_and_grad(W, b, x, t, mean, std)
            W[l][o, i] -= 2 * h
            lm, _, _ = mo.loss_and_grad(W, b, x, t, mean, std)
            W[l][o, i] += h
            assert dW[l][o, i] == pytest.approx((lp - lm) / (2 * h), rel=1e-6, abs=1e-9)
        b[l][0] += h
        lp, _, _ = mo.loss_and_grad(W, b, x, t, mean, std)
        b[l][0] -= 2 * h
        lm, _, _ = mo.loss_and_grad(W, b, x, t, mean, std)
        b[l][0] += h
        assert db[l][0] == pytest.approx((lp - lm) / (2 * h), rel=1e-6, abs=1e-9)


def test_nan_target_is_left_out():
    """A NaN target adds what a target equal to the network's own output adds:
    nothing, to the loss and to every gradient."""
    W, b = _tiny(4)
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, (6, 7))
    t = rng.normal(0, 1, (6, 5))
    t[:, 3] = 1.0
    mean, std = rng.normal(0, 0.1, 5), rng.uniform(0.5, 2, 5)
    mean[3], std[3] = 0.0, 1.0
    y, _ = mo.forward(W, b, x)
    t_nan, t_same = t.copy(), t.copy()
    for i, k in [(1, 0), (1, 2), (4, 1), (5, 4)]:
        t_nan[i, k] = np.nan
        t_same[i, k] = y[i, k] * std[k] + mean[k]
    l1, dW1, db1 = mo.loss_and_grad(W, b, x, t_nan, mean, std)
    l2, dW2, db2 = mo.loss_and_grad(W, b, x, t_same, mean, std)
    assert np.isfinite(l1) and l1 == pytest.approx(l2, rel=1e-12)
    for a, c in zip(dW1 + db1, dW2 + db2):
        assert np.allclose(a, c, rtol=1e-10, atol=1e-14)


def test_adam_two_steps_by_hand():
    p = [np.array([1.0])]
    m, v = [np.zeros(1)], [np.zeros(1)]
    mo.adam(p, [np.array([0.5])], m, v, 1, 0.1)
    # step 1: mhat = g, vhat = g^2 -> p -= lr * g/|g| = 0.1
    assert p[0][0] == pytest.approx(0.9, abs=1e-7)
    mo.adam(p, [np.array([-0.25])], m, v, 2, 0.1)
    m2 = 0.9 * 0.05 + 0.1 * -0.25
    v2 = 0.999 * (0.001 * 0.25) + 0.001 * 0.0625
    mh, vh = m2 / (1 - 0.81), v2 / (1 - 0.999 ** 2)
    p1 = 1.0 - 0.1 * 0.5 / (0.5 + 1e-8)
    assert p[0][0] == pytest.approx(p1 - 0.1 * mh / (math.sqrt(vh) + 1e-8), rel=1e-12)


@pytest.mark.parametrize("mode", ["qP", "qSV", "qSH"])
def test_elastic_baseline_matches_exact_cache(mode):
    """Elastic limit: the baseline is the exact ray velocity and direction."""
    aR = np.array([14.4e6, 4.5e6, 9.0e6, 2.25e6, 3.0e6])
    A = co.stiffness_tensor(aR.astype(complex))
    th = np.array([0.2, 0.7, 1.2])
    Vg, psi = mo.elastic_baseline(aR, th, mode)
    for i, t in enumerate(th):
        s = co.solve_direction(A, t, mode, "OEV", 0.05 * math.pi / 180, 600)
        assert Vg[i] == pytest.approx(s["V"], rel=1e-11)
        assert psi[i] == pytest.approx(math.atan2(s["r"][0], s["r"][2]), abs=1e-11)


@pytest.mark.parametrize("mode", ["qP", "qSV", "qSH"])
def test_attenuation_baseline_isotropic_is_exact(mode):
    """An isotropic anelastic solid carries homogeneous waves in every
    direction (vartheta = 0, ray along the slowness), so there the baseline is
    the exact attenuation of the cache solve."""
    a33, a44 = 9.0e6 * (1 - 1j / 50), 2.25e6 * (1 - 1j / 30)
    a = np.array([a33, a33 - 2 * a44, a33, a44, a44])
    A = co.stiffness_tensor(a)
    th = np.array([0.1, 0.6, 1.3])
    A0 = mo.attenuation_baseline(a, th, mode, th)
    for i, t in enumerate(th):
        s = co.solve_direction(A, t, mode, "MEV", 0.05 * math.pi / 180, 600)
        assert s["flag"] == 0 and abs(s["vartheta"]) < 1e-12
        assert A0[i] == pytest.approx(s["A"], rel=1e-10)


@pytest.mark.parametrize("mode", ["qP", "qSV", "qSH"])
def test_attenuation_baseline_on_vti_axis_is_exact(mode):
    """Along the symmetry axis of a VTI solid the exact wave is homogeneous
    and the ray vertical, whatever the anisotropy and the quality factors."""
    aR = np.array([14.4e6, 4.5e6, 9.0e6, 2.25e6, 3.0e6])
    a = aR * (1 - 1j / np.array([40.0, 40.0, 40.0, 25.0, 25.0]))
    s = co.solve_direction(co.stiffness_tensor(a), 0.0, mode, "MEV", 0.05 * math.pi / 180, 600)
    A0 = mo.attenuation_baseline(a, np.array([0.0]), mode, np.array([0.0]))
    assert s["flag"] == 0
    assert A0[0] == pytest.approx(s["A"], rel=1e-10)
    # and the positive value Im(1/c) of a decaying wave
    assert A0[0] > 0


def test_attenuation_baseline_elastic_is_zero():
    aR = np.array([14.4e6, 4.5e6, 9.0e6, 2.25e6, 3.0e6])
    th = np.linspace(0, math.pi / 2, 5)
    for mode in ("qP", "qSV", "qSH"):
        assert np.all(mo.attenuation_baseline(aR.astype(complex), th, mode, th) == 0.0)


def test_features_scale_and_range():
    u, out = mo.features(np.array([0.0, math.pi / 2]), np.array([0.49, 0.6]), np.array([0.04, 0.31]),
                         np.array([-0.11, 0.21]), np.array([0.0, 0.21]), np.array([0.004, 0.051]),
                         np.array([0.004, 0.051]))
    assert np.allclose(u[0], -1) and np.allclose(u[1], 1) and not out.any()
    _, out2 = mo.features(np.array([0.1]), np.array([0.7]), np.array([0.1]), np.array([0.0]),
                          np.array([0.1]), np.array([0.01]), np.array([0.01]))
    assert out2[0]


def test_bf16_matches_an_independent_rounding():
    """bf16 against torch's float32 -> bfloat16 cast (round to nearest even),
    on random values over many binades, exact halfway cases, signed zeros,
    subnormals and values near the top of the range; and two halfway cases by
    hand: 1 + 2^-8 rounds down to the even 1, 1 + 3*2^-8 up to the even
    1 + 2^-6."""
    import torch
    rng = np.random.default_rng(3)
    x = rng.standard_normal(20000) * np.exp(rng.uniform(-60, 60, 20000))
    # float32 patterns whose low 16 bits are exactly 0x8000: halfway between
    # two bfloat16 values, half with an even and half with an odd upper part
    expo = rng.integers(1, 254, 4000).astype(np.uint32)
    mant = rng.integers(0, 128, 4000).astype(np.uint32)
    bits = (((expo << np.uint32(7)) | mant) << np.uint32(16)) | np.uint32(0x8000)
    halfway = bits.view(np.float32).astype(np.float64) * np.where(rng.random(4000) < 0.5, -1.0, 1.0)
    subnormal = np.array([1e-40, -3e-42, 1.17e-38, 5e-45, 2.3e-39], np.float64)
    special = np.array([0.0, -0.0, 3.3e38, -3.3e38, 3.39e38, 1.0, -1.0, 65504.0, np.inf, -np.inf])
    for vals in (x, halfway, subnormal, special):
        f32 = vals.astype(np.float32)
        want = torch.tensor(f32).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
        got = mo.bf16(f32)
        assert np.array_equal(got, want)
        assert np.array_equal(np.signbit(got), np.signbit(want))
    assert mo.bf16(np.float32(1 + 2.0 ** -8)) == 1.0
    assert mo.bf16(np.float32(1 + 3 * 2.0 ** -8)) == 1 + 2.0 ** -6
    assert mo.bf16(np.float32(1 + 2.0 ** -8 + 2.0 ** -20)) == 1 + 2.0 ** -7   # just past halfway rounds up


def test_encode_targets_hand_cases():
    """Each output by hand: V/Vg - 1, log(A/A0) (with the 1e-30 floor), the ray
    angle difference wrapped into (-pi, pi], the validity, vartheta, and the
    NaN mask of far qSV roots."""
    V = np.array([2100.0, 2000.0, 1500.0, 1800.0])
    Vg = np.array([2000.0, 2000.0, 1500.0, 2000.0])
    A = np.array([2e-5, 1e-5, 3e-6, 0.0])
    A0 = np.array([1e-5, 1e-5, 3e-6, 1e-5])
    psi = np.array([0.3, 3.1, -3.1, 0.0])
    psi_el = np.array([0.1, -3.1, 3.1, 0.0])
    flag = np.array([0, 0, 0, 1])
    vt = np.array([0.01, -0.02, 0.05, np.nan])
    t = mo.encode_targets(V, A, psi, flag, vt, Vg, psi_el, A0, vt_max=0.03)
    assert np.allclose(t[0], [0.05, math.log(2.0), 0.2, 1.0, 0.01], rtol=1e-14, atol=1e-15)
    assert np.allclose(t[1], [0.0, 0.0, 6.2 - 2 * math.pi, 1.0, -0.02], rtol=0, atol=1e-14)
    assert np.all(np.isnan(t[2, :3])) and t[2, 3] == 1.0 and t[2, 4] == 0.05
    assert np.array_equal(t[3], [0.0, 0.0, 0.0, 0.0, 0.0])
    tiny = mo.encode_targets(np.array([1.0]), np.array([1e-40]), np.array([0.0]), np.array([0]),
                             np.array([0.0]), np.array([1.0]), np.array([0.0]), np.array([1e-30]))
    assert tiny[0, 1] == 0.0                                     # both floored at 1e-30


def test_decode_hand_cases_and_round_trip():
    """decode by hand (logit 0 -> p = 1/2, log 3 -> p = 3/4) and as the inverse
    of encode_targets followed by the standardisation y = (t - mean)/std."""
    out_mean = np.array([0.02, 0.1, -0.01, 0.0, 0.003])
    out_std = np.array([0.05, 0.3, 0.02, 1.0, 0.01])
    y = np.array([[0.0, 0.0, 0.0, 0.0, 0.0], [1.0, -1.0, 2.0, math.log(3.0), -0.5]])
    V, A, psi, p, vt = mo.decode(y, out_mean, out_std, np.array([2000.0, 2000.0]), np.array([0.4, 0.4]),
                                 np.array([1e-5, 1e-5]))
    assert np.allclose(V, [2000.0 * 1.02, 2000.0 * 1.07], rtol=1e-14)
    assert np.allclose(A, [1e-5 * math.exp(0.1), 1e-5 * math.exp(-0.2)], rtol=1e-14)
    assert np.allclose(psi, [0.39, 0.43], rtol=0, atol=1e-15)
    assert np.allclose(p, [0.5, 0.75], rtol=1e-14)
    assert np.allclose(vt, [0.003, -0.002], rtol=0, atol=1e-16)
    rng = np.random.default_rng(8)
    n = 500
    Vg = rng.uniform(1500, 4500, n)
    psi_el = rng.uniform(-math.pi, math.pi, n)
    A0 = rng.uniform(1e-6, 1e-4, n)
    V = Vg * rng.uniform(0.9, 1.1, n)
    A = A0 * rng.uniform(0.5, 2.0, n)
    psi = np.angle(np.exp(1j * (psi_el + rng.uniform(-0.3, 0.3, n))))
    vt = rng.uniform(-0.05, 0.05, n)
    t = mo.encode_targets(V, A, psi, np.zeros(n, int), vt, Vg, psi_el, A0)
    y = (t - out_mean) / out_std
    V2, A2, psi2, p2, vt2 = mo.decode(y, out_mean, out_std, Vg, psi_el, A0)
    assert np.allclose(V2, V, rtol=1e-12)
    assert np.allclose(A2, A, rtol=1e-12)
    assert np.allclose(np.angle(np.exp(1j * (psi2 - psi))), 0.0, atol=1e-12)
    assert np.allclose(vt2, vt, rtol=0, atol=1e-15)
    assert np.all(p2 > 0.73)                         # validity 1 -> logit (1 - 0)/1 = 1 -> p = 0.731
