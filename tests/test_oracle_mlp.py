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
