"""FP64 oracle of the cache surrogate -- TEST INFRASTRUCTURE ONLY.

Only tests, the smoke check and the benchmark's CPU-baseline leg may call this.

The surrogate replaces the homogeneity solve of one cache entry (the paper's
Eq. 9-11 at a folded slowness angle) by a small network: per wave mode an MLP
7 -> 256 -> 256 -> 256 -> 256 -> 5 with SiLU hidden activations predicts a
correction to the exact *elastic* ray quantities of the same medium.  This
module restates, in plain numpy double precision:

* ``elastic_baseline``  the elastic phase velocity of the real moduli (the
  eigenvalue of the 2x2 x-z Christoffel block, or a66 sin^2 + a44 cos^2 for
  qSH), its angular derivative by a complex step, and from them the group
  velocity Vg = sqrt(V^2 + V'^2) and ray angle psi = theta + atan2(V', V).
* ``attenuation_baseline``  the attenuation A0 of the homogeneous plane wave
  whose slowness points along theta: Im(1/c) for the complex phase velocity
  c = sqrt(lambda) of the complex Christoffel block, projected on the elastic
  ray direction, cos(psi_el - theta) Im(1/c).
* ``features`` / ``encode_targets`` / ``decode``  the fixed input scaling and
  the output parametrisation (V/Vg - 1, log(A/A0), psi - psi_el, validity
  logit, vartheta).
* ``forward`` / ``backward`` / ``adam``  the network, the gradient of the
  masked mean-square + logistic loss, and Adam with bias correction.

Parity status: forward and backward are pinned by finite differences and by
explicit loops; the elastic baseline is pinned by the oracle's own exact cache
in the elastic limit, the attenuation baseline by the exact cache where the
exact wave is homogeneous (isotropic media, and the symmetry axis of a VTI
medium); ``bf16`` by an independent round-to-nearest-even cast (exact
halfway cases, signed zeros, subnormals, the top of the range) and two
halfway cases by hand; ``encode_targets`` and ``decode`` by hand-computed
cases and by their round trip.  The learned weights have no pin: they are an
approximation whose error the tests measure against the exact cache.
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_HID, N_LAYERS, N_OUT = 7, 256, 4, 5
# fixed input ranges (the training range of the seeded TTI media)
IN_LO = np.array([0.0, 0.49, 0.04, -0.11, 0.0, 0.004, 0.004])
IN_HI = np.array([math.pi / 2, 0.6, 0.31, 0.21, 0.21, 0.051, 0.051])


def elastic_baseline(aR, theta, mode):
    """Elastic group velocity and ray angle (x from +z toward +x) for real
    moduli aR = (a11, a13, a33, a44, a66) at slowness angles theta."""
    a11, a13, a33, a44, a66 = [float(v) for v in aR]
    h = 1e-30

    def phase(t):
        s2, c2 = np.sin(t) ** 2, np.cos(t) ** 2
        if mode == "qSH":
            lam = a66 * s2 + a44 * c2
        else:
            g11 = a11 * s2 + a44 * c2
            g33 = a44 * s2 + a33 * c2
            g13 = (a13 + a44) * np.sin(t) * np.cos(t)
            root = np.sqrt((g11 - g33) ** 2 + 4 * g13 * g13)
            lam = 0.5 * (g11 + g33 + (root if mode == "qP" else -root))
        return np.sqrt(lam)

    z = np.asarray(theta, dtype=np.float64) + 1j * h
    Vc = phase(z)
    V, dV = Vc.real, Vc.imag / h
    return np.sqrt(V * V + dV * dV), np.asarray(theta) + np.arctan2(dV, V)


def attenuation_baseline(a, theta, mode, psi_el):
    """Homogeneous-wave attenuation for complex moduli a = (a11, a13, a33,
    a44, a66) (a = aR - i aI) at slowness angles theta, projected on the ray
    direction psi_el."""
    a11, a13, a33, a44, a66 = [complex(v) for v in a]
    t = np.asarray(theta, dtype=np.float64)
    out = np.zeros(t.shape)
    for idx in np.ndindex(t.shape):
        s, c = math.sin(t[idx]), math.cos(t[idx])
        if mode == "qSH":
            lam = a66 * s * s + a44 * c * c
        else:
            G = np.array([[a11 * s * s + a44 * c * c, (a13 + a44) * s * c],
                          [(a13 + a44) * s * c, a44 * s * s + a33 * c * c]])
            ev = np.linalg.eigvals(G)
            ev = ev[np.argsort(ev.real)]
            lam = ev[1] if mode == "qP" else ev[0]
        slowness = 1.0 / np.sqrt(lam)
        out[idx] = slowness.imag * math.cos(float(np.asarray(psi_el)[idx]) - t[idx])
    return out


def features(theta_fold, rs, eps, delta, gamma, inv_qp, inv_qs):
    """Inputs scaled to [-1, 1] over the training range; also returns the
    mask of samples outside that range."""
    x = np.stack([theta_fold, rs, eps, delta, gamma, inv_qp, inv_qs], axis=-1).astype(np.float64)
    u = 2.0 * (x - IN_LO) / (IN_HI - IN_LO) - 1.0
    outside = np.any(np.abs(u) > 1.0, axis=-1)
    return u, outside


def encode_targets(V, A, psi, flag, vartheta, Vg, psi_el, A0, vt_max=None):
    """Network targets: (V/Vg - 1, log(A/A0), psi - psi_el, valid, vartheta).
    A and A0 share their unit; either one under 1e-30 of it counts as 1e-30.
    With vt_max, samples with |vartheta| > vt_max get NaN for outputs 0-2
    (left out of the fit of those outputs)."""
    valid = (np.asarray(flag) == 0)
    t = np.zeros(np.shape(V) + (N_OUT,))
    t[..., 0] = np.where(valid, V / Vg - 1.0, 0.0)
    ratio = np.maximum(np.where(valid, A, 1.0), 1e-30) / np.maximum(A0, 1e-30)
    t[..., 1] = np.where(valid, np.log(ratio), 0.0)
    t[..., 2] = np.where(valid, np.angle(np.exp(1j * (psi - psi_el))), 0.0)
    t[..., 3] = valid.astype(np.float64)
    t[..., 4] = np.where(valid, vartheta, 0.0)
    if vt_max is not None:
        far = valid & (np.abs(vartheta) > vt_max)
        t[far, 0:3] = np.nan
    return t


def init_params(seed):
    """He-style initialisation; W[l] is [out, in], b[l] is [out]."""
    rng = np.random.default_rng(seed)
    sizes = [N_IN] + [N_HID] * N_LAYERS + [N_OUT]
    W, b = [], []
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        W.append(rng.normal(0.0, math.sqrt(2.0 / fan_in), (fan_out, fan_in)))
        b.append(np.zeros(fan_out))
    return W, b


def bf16(a):
    """Round to bfloat16 (round to nearest even), via float32, returned as float64."""
    a32 = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = a32.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(x):
    return x / (1.0 + np.exp(-x))


def dsilu(x):
    s = 1.0 / (1.0 + np.exp(-x))
    return s * (1.0 + x * (1.0 - s))


def forward(W, b, x, quantize=False):
    """Returns the output and the pre-activations of every layer.  With
    quantize=True the inputs of every product (activations, weights) are
    rounded to bfloat16 first, as a BF16-operand network computes."""
    q = bf16 if quantize else (lambda a: a)
    pre, h = [], q(x)
    for l in range(len(W)):
        z = h @ q(W[l]).T + b[l]
        pre.append(z)
        h = q(silu(z)) if l < len(W) - 1 else z
    return h, pre


def loss_and_grad(W, b, x, target, out_mean, out_std, quantize=False):
    """Mean over the batch of: sum over outputs 0,1,2,4 of ((y - t')^2)/2 on
    valid samples whose target is not NaN (t' = standardised target) +
    logistic loss of output 3.
    Returns (loss, dW, db).  With quantize=True every product operand
    (activations, weights and back-propagated gradients) is rounded to
    bfloat16 first, as BF16-operand training computes."""
    q = bf16 if quantize else (lambda a: a)
    y, pre = forward(W, b, x, quantize)
    n = x.shape[0]
    valid = target[:, 3] > 0.5
    tstd = (target - out_mean) / out_std
    g = np.zeros_like(y)
    loss = 0.0
    for k in (0, 1, 2, 4):
        use = valid & ~np.isnan(tstd[:, k])
        d = np.where(use, y[:, k] - np.where(use, tstd[:, k], 0.0), 0.0)
        loss += 0.5 * np.sum(d * d)
        g[:, k] = d
    p = 1.0 / (1.0 + np.exp(-y[:, 3]))
    loss += np.sum(np.logaddexp(0.0, y[:, 3]) - target[:, 3] * y[:, 3])
    g[:, 3] = p - target[:, 3]
    loss /= n
    g /= n
    dW, db = [None] * len(W), [None] * len(W)
    for l in reversed(range(len(W))):
        h_in = q(x) if l == 0 else q(silu(pre[l - 1]))
        dW[l] = q(g).T @ h_in
        db[l] = g.sum(axis=0)
        if l > 0:
            g = (q(g) @ q(W[l])) * dsilu(pre[l - 1])
    return loss, dW, db


def adam(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update with bias correction (in place); step counts from 1."""
    for p, g, mm, vv in zip(params, grads, m, v):
        mm *= beta1
        mm += (1 - beta1) * g
        vv *= beta2
        vv += (1 - beta2) * g * g
        mhat = mm / (1 - beta1 ** step)
        vhat = vv / (1 - beta2 ** step)
        p -= lr * mhat / (np.sqrt(vhat) + eps)


def decode(y, out_mean, out_std, Vg, psi_el, A0):
    """Network output -> (V, A, psi, p_valid, vartheta)."""
    t = y * out_std + out_mean
    V = Vg * (1.0 + t[..., 0])
    A = A0 * np.exp(t[..., 1])
    psi = psi_el + t[..., 2]
    p_valid = 1.0 / (1.0 + np.exp(-y[..., 3]))
    return V, A, psi, p_valid, t[..., 4]
