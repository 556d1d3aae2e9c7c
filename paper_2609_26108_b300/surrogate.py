"""Training and use of the cache surrogate (one MLP per wave mode).

Orchestration only: the exact cache, the training pairs, every training step
and the surrogate cache run in libchert's kernels (`chert_build_cache`,
`chert_surrogate_dataset`, `chert_mlp_train_step`, `chert_surrogate_cache`).
"""
from __future__ import annotations

import math

import numpy as np

from . import chert, inputs


def pack_params(layers, out_mean, out_std):
    """Flat float32 parameter vector (the ABI's layout) from [(W, b), ...]."""
    parts = []
    for W, b in layers:
        parts += [np.asarray(W, np.float64).reshape(-1), np.asarray(b, np.float64).reshape(-1)]
    parts += [np.asarray(out_mean, np.float64), np.asarray(out_std, np.float64)]
    v = np.concatenate(parts).astype(np.float32)
    assert v.size == chert.mlp_param_count()
    return v


def unpack_params(vec):
    """[(W, b), ...], out_mean, out_std from a flat parameter vector."""
    v = np.asarray(vec, np.float64)
    sizes = [7, 256, 256, 256, 256, 5]
    o, layers = 0, []
    for a, b in zip(sizes[:-1], sizes[1:]):
        W = v[o:o + a * b].reshape(b, a); o += a * b
        bb = v[o:o + b]; o += b
        layers.append((W, bb))
    return layers, v[o:o + 5], v[o + 5:o + 10]


def exact_training_set(classes, modes, M, precision="mixed"):
    """(x, t) per mode from the exact cache of `classes` (device tensors)."""
    d_cls = chert.classes_to_device(chert.classes_from_layers(classes))
    cache = chert.build_cache(d_cls, len(classes), modes, M, kernel="MEV", precision=precision)
    return {m: chert.surrogate_dataset(d_cls, len(classes), M, m, i, cache) for i, m in enumerate(modes)}


def standardisation(t):
    """Mean/std of the raw targets over valid samples, NaN targets left out
    (output 3 left as is)."""
    import torch
    valid = t[:, 3] > 0.5
    tv = t[valid].double()
    mean = tv.nanmean(0)
    var = ((tv - mean) ** 2).nanmean(0)
    std = var.sqrt().clamp_min(1e-12)
    mean[3], std[3] = 0.0, 1.0
    return mean.cpu().numpy(), std.cpu().numpy()


def train(x, t, steps=2000, batch=4096, lr=2e-3, seed=0, log_every=0):
    """Train one network on (x [n, 8], t [n, 5]) device tensors; returns the
    parameter tensor and the loss history."""
    import torch
    mean, std = standardisation(t)
    init = inputs.mlp_init(seed)
    params = torch.as_tensor(pack_params(init, mean, std), device=x.device)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    gen = torch.Generator(device=x.device)
    gen.manual_seed(seed)
    ws = torch.empty(int(chert.lib().chert_mlp_workspace_bytes(batch, 1)), dtype=torch.uint8, device=x.device)
    loss = torch.zeros(1, dtype=torch.float32, device=x.device)
    history = []
    for step in range(1, steps + 1):
        idx = torch.randint(0, x.shape[0], (batch,), device=x.device, generator=gen)
        rate = lr * 0.5 * (1 + math.cos(math.pi * (step - 1) / steps))     # cosine decay
        chert.mlp_train_step(params, m, v, step, rate, x[idx].contiguous(), t[idx].contiguous(),
                             workspace=ws, loss=loss)
        if log_every and step % log_every == 0:
            history.append((step, float(loss.item())))
    return params, history


def per_cell_cache(d_classes, n_cells, modes, M, params_per_mode=None, precision="mixed", out=None, stream=None):
    """Cache with one class per cell: exact (params_per_mode None) or from the
    networks, with every solve they hand back (flag 2: outside the training
    range, unsure validity, qSV branch region) recomputed by the exact solver
    -- chert_cache_surrogate, which keeps the fallback list on the device, so
    this enqueues without a host read (and can be captured into a graph).
    out: optional preallocated cache arrays (the layout of build_cache).
    The surrogate form's cache.n_fallback reads the number of exact solves
    (one device-to-host copy)."""
    if params_per_mode is None:
        return chert.build_cache(d_classes, n_cells, modes, M, kernel="MEV", precision=precision, out=out,
                                 stream=stream)
    return chert.cache_surrogate(params_per_mode, d_classes, n_cells, modes, M, kernel="MEV",
                                 precision=precision, out=out, stream=stream)
