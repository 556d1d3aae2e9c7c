"""What the cache surrogate gains on per-cell media (the paper's class-grouping
ablation): traveltimes of a folded and faulted model whose every node has its
own medium, computed with (a) the exact solver per cell -- the reference --,
(b) the method without the network, i.e. the exact solver on coarse classes
(one per layer, parameters averaged, as the paper's grouping does), and (c)
the networks per cell (exact fallback outside their training range)."""
import numpy as np
import pytest

from paper_2609_26108_b300 import chert, inputs, surrogate

pytestmark = pytest.mark.gpu

MODES = ["qP", "qSV", "qSH"]


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    from paper_2609_26108_b300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def _fields(torch, cache, model, cls, sources):
    d_cls = torch.as_tensor(cls.astype(np.int32), device="cuda")
    tR, tI, _, _ = chert.traveltime(cache, model.nx, model.nz, model.dx, d_cls, inputs.stencil_2d(5), sources,
                                    parents=False)
    torch.cuda.synchronize()
    return tR.cpu().numpy(), tI.cpu().numpy()


def test_surrogate_beats_coarse_grouping_per_cell(torch_dev):
    model = inputs.folded_faulted(nx=121, nz=61, n_layers=5, n_sources=3, seed=5)
    n = model.nx * model.nz
    p = model.params
    keys = ["vp0", "vs0", "eps", "delta", "gamma", "qp", "qs", "tilt"]
    d_cells = chert.classes_to_device(chert.classes_from_arrays(**{k: p[k] for k in keys}))
    M = 45
    exact = surrogate.per_cell_cache(d_cells, n, MODES, M)
    # (b) one class per layer, parameters averaged
    L = model.layer_of_node
    n_l = int(L.max()) + 1
    avg = {k: np.array([p[k][L == i].mean() for i in range(n_l)]) for k in keys}
    d_layers = chert.classes_to_device(chert.classes_from_arrays(**avg))
    grouped = chert.build_cache(d_layers, n_l, MODES, M, kernel="MEV", precision="mixed")
    # (c) networks trained on other seeded media
    train_sets = surrogate.exact_training_set(inputs.random_tti_classes(512, seed=21), MODES, 30)
    params = [surrogate.train(*train_sets[m], steps=1500, batch=2048, lr=2e-3, seed=1)[0] for m in MODES]
    surr = surrogate.per_cell_cache(d_cells, n, MODES, M, params)
    print("solves recomputed exactly: %d of %d" % (surr.n_fallback, n * len(MODES) * (M + 1)))
    src = [int(s) for s in model.sources]
    ref = _fields(torch_dev, exact, model, np.arange(n), src)
    grp = _fields(torch_dev, grouped, model, L, src)
    sur = _fields(torch_dev, surr, model, np.arange(n), src)
    for comp in (0, 1):
        for mi, m in enumerate(MODES):
            r = ref[comp][:, mi]
            ok = np.isfinite(r) & (r > 0)
            e_g = np.median(np.abs(grp[comp][:, mi][ok] - r[ok]) / r[ok])
            e_s = np.median(np.abs(sur[comp][:, mi][ok] - r[ok]) / r[ok])
            print("component %d %s: median rel error grouped %.3e, surrogate %.3e" % (comp, m, e_g, e_s))
            assert e_s < 0.05 * e_g, (comp, m, e_s, e_g)
