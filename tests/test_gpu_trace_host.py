"""chert_trace_host (the whole path as one call on host buffers) returns the
same fields and raypaths, bit for bit, as the same steps run on device
buffers (Tracer: cache build, traveltime with parents, raypaths), and reports
the same errors."""
import math

import numpy as np
import pytest

from paper_2609_26108_b300 import chert, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    from paper_2609_26108_b300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.mark.parametrize("precision,pinned,scheduler,n_sources",
                         [("mixed", True, "hybrid", 5), ("fp64", True, "hybrid", 5), ("mixed", False, "hybrid", 5),
                          ("mixed", True, "block_heap", 5), ("mixed", True, "hybrid", 120),
                          ("fp64", False, "hybrid", 120)])
def test_trace_host_equals_device_path(torch_dev, precision, pinned, scheduler, n_sources):
    """Page-locked and pageable outputs, two schedulers, and 120 sources x 3
    modes: more field components than two resident CTAs a SM, so the call
    relaxes the sources in waves and copies each wave back while the next
    relaxes."""
    torch = torch_dev
    prev = chert.set_relax_scheduler(scheduler)
    try:
        _trace_host_case(torch, precision, pinned, n_sources)
    finally:
        chert.set_relax_scheduler(prev)


def _trace_host_case(torch, precision, pinned, n_sources):
    from paper_2609_26108_b300.pipeline import HostTracer, Tracer
    model = inputs.layered_tti(nx=83, nz=61, n_layers=4, n_sources=n_sources)
    off = inputs.stencil_2d(4)
    rcv = np.array([0, 41, 82, 83 * 60 + 7, 83 * 30 + 30], np.int64)
    M, h, K = 18, 0.02 * math.pi / 180, 1500
    classes = chert.classes_from_layers(model.layers)
    d_classes = chert.classes_to_device(classes)
    cls = model.class_of_node.astype(np.int32)
    rel = "fp64" if precision == "fp64" else "fp32"
    ns = len(model.sources)
    tr = Tracer(4, ["qP", "qSV", "qSH"], M, model.nx, model.nz, model.dx, off, ns, rcv, cache_precision=precision,
                precision=rel, scan_step=h, scan_half=K, path_cap=256)
    tr.set_inputs(d_classes, torch.as_tensor(cls, device="cuda"), model.sources)
    tR, tI, _, _ = tr.run()
    torch.cuda.synchronize()
    ht = HostTracer(4, ["qP", "qSV", "qSH"], M, model.nx, model.nz, model.dx, off, ns, rcv, precision=precision,
                    scan_step=h, scan_half=K, path_cap=256, pinned=pinned)
    assert ht.h_tau[0].is_pinned() == pinned
    h_src = torch.as_tensor(np.asarray(model.sources, np.int64)).pin_memory()
    for _ in range(2):                               # twice: nothing carries over between calls
        hR, hI, hp, hl = ht.run(d_classes.cpu().pin_memory(), torch.as_tensor(cls).pin_memory(), h_src)
        assert torch.equal(hR, tR.cpu()) and torch.equal(hI, tI.cpu())
        nf = 3 * ns
        for c in (0, 1):
            assert torch.equal(hl[c], tr.paths[1][c * nf:(c + 1) * nf].cpu())
            for f in range(nf):
                for r in range(len(rcv)):
                    n = int(hl[c, f, r])
                    assert n > 0
                    assert torch.equal(hp[c, f, r, :n], tr.paths[0][c * nf + f, r, :n].cpu())


def test_trace_host_reports_bad_class_map(torch_dev):
    from paper_2609_26108_b300.pipeline import HostTracer
    torch = torch_dev
    model = inputs.layered_tti(nx=20, nz=15, n_layers=2, n_sources=1)
    classes = chert.classes_from_layers(model.layers)
    ht = HostTracer(2, ["qP"], 6, model.nx, model.nz, model.dx, inputs.stencil_2d(2), 1, [5], scan_step=0.05 * math.pi / 180,
                    scan_half=600, path_cap=64)
    cls = model.class_of_node.astype(np.int32)
    cls[7] = 5                                        # outside [0, 2)
    with pytest.raises(chert.ChertError) as e:
        ht.run(chert.classes_to_device(classes).cpu().pin_memory(), torch.as_tensor(cls).pin_memory(),
               torch.as_tensor(np.asarray(model.sources, np.int64)).pin_memory())
    assert e.value.code == chert.EINVAL
