"""The whole CHERT hot path as one object (Algorithm 2 of the paper).

``Tracer`` holds the device buffers of one problem size and runs, per call,
cache build -> direction lookup + relaxation + parents -> raypaths, all in
libchert's kernels on the current torch stream.  ``run()`` works on resident
device inputs; ``run_host()`` is the end-to-end call for host data: it copies
the inputs from (pinned) host memory, runs the path and copies the traveltime
fields back.
"""
from __future__ import annotations

import math

import numpy as np

from . import chert


class Tracer:
    def __init__(self, n_classes, modes, M, nx, nz, dx, offsets, n_sources, receivers,
                 kernel="MEV", cache_precision="mixed", precision="fp32",
                 scan_step=0.001 * math.pi / 180, scan_half=30000, max_cycles=64, path_cap=1024,
                 device="cuda"):
        import torch
        self.torch = torch
        self.n_classes, self.modes, self.M = n_classes, list(modes), M
        self.nx, self.nz, self.dx = nx, nz, dx
        self.offsets = np.ascontiguousarray(np.asarray(offsets, np.int32).reshape(-1, 3))
        self.n_sources = n_sources
        self.receivers = np.asarray(receivers, np.int64)
        self.kernel, self.scan_step, self.scan_half = kernel, scan_step, scan_half
        self.max_cycles, self.path_cap = max_cycles, path_cap
        self.cprec = chert.PRECISION_IDS[cache_precision]
        self.prec = chert.PRECISION_IDS[precision]
        if (self.cprec == chert.FP64) != (self.prec == chert.FP64):
            raise ValueError("cache storage and relaxation must both be fp64 or both float")
        fd = torch.float64 if self.prec == chert.FP64 else torch.float32
        nm, nd, n = len(self.modes), 4 * M, nx * nz
        shape = (nm, n_classes, nd)
        self.cache_out = {k: torch.empty(shape, dtype=fd, device=device)
                          for k in ("V", "A", "Q", "rx", "rz", "theta", "vartheta")}
        self.cache_out["flag"] = torch.empty(shape, dtype=torch.uint8, device=device)
        fshape = (n_sources, nm, n)
        self.tau = (torch.empty(fshape, dtype=fd, device=device), torch.empty(fshape, dtype=fd, device=device),
                    torch.empty(fshape, dtype=torch.int32, device=device),
                    torch.empty(fshape, dtype=torch.int32, device=device))
        wsb = chert.workspace_bytes(nm, n_classes, len(self.offsets), self.prec, n_sources, nx, nz)
        self.workspace = torch.empty(wsb, dtype=torch.uint8, device=device)
        nf = n_sources * nm
        self.d_rcv = torch.as_tensor(self.receivers, device=device)
        self.paths = (torch.empty((2 * nf, len(self.receivers), path_cap), dtype=torch.int64, device=device),
                      torch.empty((2 * nf, len(self.receivers)), dtype=torch.int64, device=device))
        self.d_classes = torch.empty(n_classes * 104, dtype=torch.uint8, device=device)
        self.d_cls = torch.empty(n, dtype=torch.int32, device=device)
        self.sources = np.zeros(n_sources, np.int64)
        self.d_field_src = torch.empty(2 * nf, dtype=torch.int64, device=device)
        self.launches_per_run = 6   # cache build, lookup, class check, relaxation, 2 x raypaths

    # -- inputs --------------------------------------------------------------
    def set_inputs(self, d_classes, d_cls, sources):
        """Resident device inputs: packed classes (uint8), class map (int32), sources (host)."""
        self.d_classes.copy_(d_classes)
        self.d_cls.copy_(d_cls)
        self._set_sources(sources)

    def _set_sources(self, sources):
        self.sources = np.ascontiguousarray(np.asarray(sources, np.int64))
        nm = len(self.modes)
        per_field = np.repeat(self.sources, nm)
        self.d_field_src.copy_(self.torch.as_tensor(np.concatenate([per_field, per_field])))

    # -- the path ------------------------------------------------------------
    def run(self, stream=None, events=None):
        """Cache build + traveltime (+ parents) + raypaths on resident inputs.

        events: optional list of 3 torch.cuda.Event to bracket the cache build
        and the relaxation (recorded on the current stream)."""
        if events:
            events[0].record()
        self.cache = chert.build_cache(self.d_classes, self.n_classes, self.modes, self.M, self.scan_step,
                                       self.scan_half, self.kernel, self.cprec, stream, out=self.cache_out)
        if events:
            events[1].record()
        chert.traveltime(self.cache, self.nx, self.nz, self.dx, self.d_cls, self.offsets, self.sources,
                         self.max_cycles, True, stream, out=self.tau, workspace=self.workspace)
        if events:
            events[2].record()
        nf = self.n_sources * len(self.modes)
        fsrc = self.d_field_src[:nf]
        for comp in (0, 1):          # propagation and attenuation raypaths (Eq. 33)
            chert.raypath(self.tau[2 + comp].reshape(nf, -1), fsrc, self.d_rcv, self.path_cap, stream,
                          out=(self.paths[0][comp * nf:(comp + 1) * nf],
                               self.paths[1][comp * nf:(comp + 1) * nf]))
        return self.tau

    def run_host(self, h_classes, h_cls, h_sources, h_tauR, h_tauI, stream=None):
        """End-to-end call on host buffers: H2D copies of the inputs (pinned
        host tensors), the path, D2H copies of both traveltime fields."""
        self.d_classes.copy_(h_classes, non_blocking=True)
        self.d_cls.copy_(h_cls, non_blocking=True)
        self._set_sources(h_sources)
        self.run(stream)
        h_tauR.copy_(self.tau[0], non_blocking=True)
        h_tauI.copy_(self.tau[1], non_blocking=True)
        self.torch.cuda.current_stream().synchronize()
        return h_tauR, h_tauI

    def h2d_bytes(self):
        return self.d_classes.numel() + self.d_cls.numel() * 4 + self.sources.size * 8

    def d2h_bytes(self):
        return self.tau[0].numel() * self.tau[0].element_size() * 2
