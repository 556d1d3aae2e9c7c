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

    @property
    def launches_per_run(self):
        """Kernels of one run: the cache build's main pass and, for scans
        beyond 2,048 grid points per side, its finish pass; lookup, class check,
        the row-class check (standard stencils of radius 2 to 5 on lattices of
        at most 2,048 rows), relaxation,
        2 x raypaths; the hybrid scheduler adds the block-heap continuation
        (launched always, returning at once for converged fields)."""
        from .inputs import stencil_2d
        reach = int(np.max(np.abs(self.offsets[:, [0, 2]])))
        sched = chert.relax_scheduler()
        hybrid = sched == "hybrid" and self.max_cycles > 6 and reach <= 8
        standard = len(self.offsets) == len(stencil_2d(reach))
        rows = sched != "block_heap" and standard and 2 <= reach <= 5 and max(self.nx, self.nz) <= 2048
        return (2 if self.scan_half > 2048 else 1) + 3 + int(rows) + 2 + int(hybrid)

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


class HostTracer:
    """The whole path as one library call on host buffers (chert_trace_host):
    holds the device scratch and the page-locked host outputs of one problem
    size.  ``run`` takes page-locked host inputs (packed classes uint8, class
    map int32, sources int64) and returns (tauR, tauI, paths, lengths) host
    tensors."""

    def __init__(self, n_classes, modes, M, nx, nz, dx, offsets, n_sources, receivers, kernel="MEV",
                 precision="mixed", scan_step=0.001 * math.pi / 180, scan_half=30000, max_cycles=64, path_cap=1024,
                 device="cuda", pinned=True):
        """pinned: page-locked outputs (the kernels write the results into
        them in place); False: pageable ones (copied at the end of the call)."""
        import torch
        self.n_classes, self.modes, self.M = n_classes, list(modes), M
        self.nx, self.nz, self.dx = nx, nz, dx
        self.offsets = np.ascontiguousarray(np.asarray(offsets, np.int32).reshape(-1, 3))
        self.kernel, self.precision, self.scan_step, self.scan_half = kernel, precision, scan_step, scan_half
        self.max_cycles = max_cycles
        prec = chert.PRECISION_IDS[precision]
        nm, n = len(self.modes), nx * nz
        nf = n_sources * nm
        self.h_rcv = torch.as_tensor(np.asarray(receivers, np.int64)).pin_memory()
        fd = torch.float64 if prec == chert.FP64 else torch.float32
        pin = (lambda t: t.pin_memory()) if pinned else (lambda t: t)
        self.h_tau = (pin(torch.empty((n_sources, nm, n), dtype=fd)), pin(torch.empty((n_sources, nm, n), dtype=fd)))
        self.h_paths = pin(torch.empty((2, nf, len(self.h_rcv), path_cap), dtype=torch.int64))
        self.h_lens = pin(torch.empty((2, nf, len(self.h_rcv)), dtype=torch.int64))
        nb = chert.trace_host_scratch_bytes(n_classes, nm, M, nx, nz, len(self.offsets), n_sources,
                                            len(self.h_rcv), path_cap, prec)
        self.scratch = torch.empty(nb, dtype=torch.uint8, device=device)

    def run(self, h_classes, h_cls, h_sources, stream=None):
        chert.trace_host(h_classes, self.n_classes, self.modes, self.M, self.nx, self.nz, self.dx, h_cls,
                         self.offsets, h_sources, self.h_rcv, self.h_tau[0], self.h_tau[1], self.h_paths,
                         self.h_lens, self.scratch, self.scan_step, self.scan_half, self.kernel, self.precision,
                         self.max_cycles, stream)
        return self.h_tau[0], self.h_tau[1], self.h_paths, self.h_lens

    def h2d_bytes(self, h_classes, h_cls, h_sources):
        return sum(t.numel() * t.element_size() for t in (h_classes, h_cls, h_sources, self.h_rcv))

    def d2h_bytes(self):
        return sum(t.numel() * t.element_size() for t in (*self.h_tau, self.h_paths, self.h_lens))


class Problem:
    """One traveltime problem of a batch: its classes (packed, device), cache
    geometry (2D: M; 3D: n_az, n_pol), lattice, class map (device int32),
    stencil, sources and receivers."""

    def __init__(self, d_classes, n_classes, modes, nx, nz, dx, d_cls, offsets, sources, receivers=None,
                 M=90, n_az=0, n_pol=0, ny=1, cache_precision="mixed", scan_step=0.001 * math.pi / 180,
                 scan_half=30000, kernel="MEV", max_cycles=64, path_cap=1024, surrogate_params=None,
                 relax_precision=None):
        """surrogate_params: one network parameter vector per mode (2D only):
        the cache comes from chert_cache_surrogate (networks, exact fallback
        on the device) instead of the exact build.  relax_precision: the
        relaxation's precision if not the cache's (e.g. "fp32_acc64" in 3D)."""
        self.surrogate_params = surrogate_params
        self.relax_precision = relax_precision
        self.d_classes, self.n_classes, self.modes = d_classes, n_classes, list(modes)
        self.nx, self.ny, self.nz, self.dx = nx, ny, nz, dx
        self.d_cls = d_cls
        self.offsets = np.ascontiguousarray(np.asarray(offsets, np.int32).reshape(-1, 3))
        self.sources = np.asarray(sources, np.int64).reshape(-1)
        self.receivers = None if receivers is None else np.asarray(receivers, np.int64).reshape(-1)
        self.M, self.n_az, self.n_pol = M, n_az, n_pol
        self.cache_precision, self.scan_step, self.scan_half, self.kernel = cache_precision, scan_step, scan_half, kernel
        self.max_cycles, self.path_cap = max_cycles, path_cap

    @property
    def n_fields(self):
        return len(self.sources) * len(self.modes)


class GraphBatch:
    """Many problems (sources x modes on several models, 2D and 3D) recorded
    once into one CUDA graph and replayed as one launch.  Each problem is
    captured on its own stream (forked from and joined to the capture
    stream), so the graph's branches run concurrently and fill the SMs that
    one problem's fields leave idle.  Every step is libchert's: cache build
    (exact, or the surrogate with its exact fallback), lookup + relaxation +
    parents (``chert_traveltime_enqueue``: device sources, device status, no
    host synchronisation), raypaths.

    persistent_3d: the 3D problems' relaxations run as ONE persistent launch
    (``chert_traveltime_batch``) once all their caches are built; they must
    share modes, stencil, precision and cycle cap.  persistent_2d: the same
    for the 2D problems (one persistent launch per launch shape of the
    specialised kernel, sweeps scheduler).  Problems with the same classes
    tensor and cache settings share one cache build."""

    def __init__(self, problems, device="cuda", persistent_3d=False, persistent_2d=False):
        import torch
        self.torch = torch
        self.problems = list(problems)
        self.persistent_3d = persistent_3d
        self.cache_owner = []                # index of the problem whose cache each problem reads
        keys = {}
        for i, p in enumerate(self.problems):
            k = (id(p.d_classes), p.n_classes, tuple(p.modes), p.M, p.n_az, p.n_pol, p.cache_precision,
                 p.scan_step, p.scan_half, p.kernel, id(p.surrogate_params))
            self.cache_owner.append(keys.setdefault(k, i))
        self.state = [self._allocate(p, device, self.cache_owner[i] == i) for i, p in enumerate(self.problems)]
        # batched groups: the 3D problems and the 2D problems, each relaxed by
        # one chert_traveltime_batch call on a stream and counter of its own
        self.groups = []
        for want, dims in ((persistent_3d, lambda p: p.ny > 1), (persistent_2d, lambda p: p.ny == 1)):
            members = [i for i, p in enumerate(self.problems) if dims(p)]
            if not want or not members:
                continue
            q = [self.problems[i] for i in members]
            same = all(p.modes == q[0].modes and np.array_equal(p.offsets, q[0].offsets) and
                       p.cache_precision == q[0].cache_precision and p.relax_precision == q[0].relax_precision and
                       p.max_cycles == q[0].max_cycles for p in q)
            if not same:
                raise ValueError("a persistent group's problems must share modes, stencil, precision and cycle cap")
            self.groups.append({"members": members, "counter": torch.zeros(1, dtype=torch.int64, device=device),
                                "stream": torch.cuda.Stream(device=device)})
        self.batched = {i for g in self.groups for i in g["members"]}
        self.graph = None

    def _allocate(self, p, device, owns_cache):
        torch = self.torch
        prec = chert.PRECISION_IDS[p.cache_precision]
        rprec = prec if p.relax_precision is None else chert.PRECISION_IDS[p.relax_precision]
        fd = torch.float64 if prec == chert.FP64 else torch.float32
        td = torch.float64 if rprec in (chert.FP64, chert.FP32_ACC64) else torch.float32
        nd = p.n_az * p.n_pol if p.n_az else 4 * p.M
        shape = (len(p.modes), p.n_classes, nd)
        keys = ("V", "A", "Q", "rx", "rz", "theta", "vartheta") + (("ry", "phi") if p.n_az else ())
        cache_out = None
        if owns_cache:
            cache_out = {k: torch.empty(shape, dtype=fd, device=device) for k in keys}
            cache_out["flag"] = torch.empty(shape, dtype=torch.uint8, device=device)
        n = p.nx * p.ny * p.nz
        fshape = (len(p.sources), len(p.modes), n)
        tau = (torch.empty(fshape, dtype=td, device=device), torch.empty(fshape, dtype=td, device=device),
               torch.empty(fshape, dtype=torch.int32, device=device),
               torch.empty(fshape, dtype=torch.int32, device=device))
        if p.ny == 1:
            wsb = chert.workspace_bytes(len(p.modes), p.n_classes, len(p.offsets), rprec, len(p.sources), p.nx, p.nz)
        else:
            wsb = chert.workspace_bytes(len(p.modes), p.n_classes, len(p.offsets), rprec, len(p.sources))
        st = {"cache_out": cache_out, "tau": tau,
              "ws": torch.empty(wsb, dtype=torch.uint8, device=device),
              "d_src": torch.as_tensor(p.sources, device=device),
              "status": torch.zeros(2, dtype=torch.int32, device=device),
              "stream": torch.cuda.Stream(device=device)}
        if p.receivers is not None:
            nf = p.n_fields
            st["d_fsrc"] = torch.as_tensor(np.repeat(p.sources, len(p.modes)), device=device)
            st["d_rcv"] = torch.as_tensor(p.receivers, device=device)
            st["paths"] = (torch.empty((2, nf, len(p.receivers), p.path_cap), dtype=torch.int64, device=device),
                           torch.empty((2, nf, len(p.receivers)), dtype=torch.int64, device=device))
        return st

    def _build_cache(self, p, st, stream):
        if p.surrogate_params is not None:
            if p.n_az:
                raise ValueError("the surrogate cache is 2D")
            cache = chert.cache_surrogate(p.surrogate_params, p.d_classes, p.n_classes, p.modes, p.M, p.scan_step,
                                          p.scan_half, p.kernel, p.cache_precision, stream, out=st["cache_out"])
        elif p.n_az:
            cache = chert.build_cache_3d(p.d_classes, p.n_classes, p.modes, p.n_az, p.n_pol, p.scan_step,
                                         p.scan_half, p.kernel, p.cache_precision, stream, out=st["cache_out"])
        else:
            cache = chert.build_cache(p.d_classes, p.n_classes, p.modes, p.M, p.scan_step, p.scan_half,
                                      p.kernel, p.cache_precision, stream, out=st["cache_out"])
        st["cache"] = cache

    def _raypaths(self, p, st, stream):
        if p.receivers is not None:
            nf = p.n_fields
            for comp in (0, 1):
                chert.raypath(st["tau"][2 + comp].reshape(nf, -1), st["d_fsrc"], st["d_rcv"], p.path_cap, stream,
                              out=(st["paths"][0][comp], st["paths"][1][comp]))

    def _relax(self, i, stream):
        p, st = self.problems[i], self.state[i]
        cache = self.state[self.cache_owner[i]]["cache"]
        prec = None if p.relax_precision is None else chert.PRECISION_IDS[p.relax_precision]
        chert.traveltime_enqueue(cache, p.nx, p.nz, p.dx, p.d_cls, p.offsets, st["d_src"], st["tau"], st["ws"],
                                 st["status"], p.max_cycles, p.ny, stream, precision=prec)
        self._raypaths(p, st, stream)

    def _relax_group(self, g, stream):
        items = []
        for i in g["members"]:
            p, st = self.problems[i], self.state[i]
            items.append({"cache": self.state[self.cache_owner[i]]["cache"], "nx": p.nx, "ny": p.ny, "nz": p.nz,
                          "dx": p.dx, "d_cls": p.d_cls, "d_sources": st["d_src"], "out": st["tau"],
                          "workspace": st["ws"], "d_status": st["status"]})
        p0 = self.problems[g["members"][0]]
        chert.traveltime_batch(items, p0.offsets, g["counter"], p0.max_cycles, stream,
                               precision=p0.relax_precision)
        for i in g["members"]:
            self._raypaths(self.problems[i], self.state[i], stream)

    def run_eager(self):
        """One pass without the graph (also loads every kernel before capture)."""
        for i, (p, st) in enumerate(zip(self.problems, self.state)):
            if self.cache_owner[i] == i:
                self._build_cache(p, st, None)
        for i in range(len(self.problems)):
            if i not in self.batched:
                self._relax(i, None)
        for g in self.groups:
            self._relax_group(g, None)

    def _timed(self, fn, repeats):
        torch = self.torch
        best = float("inf")
        for _ in range(repeats):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        return best

    def autotune(self, repeats=1):
        """Launch shapes for this batch, chosen by timing its relaxations on
        the caches of one eager pass (run it first): the 3D tile shape
        (chert_set_relax3d_tile: 32 x 16 or 64 x 8) on the 3D problems, and
        the points per thread of the 2D kernel (1, 2 or 4) on the 2D ones.
        The fastest of each is kept for the process, so a later capture
        records it; results do not depend on either.  Returns
        {"tile3d": {tile: ms}, "ppt2d": {ppt: ms}, "chosen": {...}}."""
        out = {"tile3d": {}, "ppt2d": {}, "chosen": {}}
        three = [i for i, p in enumerate(self.problems) if p.ny > 1]
        two = [i for i, p in enumerate(self.problems) if p.ny == 1]
        g3 = [g for g in self.groups if self.problems[g["members"][0]].ny > 1]
        g2 = [g for g in self.groups if self.problems[g["members"][0]].ny == 1]
        if three:
            run3 = (lambda: self._relax_group(g3[0], None)) if g3 else \
                (lambda: [self._relax(i, None) for i in three])
            for tile in (0, 1):
                chert.set_relax3d_tile(tile)
                out["tile3d"][tile] = self._timed(run3, repeats)
            best = _pick(out["tile3d"])
            chert.set_relax3d_tile(best)
            out["chosen"]["tile3d"] = best
        if two:
            line = max(max(self.problems[i].nx, self.problems[i].nz) for i in two)
            for ppt in (1, 2, 4):
                if (line + ppt - 1) // ppt > 512:
                    continue
                chert.lib().chert_set_relax_points_per_thread(ppt)
                run2 = (lambda: self._relax_group(g2[0], None)) if g2 else \
                    (lambda: [self._relax(i, None) for i in two])
                out["ppt2d"][ppt] = self._timed(run2, repeats)
            best = _pick(out["ppt2d"])
            chert.lib().chert_set_relax_points_per_thread(best)
            out["chosen"]["ppt2d"] = best
        return out

    def capture(self, warm=True):
        """Record the batch into one CUDA graph (warm: one eager pass first, to
        load every kernel; skip it when a pass has already run)."""
        torch = self.torch
        if warm:
            self.run_eager()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            main = torch.cuda.current_stream()
            # caches, each on its problem's stream
            for i, (p, st) in enumerate(zip(self.problems, self.state)):
                st["stream"].wait_stream(main)
                if self.cache_owner[i] == i:
                    with torch.cuda.stream(st["stream"]):
                        self._build_cache(p, st, st["stream"])
            # relaxations: each problem after its cache's build; a batched
            # group after every one of its problems' caches
            for i, st in enumerate(self.state):
                if i in self.batched:
                    continue
                s = st["stream"]
                s.wait_stream(self.state[self.cache_owner[i]]["stream"])
                with torch.cuda.stream(s):
                    self._relax(i, s)
            for grp in self.groups:
                sg = grp["stream"]
                sg.wait_stream(main)
                for i in grp["members"]:
                    sg.wait_stream(self.state[self.cache_owner[i]]["stream"])
                with torch.cuda.stream(sg):
                    self._relax_group(grp, sg)
                main.wait_stream(sg)
            for st in self.state:
                main.wait_stream(st["stream"])
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def check(self):
        """Host read of every problem's status (one synchronisation); raises
        like chert_traveltime on a cycle cap or a bad class map."""
        for p, st in zip(self.problems, self.state):
            first, bad = (int(v) for v in st["status"].cpu().tolist())
            if bad:
                raise chert.ChertError(chert.EINVAL, "class map holds ids outside [0, %d)" % p.n_classes)
            if first >= 0:
                raise chert.ChertError(chert.ETIMEOUT, "field %d component %d did not converge in %d cycles"
                                       % (first // 2, first % 2, p.max_cycles))

    def fields(self, i):
        return self.state[i]["tau"]

    @property
    def n_fields(self):
        return sum(p.n_fields for p in self.problems)


def per_node_classes(classes, class_of_node):
    """Packed chert_class records of every node's medium (host uint8 [n*104]):
    the input of the no-cache form, where each node carries its own medium."""
    import ctypes
    arr = (chert.chert_class * len(classes))(*classes)
    raw = np.frombuffer(bytes(arr), dtype=np.uint8).reshape(len(classes), ctypes.sizeof(chert.chert_class))
    return np.ascontiguousarray(raw[np.asarray(class_of_node).reshape(-1)]).reshape(-1)


def no_cache_traveltime(d_node_classes, nx, nz, dx, offsets, sources, modes, M, scan_step=0.001 * math.pi / 180,
                        scan_half=30000, kernel="MEV", precision="mixed", max_cycles=64, stream=None):
    """The no-cache (MSPM-style) form of the paper's Algorithm 1 with this
    library's kernels: for every (source, mode) field, every node's own
    directional table is solved afresh from its medium (chert_build_cache with
    one class per node; nothing shared between nodes or fields), then looked
    up and relaxed (chert_traveltime, class map = node index).  Where nodes
    share a medium the tables equal the class cache's entries, so the fields
    and parents equal those of the cached path bit for bit; only the cost
    differs.  d_node_classes: device uint8 [n*104] (per_node_classes).
    Returns (tauR, tauI, parR, parI) tensors [n_sources, n_modes, nz*nx]."""
    import torch
    n = nx * nz
    dev = d_node_classes.device
    own = torch.arange(n, dtype=torch.int32, device=dev)
    prec = chert.PRECISION_IDS[precision]
    fd = torch.float64 if prec == chert.FP64 else torch.float32
    src = np.asarray(sources, np.int64).reshape(-1)
    out = (torch.empty((len(src), len(modes), n), dtype=fd, device=dev),
           torch.empty((len(src), len(modes), n), dtype=fd, device=dev),
           torch.empty((len(src), len(modes), n), dtype=torch.int32, device=dev),
           torch.empty((len(src), len(modes), n), dtype=torch.int32, device=dev))
    ws = torch.empty(chert.workspace_bytes(1, n, len(np.asarray(offsets).reshape(-1, 3)), prec, 1, nx, nz),
                     dtype=torch.uint8, device=dev)
    for si, s in enumerate(src):
        for mi, mode in enumerate(modes):
            tables = chert.build_cache(d_node_classes, n, [mode], M, scan_step, scan_half, kernel, precision, stream)
            f = chert.traveltime(tables, nx, nz, dx, own, offsets, [int(s)], max_cycles, True, stream, workspace=ws)
            for k in range(4):
                out[k][si, mi].copy_(f[k][0, 0])
            del tables, f
    return out


def autotune_points_per_thread(tracer, candidates=(1, 2, 4), repeats=3):
    """Time the relaxation of ``tracer``'s problem (its full run) with each
    launch shape of the specialised 2D kernel and keep the fastest for the
    process (chert_set_relax_points_per_thread); a shape other than the
    smallest must win by more than 3%.  The results are identical for every
    shape; only the time differs.  Returns (best, {ppt: ms})."""
    import torch
    line = max(tracer.nx, tracer.nz)
    times = {}
    for ppt in candidates:
        if (line + ppt - 1) // ppt > 512:
            continue
        chert.lib().chert_set_relax_points_per_thread(ppt)
        tracer.run()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        best = float("inf")
        for _ in range(repeats):
            tracer.run(events=ev)
            torch.cuda.synchronize()
            best = min(best, ev[1].elapsed_time(ev[2]))
        times[ppt] = best
    choice = _pick(times)
    chert.lib().chert_set_relax_points_per_thread(choice)
    return choice, times


def _pick(times, margin=0.03):
    """The fastest shape, but the first candidate (the smallest) unless another
    is faster by more than `margin`: timing noise does not flip a tie."""
    first = min(times)
    best = min(times, key=times.get)
    return best if times[best] < (1 - margin) * times[first] else first
