"""Python binding of libchert.so (argument marshalling only).

Every step of the hot path runs in the library's CUDA kernels; this module only
turns torch tensors into pointers and sizes and checks status codes.  Device
memory comes from torch (caller-owned buffers and the relaxation workspace);
the library itself allocates no device memory.  There is no CPU fallback: if
the library is missing or a tensor is not on a CUDA device, calls raise.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libchert.so")

QP, QSV, QSH = 0, 1, 2
MODE_IDS = {"qP": QP, "qSV": QSV, "qSH": QSH}
OEV, MEV = 0, 1
KERNEL_IDS = {"OEV": OEV, "MEV": MEV}
FP64, FP32, MIXED, FP32_ACC64 = 0, 1, 2, 3
PRECISION_IDS = {"fp64": FP64, "fp32": FP32, "mixed": MIXED, "fp32_acc64": FP32_ACC64}

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT = 0, -1, -2, -3, -4


class ChertError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libchert error %d: %s" % (code, msg))
        self.code = code


class chert_class(ctypes.Structure):
    _fields_ = [("aR", ctypes.c_double * 5), ("aI", ctypes.c_double * 5), ("rho", ctypes.c_double),
                ("tilt", ctypes.c_double), ("azim", ctypes.c_double)]


class chert_cache_arrays(ctypes.Structure):
    _fields_ = [("V", ctypes.c_void_p), ("A", ctypes.c_void_p), ("Q", ctypes.c_void_p),
                ("rx", ctypes.c_void_p), ("rz", ctypes.c_void_p), ("theta", ctypes.c_void_p),
                ("vartheta", ctypes.c_void_p), ("flag", ctypes.c_void_p), ("ry", ctypes.c_void_p),
                ("phi", ctypes.c_void_p)]


class chert_lattice(ctypes.Structure):
    _fields_ = [("cache", ctypes.c_void_p), ("n_classes", ctypes.c_int), ("n_dir", ctypes.c_int),
                ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("dx", ctypes.c_double),
                ("d_class_of_node", ctypes.c_void_p), ("d_sources", ctypes.c_void_p), ("n_sources", ctypes.c_int),
                ("d_tauR", ctypes.c_void_p), ("d_tauI", ctypes.c_void_p), ("d_parR", ctypes.c_void_p),
                ("d_parI", ctypes.c_void_p), ("d_workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t),
                ("d_status", ctypes.c_void_p)]


class chert_cache_params(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("scan_step", ctypes.c_double), ("scan_half", ctypes.c_int),
                ("kernel", ctypes.c_int), ("precision", ctypes.c_int)]


_lib = None


def lib():
    """Load libchert.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libchert.so not built: run python -m paper_2609_26108_b300.build")
    L = ctypes.CDLL(LIB_PATH)
    P, I, D, I64, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_size_t
    L.chert_last_error.restype = ctypes.c_char_p
    L.chert_thomsen_to_class.argtypes = [D] * 10 + [ctypes.POINTER(chert_class)]
    L.chert_moduli_to_class.argtypes = [P, P, D, D, D, ctypes.POINTER(chert_class)]
    L.chert_moduli_to_class.restype = ctypes.c_int
    L.chert_thomsen_to_classes.argtypes = [I64] + [P] * 11
    L.chert_thomsen_to_classes.restype = ctypes.c_int
    L.chert_build_cache.argtypes = [P, I, P, I, ctypes.POINTER(chert_cache_params),
                                    ctypes.POINTER(chert_cache_arrays), P]
    L.chert_edge_table.argtypes = [ctypes.POINTER(chert_cache_arrays), I, I, I, I, P, I, P, P, P, P]
    L.chert_build_cache_items.argtypes = [P, I, P, I, ctypes.POINTER(chert_cache_params), P, I64,
                                          ctypes.POINTER(chert_cache_arrays), P]
    L.chert_build_cache_items.restype = ctypes.c_int
    L.chert_build_cache_3d.argtypes = [P, I, P, I, I, I, ctypes.POINTER(chert_cache_params),
                                       ctypes.POINTER(chert_cache_arrays), P]
    L.chert_build_cache_3d.restype = ctypes.c_int
    L.chert_traveltime_workspace_bytes.argtypes = [I, I, I, I, I]
    L.chert_traveltime_workspace_bytes.restype = SZ
    L.chert_traveltime_workspace_bytes_grid.argtypes = [I, I, I, I, I, I, I, I]
    L.chert_traveltime_workspace_bytes_grid.restype = SZ
    L.chert_traveltime.argtypes = [ctypes.POINTER(chert_cache_arrays), I, I, I, I, I, I, D, P, P, I,
                                   P, I, I, I, P, P, P, P, P, SZ, P]
    L.chert_raypath.argtypes = [P, I, I64, P, P, I, I64, P, P, P]
    L.chert_parent_ties.argtypes = [P, P, I, I, I, I, I, I, D, P, P, I, P, I, P, P, D, P, P, P, P]
    L.chert_parent_ties.restype = ctypes.c_int
    L.chert_trace_host_scratch_bytes.argtypes = [I, I, I, I, I, I, I, I, I64, I]
    L.chert_trace_host_scratch_bytes.restype = SZ
    L.chert_trace_host.argtypes = [P, I, P, I, ctypes.POINTER(chert_cache_params), I, I, D, P, P, I, P, I, I, P, I,
                                   I64, P, P, P, P, P, SZ, P]
    L.chert_trace_host.restype = ctypes.c_int
    L.chert_set_surrogate_qsv_angle.argtypes = [D]
    L.chert_set_surrogate_qsv_angle.restype = D
    L.chert_fma_rate.argtypes = [I, I, ctypes.POINTER(ctypes.c_double), P]
    L.chert_fma_rate.restype = ctypes.c_int
    L.chert_cache_eval_counter.argtypes = [I, P]
    L.chert_cache_eval_counter.restype = ctypes.c_int
    L.chert_traveltime_enqueue.argtypes = [ctypes.POINTER(chert_cache_arrays), I, I, I, I, I, I, D, P, P, I,
                                           P, I, I, I, P, P, P, P, P, SZ, P, P]
    L.chert_traveltime_enqueue.restype = ctypes.c_int
    L.chert_traveltime_batch.argtypes = [P, I, I, I, P, I, I, P, P]
    L.chert_traveltime_batch.restype = ctypes.c_int
    L.chert_set_cache_finish_threads.argtypes = [I]
    L.chert_set_cache_finish_threads.restype = ctypes.c_int
    L.chert_set_relax3d_tile.argtypes = [I]
    L.chert_set_relax3d_tile.restype = ctypes.c_int
    L.chert_set_relax_points_per_thread.argtypes = [I]
    L.chert_set_relax_points_per_thread.restype = ctypes.c_int
    L.chert_set_relax_scheduler.argtypes = [I]
    L.chert_set_relax_scheduler.restype = ctypes.c_int
    L.chert_traveltime_static.argtypes = [ctypes.POINTER(chert_cache_arrays), I, I, I, I, I, I, D, P, P,
                                          I, P, I, I, I, P, P, P, P, P]
    L.chert_traveltime_static_limit.restype = SZ
    L.chert_traveltime_static_limit.argtypes = []
    L.chert_mlp_param_count.restype = SZ
    L.chert_mlp_param_count.argtypes = []
    L.chert_mlp_workspace_bytes.restype = SZ
    L.chert_mlp_workspace_bytes.argtypes = [I64, I]
    L.chert_mlp_forward.argtypes = [P, P, I64, P, P, SZ, P]
    L.chert_mlp_set_tensor_cores.argtypes = [I]
    L.chert_mlp_set_tensor_cores.restype = I
    L.chert_mlp_train_step.argtypes = [P, P, P, I, ctypes.c_float, P, P, I64, P, P, P, SZ, P]
    L.chert_surrogate_dataset.argtypes = [P, I, I, I, I, ctypes.POINTER(chert_cache_arrays), I, P, P,
                                          P, SZ, P]
    L.chert_surrogate_cache_workspace_bytes.restype = SZ
    L.chert_surrogate_cache_workspace_bytes.argtypes = [I, I]
    L.chert_surrogate_cache.argtypes = [P, P, I, P, I, I, I, ctypes.POINTER(chert_cache_arrays), P, SZ, P]
    L.chert_angular_coverage.argtypes = [ctypes.POINTER(chert_cache_arrays), I, I, I, I, P, I, P, P, P, P, P]
    L.chert_angular_coverage.restype = ctypes.c_int
    L.chert_mlp_check.argtypes = [P]
    L.chert_mlp_check.restype = ctypes.c_int
    L.chert_mlp_set_wait_limit.argtypes = [ctypes.c_longlong]
    L.chert_mlp_set_wait_limit.restype = ctypes.c_longlong
    L.chert_cache_surrogate_workspace_bytes.restype = SZ
    L.chert_cache_surrogate_workspace_bytes.argtypes = [I, I, I]
    L.chert_cache_surrogate.argtypes = [P, P, I, P, I, ctypes.POINTER(chert_cache_params),
                                        ctypes.POINTER(chert_cache_arrays), P, SZ, P, P]
    L.chert_cache_surrogate.restype = ctypes.c_int
    for name in ("chert_thomsen_to_class", "chert_build_cache", "chert_edge_table",
                 "chert_traveltime", "chert_raypath", "chert_traveltime_static", "chert_mlp_forward",
                 "chert_mlp_train_step", "chert_surrogate_dataset", "chert_surrogate_cache"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc):
    if rc != OK:
        raise ChertError(rc, lib().chert_last_error().decode())


def _torch():
    import torch
    return torch


def _dev_ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensor must be on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _fdtype(precision):
    torch = _torch()
    return torch.float64 if precision in (FP64, FP32_ACC64) else torch.float32


# ------------------------------------------------------------------ classes
def thomsen_to_class(vp0, vs0, eps, delta, gamma, qp, qs, rho=2200.0, tilt=0.0, azim=0.0):
    out = chert_class()
    _check(lib().chert_thomsen_to_class(vp0, vs0, eps, delta, gamma, qp, qs, rho, tilt, azim,
                                        ctypes.byref(out)))
    return out


def table_class(aR, q, rho=2200.0, tilt=0.0, azim=0.0):
    """A class from real moduli and per-component Q (Eq. 2: aI = aR/Q)."""
    c = chert_class()
    a = (ctypes.c_double * 5)(*[float(v) for v in aR])
    qq = (ctypes.c_double * 5)(*[float(v) for v in q])
    _check(lib().chert_moduli_to_class(a, qq, float(rho), float(tilt), float(azim), ctypes.byref(c)))
    return c


def classes_from_layers(layers):
    """chert_class records for ThomsenLayer / TableLayer descriptions."""
    out = []
    for L in layers:
        if hasattr(L, "vp0"):
            out.append(thomsen_to_class(L.vp0, L.vs0, L.eps, L.delta, L.gamma, L.qp, L.qs,
                                        L.rho, L.tilt, L.azim))
        else:
            out.append(table_class(L.aR, L.q, L.rho, L.tilt, L.azim))
    return out


def classes_from_arrays(vp0, vs0, eps, delta, gamma, qp, qs, rho=None, tilt=None, azim=None):
    """Packed chert_class records (numpy uint8 [n*104]) for per-cell arrays."""
    n = len(vp0)
    f = lambda a, default: np.ascontiguousarray(np.full(n, default) if a is None else a, dtype=np.float64)
    cols = [f(vp0, 0), f(vs0, 0), f(eps, 0), f(delta, 0), f(gamma, 0), f(qp, 0), f(qs, 0), f(rho, 2200.0),
            f(tilt, 0.0), f(azim, 0.0)]
    out = np.zeros(n * ctypes.sizeof(chert_class), dtype=np.uint8)
    _check(lib().chert_thomsen_to_classes(n, *[c.ctypes.data_as(ctypes.c_void_p) for c in cols],
                                          out.ctypes.data_as(ctypes.c_void_p)))
    return out


def classes_to_device(classes, device="cuda"):
    """Pack chert_class records into a device byte tensor (the ABI's array)."""
    torch = _torch()
    if isinstance(classes, np.ndarray):
        return torch.from_numpy(classes).to(device)
    arr = (chert_class * len(classes))(*classes)
    raw = np.frombuffer(bytes(arr), dtype=np.uint8).copy()
    return torch.from_numpy(raw).to(device)


# ------------------------------------------------------------------ cache
class Cache:
    """Device-resident directional cache (torch tensors [n_modes, n_classes,
    n_dir]): 2D with n_dir = 4M slowness angles, or 3D (n_az, n_pol set) with
    n_dir = n_az*n_pol global directions."""

    def __init__(self, arrays, modes, n_classes, M, precision, n_az=0, n_pol=0):
        self.arrays, self.modes, self.n_classes, self.M, self.precision = arrays, modes, n_classes, M, precision
        self.n_az, self.n_pol = n_az, n_pol

    n_fallback_dev = None     # set by cache_surrogate: device int64 [1]

    @property
    def n_fallback(self):
        """Solves that a surrogate cache recomputed exactly (0 for an exact
        cache); reading it copies one integer from the device."""
        return 0 if self.n_fallback_dev is None else int(self.n_fallback_dev.item())

    @property
    def n_dir(self):
        return self.n_az * self.n_pol if self.n_az else 4 * self.M

    def struct(self):
        a = self.arrays
        return chert_cache_arrays(*[None if a.get(k) is None else a[k].data_ptr()
                                    for k in ("V", "A", "Q", "rx", "rz", "theta", "vartheta", "flag", "ry",
                                              "phi")])

    def __getitem__(self, key):
        return self.arrays[key]


def build_cache(d_classes, n_classes, modes, M, scan_step=0.001 * math.pi / 180, scan_half=30000,
                kernel="MEV", precision="fp32", stream=None, out=None):
    """Enqueue chert_build_cache; returns a Cache of new (or given) torch tensors."""
    torch = _torch()
    prec = PRECISION_IDS[precision] if isinstance(precision, str) else precision
    mode_ids = [MODE_IDS[m] if isinstance(m, str) else m for m in modes]
    shape = (len(mode_ids), n_classes, 4 * M)
    dev = d_classes.device
    if out is None:
        fd = _fdtype(prec)
        out = {k: torch.empty(shape, dtype=fd, device=dev)
               for k in ("V", "A", "Q", "rx", "rz", "theta", "vartheta")}
        out["flag"] = torch.empty(shape, dtype=torch.uint8, device=dev)
    cache = Cache(out, mode_ids, n_classes, M, prec)
    params = chert_cache_params(M, scan_step, scan_half, KERNEL_IDS.get(kernel, kernel), prec)
    modes_arr = (ctypes.c_int * len(mode_ids))(*mode_ids)
    st = cache.struct()
    _check(lib().chert_build_cache(_dev_ptr(d_classes), n_classes, modes_arr, len(mode_ids),
                                   ctypes.byref(params), ctypes.byref(st), _stream_ptr(stream)))
    return cache


def build_cache_3d(d_classes, n_classes, modes, n_az, n_pol, scan_step=0.001 * math.pi / 180, scan_half=30000,
                   kernel="MEV", precision="fp32", stream=None, out=None):
    """Enqueue chert_build_cache_3d (global direction grid n_pol x n_az)."""
    torch = _torch()
    prec = PRECISION_IDS[precision] if isinstance(precision, str) else precision
    mode_ids = [MODE_IDS[m] if isinstance(m, str) else m for m in modes]
    shape = (len(mode_ids), n_classes, n_az * n_pol)
    dev = d_classes.device
    if out is None:
        fd = _fdtype(prec)
        out = {k: torch.empty(shape, dtype=fd, device=dev)
               for k in ("V", "A", "Q", "rx", "ry", "rz", "theta", "phi", "vartheta")}
        out["flag"] = torch.empty(shape, dtype=torch.uint8, device=dev)
    cache = Cache(out, mode_ids, n_classes, 0, prec, n_az, n_pol)
    params = chert_cache_params(1, scan_step, scan_half, KERNEL_IDS.get(kernel, kernel), prec)
    modes_arr = (ctypes.c_int * len(mode_ids))(*mode_ids)
    st = cache.struct()
    _check(lib().chert_build_cache_3d(_dev_ptr(d_classes), n_classes, modes_arr, len(mode_ids), n_az, n_pol,
                                      ctypes.byref(params), ctypes.byref(st), _stream_ptr(stream)))
    return cache


def build_cache_items(cache, d_classes, items, scan_step=0.001 * math.pi / 180, scan_half=30000, kernel="MEV",
                      precision=None, stream=None):
    """Exactly solve the listed solves (device int64 tensor) into `cache`."""
    prec = cache.precision if precision is None else (PRECISION_IDS[precision] if isinstance(precision, str)
                                                      else precision)
    params = chert_cache_params(cache.M, scan_step, scan_half, KERNEL_IDS.get(kernel, kernel), prec)
    modes_arr = (ctypes.c_int * len(cache.modes))(*cache.modes)
    st = cache.struct()
    _check(lib().chert_build_cache_items(_dev_ptr(d_classes), cache.n_classes, modes_arr, len(cache.modes),
                                         ctypes.byref(params), _dev_ptr(items), int(items.numel()),
                                         ctypes.byref(st), _stream_ptr(stream)))
    return cache


def _offsets_arr(offsets):
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32).reshape(-1, 3))
    return off, off.ctypes.data_as(ctypes.c_void_p)


def edge_table(cache, offsets, stream=None):
    """Enqueue chert_edge_table: (idx, Vsel, Asel) torch tensors [n_modes, n_classes, n_off]."""
    torch = _torch()
    off, off_p = _offsets_arr(offsets)
    nm = len(cache.modes)
    dev = cache["V"].device
    idx = torch.empty((nm, cache.n_classes, len(off)), dtype=torch.int32, device=dev)
    Vs = torch.empty(idx.shape, dtype=_fdtype(cache.precision), device=dev)
    As = torch.empty_like(Vs)
    st = cache.struct()
    _check(lib().chert_edge_table(ctypes.byref(st), nm, cache.n_classes, cache.n_dir, cache.precision,
                                  off_p, len(off), _dev_ptr(idx), _dev_ptr(Vs), _dev_ptr(As),
                                  _stream_ptr(stream)))
    return idx, Vs, As


def workspace_bytes(n_modes, n_classes, n_off, precision, n_sources, nx=None, nz=None):
    """Relaxation scratch; with the lattice size it includes the per-node
    weight area that the specialised kernel uses for many classes."""
    if nx is None:
        return int(lib().chert_traveltime_workspace_bytes(n_modes, n_classes, n_off, precision, n_sources))
    return int(lib().chert_traveltime_workspace_bytes_grid(n_modes, n_classes, n_off, precision, n_sources,
                                                           nx, 1, nz))


def traveltime(cache, nx, nz, dx, d_cls, offsets, sources, max_cycles=64, parents=True,
               stream=None, out=None, workspace=None, ny=1, precision=None):
    """chert_traveltime for all (source, mode) fields of ``cache`` on an
    nx x ny x nz lattice (ny = 1: 2D).  precision: the cache's by default;
    "fp32_acc64" (3D, float cache) accumulates the traveltimes in float-float
    and returns them as double.

    Returns (tauR, tauI, parR, parI) torch tensors [n_sources, n_modes, nz*ny*nx]."""
    torch = _torch()
    off, off_p = _offsets_arr(offsets)
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.int64).reshape(-1))
    nm, ns = len(cache.modes), len(src)
    prec = cache.precision if precision is None else (PRECISION_IDS[precision] if isinstance(precision, str)
                                                      else precision)
    dev = cache["V"].device
    shape = (ns, nm, nx * ny * nz)
    if out is None:
        fd = _fdtype(prec)
        out = (torch.empty(shape, dtype=fd, device=dev), torch.empty(shape, dtype=fd, device=dev),
               torch.empty(shape, dtype=torch.int32, device=dev) if parents else None,
               torch.empty(shape, dtype=torch.int32, device=dev) if parents else None)
    if workspace is None:
        wsb = (workspace_bytes(nm, cache.n_classes, len(off), prec, ns, nx, nz) if ny == 1
               else workspace_bytes(nm, cache.n_classes, len(off), prec, ns))
        workspace = torch.empty(wsb, dtype=torch.uint8, device=dev)
    st = cache.struct()
    _check(lib().chert_traveltime(ctypes.byref(st), nm, cache.n_classes, cache.n_dir, nx, ny, nz,
                                  float(dx), _dev_ptr(d_cls), off_p, len(off),
                                  src.ctypes.data_as(ctypes.c_void_p), ns, prec,
                                  max_cycles, _dev_ptr(out[0]), _dev_ptr(out[1]), _dev_ptr(out[2]),
                                  _dev_ptr(out[3]), _dev_ptr(workspace), workspace.numel(),
                                  _stream_ptr(stream)))
    return out


def traveltime_enqueue(cache, nx, nz, dx, d_cls, offsets, d_sources, out, workspace, d_status, max_cycles=64,
                       ny=1, stream=None, precision=None):
    """chert_traveltime_enqueue: no host synchronisation or copy (capturable
    in a CUDA graph).  d_sources: device int64 [n_sources]; out: (tauR, tauI,
    parR, parI) preallocated; d_status: device int32[2] (first field*2+comp that
    hit the cycle cap or -1, class-map error flag)."""
    off, off_p = _offsets_arr(offsets)
    nm, ns = len(cache.modes), int(d_sources.numel())
    st = cache.struct()
    _check(lib().chert_traveltime_enqueue(ctypes.byref(st), nm, cache.n_classes, cache.n_dir, nx, ny, nz,
                                          float(dx), _dev_ptr(d_cls), off_p, len(off), _dev_ptr(d_sources), ns,
                                          cache.precision if precision is None else precision, max_cycles,
                                          _dev_ptr(out[0]), _dev_ptr(out[1]), _dev_ptr(out[2]), _dev_ptr(out[3]),
                                          _dev_ptr(workspace),
                                          workspace.numel(), _dev_ptr(d_status), _stream_ptr(stream)))
    return out


def traveltime_batch(items, offsets, d_counter, max_cycles=64, stream=None, precision=None):
    """chert_traveltime_batch: several 3D lattices in one persistent launch.
    items: list of dicts with cache (Cache), nx, ny, nz, dx, d_cls, d_sources,
    out (tauR, tauI, parR, parI), workspace and d_status (as for
    traveltime_enqueue); all caches share modes and precision (precision:
    the caches' by default, or "fp32_acc64").  d_counter: device int64 [1]
    (the work counter)."""
    off, off_p = _offsets_arr(offsets)
    keep = []
    arr = (chert_lattice * len(items))()
    for i, it in enumerate(items):
        c = it["cache"]
        st = c.struct()
        keep.append(st)
        o = it["out"]
        arr[i] = chert_lattice(ctypes.addressof(st), c.n_classes, c.n_dir, it["nx"], it["ny"], it["nz"],
                               float(it["dx"]), it["d_cls"].data_ptr(), it["d_sources"].data_ptr(),
                               int(it["d_sources"].numel()), o[0].data_ptr(), o[1].data_ptr(), o[2].data_ptr(),
                               o[3].data_ptr(), it["workspace"].data_ptr(), it["workspace"].numel(),
                               it["d_status"].data_ptr())
    c0 = items[0]["cache"]
    prec = c0.precision if precision is None else (PRECISION_IDS[precision] if isinstance(precision, str)
                                                   else precision)
    _check(lib().chert_traveltime_batch(arr, len(items), len(c0.modes), prec, off_p, len(off), max_cycles,
                                        _dev_ptr(d_counter), _stream_ptr(stream)))


def set_relax3d_tile(tile):
    """3D tile shape of every later 3D relaxation: 0 (32 x 16, default) or 1
    (64 x 8); returns the previous one."""
    rc = int(lib().chert_set_relax3d_tile(int(tile)))
    if rc < 0:
        _check(rc)
    return rc


def traveltime_static(cache, nx, nz, dx, d_cls, offsets, sources, max_cycles=64, parents=True,
                      stream=None, out=None):
    """chert_traveltime_static: the relaxation without any device allocation by
    the library (its scratch is a fixed array inside libchert).  Same results
    and output layout as ``traveltime``; it synchronises the stream (no stream
    capture), and calls that overlap on the GPU race on the shared array."""
    torch = _torch()
    off, off_p = _offsets_arr(offsets)
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.int64).reshape(-1))
    nm, ns = len(cache.modes), len(src)
    dev = cache["V"].device
    shape = (ns, nm, nx * nz)
    if out is None:
        fd = _fdtype(cache.precision)
        out = (torch.empty(shape, dtype=fd, device=dev), torch.empty(shape, dtype=fd, device=dev),
               torch.empty(shape, dtype=torch.int32, device=dev) if parents else None,
               torch.empty(shape, dtype=torch.int32, device=dev) if parents else None)
    st = cache.struct()
    _check(lib().chert_traveltime_static(ctypes.byref(st), nm, cache.n_classes, cache.n_dir, nx, 1, nz,
                                         float(dx), _dev_ptr(d_cls), off_p, len(off),
                                         src.ctypes.data_as(ctypes.c_void_p), ns, cache.precision,
                                         max_cycles, _dev_ptr(out[0]), _dev_ptr(out[1]),
                                         _dev_ptr(out[2]), _dev_ptr(out[3]), _stream_ptr(stream)))
    return out


SCHEDULERS = {"sweeps": 0, "block_heap": 1, "hybrid": 2, "frontier": 3}


def set_relax_scheduler(name):
    """Scheduler of every later 2D relaxation in this process: "sweeps"
    (ordered sweep cycles), "block_heap" (block-heap marching of Eq. 32),
    "hybrid" (the default: at most 6 sweep cycles, then block-heap marching,
    from the source, for the fields that have not converged) or "frontier"
    (label correcting: pushes from the nodes that changed, atomicMin on the
    traveltimes' bit patterns).  All return the same fields and parents.
    Returns the previous name."""
    if name not in SCHEDULERS:
        raise ValueError("scheduler %r: one of %s" % (name, sorted(SCHEDULERS)))
    prev = lib().chert_set_relax_scheduler(SCHEDULERS[name])
    _check(prev if prev < 0 else 0)
    return {v: k for k, v in SCHEDULERS.items()}[prev]


def relax_scheduler():
    """Name of the current 2D relaxation scheduler."""
    return {v: k for k, v in SCHEDULERS.items()}[lib().chert_set_relax_scheduler(-1)]


def raypath(par, sources, receivers, cap=4096, stream=None, out=None):
    """chert_raypath for a batch of fields.

    par: int32 [n_fields, n_nodes] (or [n_nodes] for one field); sources: one
    source node per field; returns (paths int64 [n_fields, n_rcv, cap], lengths
    int64 [n_fields, n_rcv]), paths source-first."""
    torch = _torch()
    dev = par.device
    par2 = par.reshape(-1, par.shape[-1])
    nf, nn = par2.shape
    src = sources if torch.is_tensor(sources) else \
        torch.as_tensor(np.asarray(sources, dtype=np.int64).reshape(-1), device=dev)
    if src.numel() != nf:
        raise ValueError("need one source per field")
    rcv = receivers if torch.is_tensor(receivers) else \
        torch.as_tensor(np.asarray(receivers, dtype=np.int64).reshape(-1), device=dev)
    if out is None:
        out = (torch.full((nf, len(rcv), cap), -1, dtype=torch.int64, device=dev),
               torch.empty((nf, len(rcv)), dtype=torch.int64, device=dev))
    _check(lib().chert_raypath(_dev_ptr(par2), nf, nn, _dev_ptr(src), _dev_ptr(rcv), len(rcv), cap,
                               _dev_ptr(out[0]), _dev_ptr(out[1]), _stream_ptr(stream)))
    return out


def parent_ties(cache, nx, nz, dx, d_cls, offsets, sources, tauR, tauI, rel_tol, ny=1, precision=None,
                stream=None):
    """chert_parent_ties: the tie log of the parent rule for converged fields.

    Rebuilds the lookup tables of ``cache`` (chert_edge_table), then flags every
    node whose two best predecessor candidates lie within rel_tol of each
    other.  Returns (tieR, tieI) uint8 tensors shaped like the fields and the
    per-field counts int64 [n_fields, 2]."""
    torch = _torch()
    off, off_p = _offsets_arr(offsets)
    _, Vs, As = edge_table(cache, offsets, stream)
    prec = cache.precision if precision is None else (PRECISION_IDS[precision] if isinstance(precision, str)
                                                      else precision)
    src = sources if torch.is_tensor(sources) else \
        torch.as_tensor(np.asarray(sources, dtype=np.int64).reshape(-1), device=tauR.device)
    nm, ns = len(cache.modes), int(src.numel())
    tieR = torch.empty(tauR.shape, dtype=torch.uint8, device=tauR.device)
    tieI = torch.empty_like(tieR)
    counts = torch.empty((ns * nm, 2), dtype=torch.int64, device=tauR.device)
    _check(lib().chert_parent_ties(_dev_ptr(Vs), _dev_ptr(As), nm, cache.n_classes, prec, nx, ny, nz, float(dx),
                                   _dev_ptr(d_cls), off_p, len(off), _dev_ptr(src), ns, _dev_ptr(tauR),
                                   _dev_ptr(tauI), float(rel_tol), _dev_ptr(tieR), _dev_ptr(tieI),
                                   _dev_ptr(counts), _stream_ptr(stream)))
    return tieR, tieI, counts


def _host_ptr(t):
    if t is None:
        return None
    if t.is_cuda or not t.is_contiguous():
        raise ValueError("host tensor must be contiguous CPU memory")
    return ctypes.c_void_p(t.data_ptr())


def trace_host_scratch_bytes(n_classes, n_modes, M, nx, nz, n_off, n_sources, n_rcv, path_cap, precision):
    return int(lib().chert_trace_host_scratch_bytes(n_classes, n_modes, M, nx, nz, n_off, n_sources, n_rcv,
                                                    path_cap, precision))


def trace_host(h_classes, n_classes, modes, M, nx, nz, dx, h_cls, offsets, h_sources, h_receivers, h_tauR, h_tauI,
               h_paths, h_lens, d_scratch, scratch_step=0.001 * math.pi / 180, scan_half=30000, kernel="MEV",
               precision="mixed", max_cycles=64, stream=None):
    """chert_trace_host: the whole path on host tensors (inputs and outputs
    page-locked CPU tensors, d_scratch a device uint8 tensor of
    trace_host_scratch_bytes)."""
    prec = PRECISION_IDS[precision] if isinstance(precision, str) else precision
    mode_ids = [MODE_IDS[m] if isinstance(m, str) else m for m in modes]
    off, off_p = _offsets_arr(offsets)
    params = chert_cache_params(M, scratch_step, scan_half, KERNEL_IDS.get(kernel, kernel), prec)
    modes_arr = (ctypes.c_int * len(mode_ids))(*mode_ids)
    n_rcv = int(h_receivers.numel())
    cap = int(h_paths.shape[-1])
    _check(lib().chert_trace_host(_host_ptr(h_classes), n_classes, modes_arr, len(mode_ids), ctypes.byref(params),
                                  nx, nz, float(dx), _host_ptr(h_cls), off_p, len(off), _host_ptr(h_sources),
                                  int(h_sources.numel()), max_cycles, _host_ptr(h_receivers), n_rcv, cap,
                                  _host_ptr(h_tauR), _host_ptr(h_tauI), _host_ptr(h_paths), _host_ptr(h_lens),
                                  _dev_ptr(d_scratch), d_scratch.numel(), _stream_ptr(stream)))


def fma_rate(precision="fp32", iters=1 << 16, stream=None):
    """Measured FMA throughput of the current device in flop/s (chert_fma_rate)."""
    out = ctypes.c_double(0.0)
    prec = PRECISION_IDS[precision] if isinstance(precision, str) else precision
    _check(lib().chert_fma_rate(prec, int(iters), ctypes.byref(out), _stream_ptr(stream)))
    return out.value


class EvalCounter:
    """Context manager around chert_cache_eval_counter: counts the energy
    velocity evaluations of the cache builds run inside it (.counts =
    [float, float-float, double] after exit)."""

    def __enter__(self):
        _check(lib().chert_cache_eval_counter(1, None))
        return self

    def __exit__(self, *exc):
        c = (ctypes.c_ulonglong * 3)()
        _check(lib().chert_cache_eval_counter(0, ctypes.cast(c, ctypes.c_void_p)))
        self.counts = [int(v) for v in c]
        return False


# ------------------------------------------------------------------ surrogate
def mlp_param_count():
    return int(lib().chert_mlp_param_count())


def mlp_forward(params, x, stream=None, workspace=None):
    """Standardised network outputs y [n, 5] for features x [n, 8] (device)."""
    torch = _torch()
    n = x.shape[0]
    y = torch.empty((n, 5), dtype=torch.float32, device=x.device)
    wsb = int(lib().chert_mlp_workspace_bytes(n, 0))
    if workspace is None or workspace.numel() < wsb:
        workspace = torch.empty(wsb, dtype=torch.uint8, device=x.device)
    _check(lib().chert_mlp_forward(_dev_ptr(params), _dev_ptr(x), n, _dev_ptr(y), _dev_ptr(workspace),
                                   workspace.numel(), _stream_ptr(stream)))
    return y


def mlp_train_step(params, m, v, step, lr, x, t, stream=None, workspace=None, want_grad=False, loss=None):
    """One Adam step (lr > 0) or a gradient evaluation (lr = 0); returns (loss tensor, grad or None)."""
    torch = _torch()
    n = x.shape[0]
    wsb = int(lib().chert_mlp_workspace_bytes(n, 1))
    if workspace is None or workspace.numel() < wsb:
        workspace = torch.empty(wsb, dtype=torch.uint8, device=x.device)
    grad = torch.empty_like(params) if want_grad else None
    if loss is None:
        loss = torch.zeros(1, dtype=torch.float32, device=x.device)
    _check(lib().chert_mlp_train_step(_dev_ptr(params), _dev_ptr(m), _dev_ptr(v), int(step), float(lr),
                                      _dev_ptr(x), _dev_ptr(t), n, _dev_ptr(loss), _dev_ptr(grad),
                                      _dev_ptr(workspace), workspace.numel(), _stream_ptr(stream)))
    return loss, grad


def surrogate_dataset(d_classes, n_classes, M, mode, mode_slot, exact_cache, stream=None):
    """(x [n, 8], t [n, 5]) training pairs from an exact cache (device tensors)."""
    torch = _torch()
    n = n_classes * (M + 1)
    dev = d_classes.device
    x = torch.empty((n, 8), dtype=torch.float32, device=dev)
    t = torch.empty((n, 5), dtype=torch.float32, device=dev)
    scratch = torch.empty(13 * n + 256, dtype=torch.uint8, device=dev)
    st = exact_cache.struct()
    mid = MODE_IDS[mode] if isinstance(mode, str) else mode
    _check(lib().chert_surrogate_dataset(_dev_ptr(d_classes), n_classes, M, mid, mode_slot, ctypes.byref(st),
                                         exact_cache.precision, _dev_ptr(x), _dev_ptr(t), _dev_ptr(scratch),
                                         scratch.numel(), _stream_ptr(stream)))
    return x, t


def set_surrogate_qsv_angle(rad):
    """qSV fallback angle of surrogate_cache (radians; process-wide); returns
    the previous one."""
    return float(lib().chert_set_surrogate_qsv_angle(float(rad)))


def cache_surrogate(params_per_mode, d_classes, n_classes, modes, M, scan_step=0.001 * math.pi / 180,
                    scan_half=30000, kernel="MEV", precision="mixed", stream=None, out=None):
    """chert_cache_surrogate: the networks' cache with every solve they hand
    back recomputed by the exact solver, enqueued without a host read.
    Returns the Cache; cache.n_fallback_dev is a device int64 tensor [1] with
    the number of solves recomputed exactly."""
    torch = _torch()
    prec = PRECISION_IDS[precision] if isinstance(precision, str) else precision
    mode_ids = [MODE_IDS[m] if isinstance(m, str) else m for m in modes]
    dev = d_classes.device
    shape = (len(mode_ids), n_classes, 4 * M)
    if out is None:
        fd = _fdtype(prec)
        out = {k: torch.empty(shape, dtype=fd, device=dev)
               for k in ("V", "A", "Q", "rx", "rz", "theta", "vartheta")}
        out["flag"] = torch.empty(shape, dtype=torch.uint8, device=dev)
    cache = Cache(out, mode_ids, n_classes, M, prec)
    wsb = int(lib().chert_cache_surrogate_workspace_bytes(n_classes, len(mode_ids), M))
    if wsb == 0:
        raise ChertError(EINVAL, "cache_surrogate: bad sizes")
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    cache.n_fallback_dev = torch.zeros(1, dtype=torch.int64, device=dev)
    p = chert_cache_params(M, scan_step, scan_half, KERNEL_IDS.get(kernel, kernel), prec)
    ptrs = (ctypes.c_void_p * len(mode_ids))(*[q.data_ptr() for q in params_per_mode])
    modes_arr = (ctypes.c_int * len(mode_ids))(*mode_ids)
    st = cache.struct()
    _check(lib().chert_cache_surrogate(ptrs, _dev_ptr(d_classes), n_classes, modes_arr, len(mode_ids),
                                       ctypes.byref(p), ctypes.byref(st), _dev_ptr(ws), ws.numel(),
                                       _dev_ptr(cache.n_fallback_dev), _stream_ptr(stream)))
    cache.workspace = ws
    return cache


def angular_coverage(cache, offsets, truth_flag=None, stream=None):
    """chert_angular_coverage for a 2D Cache: (covered, mismatched, missing)
    device int32 tensors [n_modes, n_classes]."""
    torch = _torch()
    off, off_p = _offsets_arr(offsets)
    nm, nk = len(cache.modes), cache.n_classes
    dev = cache["V"].device
    outs = [torch.empty((nm, nk), dtype=torch.int32, device=dev) for _ in range(3)]
    st = cache.struct()
    _check(lib().chert_angular_coverage(ctypes.byref(st), nm, nk, cache.n_dir, cache.precision, off_p, len(off),
                                        None if truth_flag is None else _dev_ptr(truth_flag),
                                        *[_dev_ptr(t) for t in outs], _stream_ptr(stream)))
    return tuple(outs)


def mlp_check(stream=None):
    """chert_mlp_check: raises ChertError(ETIMEOUT) if a tensor-core GEMM wait
    ran out since the last check (and clears the status)."""
    _check(lib().chert_mlp_check(_stream_ptr(stream)))


def mlp_set_wait_limit(polls):
    """chert_mlp_set_wait_limit; returns the previous limit (polls < 0 queries)."""
    return int(lib().chert_mlp_set_wait_limit(int(polls)))


def surrogate_cache(params_per_mode, d_classes, n_classes, modes, M, precision="fp32", stream=None, out=None):
    """Cache arrays (same layout as build_cache) filled by the networks."""
    torch = _torch()
    prec = PRECISION_IDS[precision] if isinstance(precision, str) else precision
    mode_ids = [MODE_IDS[m] if isinstance(m, str) else m for m in modes]
    dev = d_classes.device
    shape = (len(mode_ids), n_classes, 4 * M)
    if out is None:
        fd = _fdtype(prec)
        out = {k: torch.empty(shape, dtype=fd, device=dev)
               for k in ("V", "A", "Q", "rx", "rz", "theta", "vartheta")}
        out["flag"] = torch.empty(shape, dtype=torch.uint8, device=dev)
    cache = Cache(out, mode_ids, n_classes, M, prec)
    wsb = int(lib().chert_surrogate_cache_workspace_bytes(n_classes, M))
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    ptrs = (ctypes.c_void_p * len(mode_ids))(*[p.data_ptr() for p in params_per_mode])
    modes_arr = (ctypes.c_int * len(mode_ids))(*mode_ids)
    st = cache.struct()
    _check(lib().chert_surrogate_cache(ptrs, _dev_ptr(d_classes), n_classes, modes_arr, len(mode_ids), M, prec,
                                       ctypes.byref(st), _dev_ptr(ws), ws.numel(), _stream_ptr(stream)))
    return cache
