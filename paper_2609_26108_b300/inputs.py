"""Seeded synthetic inputs shaped like the workloads of CHERT (Darwis et al.).

This module only *describes* media, grids, stencils and sources.  It holds none
of the method's arithmetic: no Thomsen-to-moduli conversion, no Christoffel
solve, no lookup and no relaxation.  Both the CUDA path (through the
``chert`` binding) and the FP64 oracle under ``oracle/`` take what these
generators return as plain arrays.

Random numbers come from NumPy's PCG64 (``numpy.random.default_rng``) with the
fixed seeds below, so every call returns the same model.

Workloads (the recipes are restated with their citations in the design notes):

* ``homogeneous_vti``  -- 2D homogeneous viscoelastic VTI, one class
  (Vp0=3000 m/s, Vs0=1500 m/s, rho=2200, eps=0.2, delta=0.1, gamma=0.1,
  Qp=60, Qs=30), 101x101 nodes at dx=10 m, one centre source.
* ``layered_tti``      -- 2D layered viscoelastic TTI, 401x401 nodes at
  dx=10 m, 8 flat layers of seeded Thomsen parameters and tilts, 64 surface
  sources.
* ``table2_layers``    -- the four visco-VTI layers that the paper prints in its
  Table 2 (moduli in (km/s)^2 and per-component quality factors).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "ThomsenLayer", "TableLayer", "Model2D",
    "homogeneous_vti", "layered_tti", "table2_layers",
    "layered_class_map_2d", "stencil_2d", "stencil_3d", "surface_sources_2d",
    "SEEDS",
]

# One seed per workload (PCG64).
SEEDS = {"homogeneous_vti": 1001, "layered_tti": 1002, "layered_tti_3d": 1004}


@dataclass(frozen=True)
class ThomsenLayer:
    """Thomsen-style description of one cache class (SI units, tilt in rad)."""
    vp0: float
    vs0: float
    eps: float
    delta: float
    gamma: float
    qp: float
    qs: float
    rho: float = 2200.0
    tilt: float = 0.0
    azim: float = 0.0


@dataclass(frozen=True)
class TableLayer:
    """Density-normalised real moduli a11,a13,a33,a44,a66 in (m/s)^2 and the
    per-component quality factors q11,q13,q33,q44,q66 (Table 2 form)."""
    aR: tuple
    q: tuple
    rho: float = 2200.0
    tilt: float = 0.0
    azim: float = 0.0


@dataclass
class Model2D:
    """A 2D model on an nx x nz node lattice (x fastest, z = depth rows)."""
    name: str
    nx: int
    nz: int
    dx: float
    layers: list
    class_of_node: np.ndarray            # uint8/uint16 [nz*nx], node = x + nx*z
    sources: np.ndarray                  # int64 node indices
    info: dict = field(default_factory=dict)


# Table 2 of the paper: four layers of a 2D viscoelastic VTI model, moduli in
# (km/s)^2 (converted to (m/s)^2 here) and quality factors per component.
_TABLE2 = [
    ((14.40, 4.50, 9.00, 2.25, 3.00), (30.0, 15.0, 20.0, 15.0, 12.0)),
    ((21.60, 6.75, 13.50, 3.38, 4.50), (45.0, 22.5, 30.0, 22.5, 18.0)),
    ((28.80, 9.00, 18.00, 4.50, 6.00), (60.0, 30.0, 40.0, 30.0, 24.0)),
    ((36.00, 11.25, 22.50, 5.63, 7.50), (75.0, 37.5, 50.0, 37.5, 30.0)),
]


def table2_layers(tilt: float = 0.0) -> list:
    """The paper's Table 2 layers as ``TableLayer`` records in SI units."""
    return [TableLayer(aR=tuple(v * 1e6 for v in aR), q=tuple(q), tilt=tilt)
            for aR, q in _TABLE2]


def stencil_2d(radius: int) -> np.ndarray:
    """Offsets (ox, oy=0, oz) with Chebyshev norm <= radius and gcd(|ox|,|oz|) = 1.

    The gcd rule keeps one offset per lattice direction, so radius 5 gives 80
    offsets.  Returned as int32 [n_off, 3], sorted by (oz, ox).
    """
    out = []
    for oz in range(-radius, radius + 1):
        for ox in range(-radius, radius + 1):
            if (ox or oz) and math.gcd(abs(ox), abs(oz)) == 1:
                out.append((ox, 0, oz))
    return np.asarray(out, dtype=np.int32)


def stencil_3d(radius: int) -> np.ndarray:
    """3D analogue of ``stencil_2d``: radius 2 gives the 26 neighbours plus the
    72 secondary directions (98 offsets).  int32 [n_off, 3], sorted by (oz, oy, ox)."""
    out = []
    for oz in range(-radius, radius + 1):
        for oy in range(-radius, radius + 1):
            for ox in range(-radius, radius + 1):
                if (ox or oy or oz) and math.gcd(math.gcd(abs(ox), abs(oy)), abs(oz)) == 1:
                    out.append((ox, oy, oz))
    return np.asarray(out, dtype=np.int32)


def layered_class_map_2d(nx: int, nz: int, n_layers: int) -> np.ndarray:
    """Flat layers of equal thickness; a node on an interface joins the deeper layer.

    Interfaces sit at depths i*(nz-1)/n_layers (in node units), i = 1..n_layers-1.
    Returns uint8 [nz*nx] with node = x + nx*z.
    """
    z = np.arange(nz, dtype=np.float64)
    bounds = np.arange(1, n_layers) * (nz - 1) / n_layers
    layer_of_row = np.searchsorted(bounds, z, side="right").astype(np.uint8)
    return np.repeat(layer_of_row, nx)


def surface_sources_2d(nx: int, n: int) -> np.ndarray:
    """n sources on the surface row z=0 at x = round(linspace(0, nx-1, n))."""
    xs = np.round(np.linspace(0, nx - 1, n)).astype(np.int64)
    return xs  # z = 0, so node index = x


def homogeneous_vti(nx: int = 101, nz: int = 101) -> Model2D:
    """2D homogeneous visco-VTI: one class, centre source, dx = 10 m."""
    layer = ThomsenLayer(vp0=3000.0, vs0=1500.0, eps=0.2, delta=0.1, gamma=0.1,
                         qp=60.0, qs=30.0, rho=2200.0)
    cls = np.zeros(nx * nz, dtype=np.uint8)
    src = np.array([(nx // 2) + nx * (nz // 2)], dtype=np.int64)
    return Model2D("homogeneous_vti_%dx%d" % (nx, nz), nx, nz, 10.0, [layer], cls, src)


def seeded_tti_layers(n_layers: int, seed: int) -> list:
    """Seeded Thomsen layers: Vp0 ~ U(2000,4500) sorted with depth,
    Vp0/Vs0 ~ U(1.7,2.0), eps ~ U(0.05,0.3), delta ~ U(-0.1,0.2),
    gamma ~ U(0,0.2), tilt ~ U(0,45 deg), Qp,Qs ~ logU(20,200) with Qs <= Qp."""
    rng = np.random.default_rng(seed)
    vp0 = np.sort(rng.uniform(2000.0, 4500.0, n_layers))
    ratio = rng.uniform(1.7, 2.0, n_layers)
    eps = rng.uniform(0.05, 0.3, n_layers)
    delta = rng.uniform(-0.1, 0.2, n_layers)
    gamma = rng.uniform(0.0, 0.2, n_layers)
    tilt = np.deg2rad(rng.uniform(0.0, 45.0, n_layers))
    qa = np.exp(rng.uniform(math.log(20.0), math.log(200.0), n_layers))
    qb = np.exp(rng.uniform(math.log(20.0), math.log(200.0), n_layers))
    qp, qs = np.maximum(qa, qb), np.minimum(qa, qb)
    return [ThomsenLayer(vp0=float(vp0[i]), vs0=float(vp0[i] / ratio[i]), eps=float(eps[i]),
                         delta=float(delta[i]), gamma=float(gamma[i]), qp=float(qp[i]),
                         qs=float(qs[i]), rho=2200.0, tilt=float(tilt[i]))
            for i in range(n_layers)]


def layered_tti(nx: int = 401, nz: int = 401, n_layers: int = 8, n_sources: int = 64,
                seed: int = SEEDS["layered_tti"]) -> Model2D:
    """2D layered visco-TTI, flat layers of equal thickness, surface sources."""
    layers = seeded_tti_layers(n_layers, seed)
    cls = layered_class_map_2d(nx, nz, n_layers)
    src = surface_sources_2d(nx, n_sources)
    return Model2D("layered_tti_%dx%d_%dL_%dsrc" % (nx, nz, n_layers, n_sources),
                   nx, nz, 10.0, layers, cls, src)


def random_class_map_2d(nx: int, nz: int, n_classes: int, seed: int) -> np.ndarray:
    """Per-node random classes (a stress case for the lookup and the relaxation)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, n_classes, nx * nz).astype(np.uint8)


def random_tti_classes(n: int, seed: int, q_lo: float = 20.0, q_hi: float = 200.0) -> list:
    """n independent seeded TTI media over the surrogate's training range
    (Vp0 ~ U(2000, 4500), Vp0/Vs0 ~ U(1.7, 2.0), eps ~ U(0.05, 0.3),
    delta ~ U(-0.1, 0.2), gamma ~ U(0, 0.2), tilt ~ U(0, 45 deg),
    Qp, Qs ~ logU(q_lo, q_hi) with Qs <= Qp)."""
    rng = np.random.default_rng(seed)
    vp0 = rng.uniform(2000.0, 4500.0, n)
    ratio = rng.uniform(1.7, 2.0, n)
    eps = rng.uniform(0.05, 0.3, n)
    delta = rng.uniform(-0.1, 0.2, n)
    gamma = rng.uniform(0.0, 0.2, n)
    tilt = np.deg2rad(rng.uniform(0.0, 45.0, n))
    qa = np.exp(rng.uniform(math.log(q_lo), math.log(q_hi), n))
    qb = np.exp(rng.uniform(math.log(q_lo), math.log(q_hi), n))
    qp, qs = np.maximum(qa, qb), np.minimum(qa, qb)
    return [ThomsenLayer(vp0=float(vp0[i]), vs0=float(vp0[i] / ratio[i]), eps=float(eps[i]),
                         delta=float(delta[i]), gamma=float(gamma[i]), qp=float(qp[i]), qs=float(qs[i]),
                         rho=2200.0, tilt=float(tilt[i])) for i in range(n)]


def mlp_init(seed: int, n_in: int = 7, n_hid: int = 256, n_layers: int = 4, n_out: int = 5) -> list:
    """Seeded He-normal initial weights [(W [out, in], b [out]), ...] (float64)."""
    rng = np.random.default_rng(seed)
    sizes = [n_in] + [n_hid] * n_layers + [n_out]
    return [(rng.normal(0.0, math.sqrt(2.0 / a), (b_, a)), np.zeros(b_)) for a, b_ in zip(sizes[:-1], sizes[1:])]


@dataclass
class CellModel2D:
    """A 2D model with its own medium at every node (one cache class per node)."""
    name: str
    nx: int
    nz: int
    dx: float
    params: dict                         # per-node arrays: vp0 vs0 eps delta gamma qp qs tilt
    layer_of_node: np.ndarray            # int32 [nz*nx]
    sources: np.ndarray


def folded_faulted(nx: int = 1701, nz: int = 351, n_layers: int = 10, n_sources: int = 64,
                   seed: int = 1003, dx: float = 10.0) -> CellModel2D:
    """Seeded folded and faulted layered visco-TTI model with per-node media.

    Interfaces z_i(x) = zbar_i + A_i sin(2 pi x / lambda_i + phi_i) (node units,
    A ~ U(3%, 6%) of the depth, lambda ~ U(0.2, 0.6) of the width); one normal
    fault at x_f ~ U(0.35, 0.65) nx dipping 60 deg with a 150 m throw (the
    hanging wall's layers sit 150 m deeper).  Per layer: Thomsen means as in
    ``seeded_tti_layers``; per node: the layer mean times (1 + g x') with
    g ~ U(-0.06, 0.06) per layer and parameter, x' = x/(nx-1) - 1/2, plus
    0.5% white noise; the symmetry axis follows the local dip of the layer's
    top interface plus the layer's tilt.  Surface sources as in layered_tti."""
    rng = np.random.default_rng(seed)
    base = seeded_tti_layers(n_layers, int(rng.integers(1 << 30)))
    x = np.arange(nx, dtype=np.float64)
    z = np.arange(nz, dtype=np.float64)
    zbar = np.arange(1, n_layers) * (nz - 1) / n_layers
    amp = rng.uniform(0.03, 0.06, n_layers - 1) * nz
    lam = rng.uniform(0.2, 0.6, n_layers - 1) * nx
    ph = rng.uniform(0.0, 2 * math.pi, n_layers - 1)
    iface = zbar[:, None] + amp[:, None] * np.sin(2 * math.pi * x[None] / lam[:, None] + ph[:, None])
    slope = amp[:, None] * (2 * math.pi / lam[:, None]) * np.cos(2 * math.pi * x[None] / lam[:, None] + ph[:, None])
    xf = rng.uniform(0.35, 0.65) * nx
    throw = 150.0 / dx
    hanging = x[None, :] > xf + z[:, None] / math.tan(math.radians(60.0))
    zz = z[:, None] - np.where(hanging, throw, 0.0)
    layer = (iface[:, None, :] <= zz[None]).sum(axis=0).astype(np.int32)           # [nz, nx]
    top = np.clip(layer - 1, 0, n_layers - 2)
    dip = np.arctan(slope[top, np.arange(nx)[None, :]])
    xp = x / (nx - 1) - 0.5
    out = {}
    for key in ("vp0", "ratio", "eps", "delta", "gamma", "qp", "qs"):
        g = rng.uniform(-0.06, 0.06, n_layers)
        if key == "ratio":
            mean = np.array([L.vp0 / L.vs0 for L in base])
        else:
            mean = np.array([getattr(L, key) for L in base])
        field_ = mean[layer] * (1.0 + g[layer] * xp[None, :])
        field_ = field_ * (1.0 + 0.005 * rng.standard_normal((nz, nx)))
        out[key] = field_
    out["ratio"] = np.clip(out["ratio"], 1.6, 2.1)
    out["qs"] = np.minimum(out["qs"], out["qp"])
    params = {"vp0": out["vp0"].reshape(-1), "vs0": (out["vp0"] / out["ratio"]).reshape(-1),
              "eps": out["eps"].reshape(-1), "delta": out["delta"].reshape(-1),
              "gamma": np.clip(out["gamma"], 0.0, None).reshape(-1), "qp": out["qp"].reshape(-1),
              "qs": out["qs"].reshape(-1),
              "tilt": (np.array([L.tilt for L in base])[layer] + dip).reshape(-1)}
    src = surface_sources_2d(nx, n_sources)
    return CellModel2D("folded_faulted_%dx%d_%dsrc" % (nx, nz, n_sources), nx, nz, dx, params,
                       layer.reshape(-1), src)


@dataclass
class Model3D:
    """A 3D layered model: classes per layer, node = x + nx*(y + ny*z)."""
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    layers: list
    class_of_node: np.ndarray
    sources: np.ndarray


def layered_tti_3d(n: int = 201, n_layers: int = 12, n_sources: int = 16,
                   seed: int = SEEDS["layered_tti_3d"], vti: bool = False) -> Model3D:
    """3D layered visco-TTI on an n^3 lattice (dx = 10 m): flat layers of equal
    thickness with the seeded Thomsen parameters of ``seeded_tti_layers`` and
    a symmetry-axis azimuth phi0 ~ U(0, 360 deg) per layer (VTI variant: no
    tilt); sources on a sqrt(n_sources)^2 grid on the surface z = 0."""
    rng = np.random.default_rng(seed + 1)
    layers = seeded_tti_layers(n_layers, seed)
    from dataclasses import replace
    azim = rng.uniform(0.0, 2 * math.pi, n_layers)
    layers = [replace(L, tilt=0.0 if vti else L.tilt, azim=0.0 if vti else float(a))
              for L, a in zip(layers, azim)]
    z = np.arange(n, dtype=np.float64)
    bounds = np.arange(1, n_layers) * (n - 1) / n_layers
    layer_of_z = np.searchsorted(bounds, z, side="right").astype(np.int32)
    cls = np.repeat(layer_of_z, n * n)
    m = int(round(math.sqrt(n_sources)))
    pos = np.round(np.linspace(0, n - 1, m + 2)[1:-1]).astype(np.int64)
    src = np.array([x + n * y for y in pos for x in pos], dtype=np.int64)
    return Model3D("layered_tti_3d_%d^3_%dsrc" % (n, len(src)), n, n, n, 10.0, layers, cls, src)


def subvolume_3d(model: Model3D, n: int, seed: int, n_sources: int) -> Model3D:
    """An n^3 block of a 3D model cut at a seeded corner (PCG64), its top face
    at the model's surface row z0, sources on a sqrt(n_sources)^2 grid on
    that face."""
    rng = np.random.default_rng(seed)
    x0 = int(rng.integers(0, model.nx - n + 1))
    y0 = int(rng.integers(0, model.ny - n + 1))
    z0 = int(rng.integers(0, model.nz - n + 1))
    cls = model.class_of_node.reshape(model.nz, model.ny, model.nx)[z0:z0 + n, y0:y0 + n, x0:x0 + n]
    m = int(round(math.sqrt(n_sources)))
    pos = np.round(np.linspace(0, n - 1, m + 2)[1:-1]).astype(np.int64)
    src = np.array([x + n * y for y in pos for x in pos], dtype=np.int64)
    return Model3D("%s_sub%d^3_at_%d_%d_%d" % (model.name, n, x0, y0, z0), n, n, n, model.dx, model.layers,
                   np.ascontiguousarray(cls).reshape(-1), src)
