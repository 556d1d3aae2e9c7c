"""Write the FP64 oracle's cache solves at the benchmark's full scan grid.

    python tests/golden/make_cache_golden.py [--procs N]

Calls only ``oracle/cache_oracle.py`` (and the seeded model descriptions of
``paper_2609_26108_b300/inputs.py``, which hold none of the method's
arithmetic).  Two files, one line per folded solve (mode, class, folded angle
j = 0..M at theta_j = j*(pi/2)/M), MEV kernel, M = 90 (1 deg cache), scan
step h = 0.001 deg, K = 30000 (the [-30, 30] deg bracket):

* ``layered_tti_cache_M90.txt``: every solve of the 8 classes of the layered
  401x401 model (PCG64 seed 1002) in qP, qSV and qSH: 2,184 solves.
* ``folded_cells_cache_M90.txt``: 48 cells of the folded and faulted per-cell
  model (seed 1003) drawn (PCG64 seed 4242) from a 241 x 101 slice of it
  (x 730..970, z 120..220, across the fault), with their Thomsen parameters,
  in qP, qSV and qSH: 13,104 solves.
* ``homogeneous_vti_cache_M90.txt``: the one class of the small homogeneous
  visco-VTI case (inputs.homogeneous_vti(): Vp0 3000, Vs0 1500, eps 0.2,
  delta 0.1, gamma 0.1, Qp 60, Qs 30) in qP, qSV and qSH: 273 solves.

``--which homogeneous`` writes that one only.

Each solve line: mode class j flag vartheta V A Q r_x r_z, with r the ray
direction in the class's symmetry-axis frame (before the tilt rotation);
float64 values written with 17 significant digits (exact round trip).
"""
from __future__ import annotations

import argparse
import math
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DEG = math.pi / 180.0
M = 90
H = 0.001 * DEG
K = 30000
MODES = ("qP", "qSV", "qSH")
SLICE = dict(x0=730, x1=971, z0=120, z1=221)     # 241 x 101 nodes
N_CELLS = 48
CELL_SEED = 4242
THOMSEN_KEYS = ("vp0", "vs0", "eps", "delta", "gamma", "qp", "qs", "tilt")


def slice_cells():
    """Node indices of the sampled cells and the slice geometry (shared with
    the tests, which rebuild the slice from the same seeded model)."""
    import numpy as np
    from paper_2609_26108_b300 import inputs
    fm = inputs.folded_faulted(n_sources=1)
    xs = np.arange(SLICE["x0"], SLICE["x1"])
    zs = np.arange(SLICE["z0"], SLICE["z1"])
    nodes = (xs[None, :] + fm.nx * zs[:, None]).reshape(-1)
    rng = np.random.default_rng(CELL_SEED)
    cells = np.sort(rng.choice(nodes, N_CELLS, replace=False))
    return fm, cells


def _solve(task):
    """One (mode, class) row of M+1 folded solves by the oracle (single thread)."""
    from threadpoolctl import threadpool_limits
    from oracle import cache_oracle as co
    mode, a5 = task
    with threadpool_limits(1):
        return co.folded_solves(co.stiffness_tensor(a5), mode, M, "MEV", H, K)


def _fmt(x):
    return repr(float(x))


def write(path, header, rows, tasks_meta):
    with open(path, "w") as f:
        for line in header:
            f.write("# " + line + "\n")
        for (mode, k), solves in zip(tasks_meta, rows):
            for j, s in enumerate(solves):
                f.write(" ".join([mode, str(k), str(j), str(int(s["flag"])), _fmt(s["vartheta"]), _fmt(s["V"]),
                                  _fmt(s["A"]), _fmt(s["Q"]), _fmt(s["r"][0]), _fmt(s["r"][2])]) + "\n")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--which", default="all", choices=["all", "homogeneous"])
    args = ap.parse_args()
    from oracle import cache_oracle as co
    from paper_2609_26108_b300 import inputs

    common = ["written by tests/golden/make_cache_golden.py from oracle/cache_oracle.py alone",
              "kernel MEV, M = %d, scan step 0.001 deg, K = %d" % (M, K),
              "columns: mode class j flag vartheta V A Q r_x r_z (r in the symmetry-axis frame)"]
    if True:                                   # the homogeneous case (every run)
        L = inputs.homogeneous_vti().layers[0]
        a5 = co.moduli_from_thomsen(L.vp0, L.vs0, L.eps, L.delta, L.gamma, L.qp, L.qs)
        meta = [(m, 0) for m in MODES]
        with mp.get_context("spawn").Pool(min(args.procs, len(meta))) as pool:
            rows = pool.map(_solve, [(m, a5) for m, _ in meta], chunksize=1)
        write(os.path.join(HERE, "homogeneous_vti_cache_M90.txt"),
              ["homogeneous visco-VTI: inputs.homogeneous_vti(), 1 class"] + common + ["tilts: " + _fmt(L.tilt)],
              rows, meta)
        if args.which == "homogeneous":
            return

    layered = inputs.layered_tti().layers
    lay_mods = [co.moduli_from_thomsen(L.vp0, L.vs0, L.eps, L.delta, L.gamma, L.qp, L.qs) for L in layered]
    fm, cells = slice_cells()
    p = fm.params
    cell_mods = [co.moduli_from_thomsen(*(float(p[key][c]) for key in THOMSEN_KEYS[:7])) for c in cells]

    lay_meta = [(m, k) for m in MODES for k in range(len(layered))]
    cell_meta = [(m, k) for m in MODES for k in range(len(cells))]
    tasks = [(m, lay_mods[k]) for m, k in lay_meta] + [(m, cell_mods[k]) for m, k in cell_meta]
    t0 = time.time()
    with mp.get_context("spawn").Pool(args.procs) as pool:
        rows = pool.map(_solve, tasks, chunksize=1)
    print("%d solves in %.0f s on %d processes" % ((M + 1) * len(tasks), time.time() - t0, args.procs))

    write(os.path.join(HERE, "layered_tti_cache_M90.txt"),
          ["layered 401x401 model: inputs.layered_tti(), 8 classes, PCG64 seed 1002"] + common +
          ["tilts: " + " ".join(_fmt(L.tilt) for L in layered)],
          rows[:len(lay_meta)], lay_meta)
    hdr = ["folded and faulted per-cell model inputs.folded_faulted() (seed 1003), %d cells drawn with PCG64 "
           "seed %d from the slice x %d..%d, z %d..%d" % (N_CELLS, CELL_SEED, SLICE["x0"], SLICE["x1"] - 1,
                                                         SLICE["z0"], SLICE["z1"] - 1)] + common
    hdr += ["cell %d %d %s" % (k, int(c), " ".join(_fmt(p[key][c]) for key in THOMSEN_KEYS))
            for k, c in enumerate(cells)]
    write(os.path.join(HERE, "folded_cells_cache_M90.txt"), hdr, rows[len(lay_meta):], cell_meta)


if __name__ == "__main__":
    main()
