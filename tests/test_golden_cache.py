"""The stored full-scan cache solves are the oracle's own output.

tests/golden/make_cache_golden.py writes them from oracle/cache_oracle.py
alone (MEV, 0.001 deg scan over [-30, 30] deg, 1 deg cache).  Here a seeded
sample of them is solved again by the oracle and must agree bit for bit, and
the files must cover every solve they claim (every mode, class and folded
angle)."""
import math

import numpy as np

from oracle import cache_oracle as co
from paper_2609_26108_b300 import inputs

from helpers import DEG, load_cache_golden

MODES = ("qP", "qSV", "qSH")


def _resolve(g, mods, picks):
    for mode, k, j in picks:
        s = co.solve_direction(co.stiffness_tensor(mods[k]), (math.pi / 2) * j / 90, mode, "MEV",
                               0.001 * DEG, 30000)
        want = g["folded"][(mode, k)][j]
        assert s["flag"] == want["flag"]
        for key in ("vartheta", "V", "A", "Q"):
            assert np.array_equal(np.float64(s[key]), np.float64(want[key]), equal_nan=True), (mode, k, j, key)
        assert np.array_equal(s["r"][[0, 2]], want["r"][[0, 2]], equal_nan=True)


def test_layered_golden_is_the_oracle():
    g = load_cache_golden("layered_tti_cache_M90.txt")
    layers = inputs.layered_tti().layers
    assert len(g["folded"]) == 3 * 8 and all(len(v) == 91 for v in g["folded"].values())
    assert np.allclose(g["tilts"], [L.tilt for L in layers], rtol=0, atol=0)
    mods = [co.moduli_from_thomsen(L.vp0, L.vs0, L.eps, L.delta, L.gamma, L.qp, L.qs) for L in layers]
    rng = np.random.default_rng(11)
    _resolve(g, mods, [(MODES[rng.integers(3)], int(rng.integers(8)), int(rng.integers(91))) for _ in range(2)])


def test_cell_golden_is_the_oracle():
    g = load_cache_golden("folded_cells_cache_M90.txt")
    assert len(g["cells"]) == 48 and len(g["folded"]) == 3 * 48
    fm = inputs.folded_faulted(n_sources=1)
    for node, p in g["cells"][:5]:
        for key, v in p.items():
            assert fm.params[key][node] == v
    mods = [co.moduli_from_thomsen(*(p[key] for key in ("vp0", "vs0", "eps", "delta", "gamma", "qp", "qs")))
            for _, p in g["cells"]]
    rng = np.random.default_rng(12)
    _resolve(g, mods, [("qSV", int(rng.integers(48)), int(rng.integers(91))) for _ in range(2)])


def test_homogeneous_golden_axes_closed_form_and_oracle():
    """The small case's golden (tests/golden/homogeneous_vti_cache_M90.txt):
    along the symmetry axis (j = 0) and across it (j = 90) of a VTI medium
    the qP, qSV and qSH waves are homogeneous plane waves with ray along the
    slowness, so vartheta = 0 and, with c^2 the modulus of the direction
    (qP: a33 / a11; qSV: a44 both ways; qSH: a44 / a66), V = 1/Re(1/c),
    A = Im(1/c), Q = -Re(c^2)/Im(c^2) (Eq. 10-11).  The C1 moduli (a11 =
    1.26e7, a13 = 5.3468744e6, a33 = 9.0e6, a44 = 2.25e6, a66 = 2.7e6) are
    checked on the way; two sampled solves are the oracle's again."""
    g = load_cache_golden("homogeneous_vti_cache_M90.txt")
    L = inputs.homogeneous_vti().layers[0]
    a = co.moduli_from_thomsen(L.vp0, L.vs0, L.eps, L.delta, L.gamma, L.qp, L.qs)
    assert np.allclose(np.real(a), [1.26e7, 5.3468744e6, 9.0e6, 2.25e6, 2.7e6], rtol=1e-8)
    assert len(g["folded"]) == 3 and all(len(v) == 91 for v in g["folded"].values())
    a11, a13, a33, a44, a66 = a
    for mode, along, across in (("qP", a33, a11), ("qSV", a44, a44), ("qSH", a44, a66)):
        for j, c2 in ((0, along), (90, across)):
            s = g["folded"][(mode, 0)][j]
            c = np.sqrt(complex(c2))
            assert s["flag"] == 0 and abs(s["vartheta"]) < 1e-13
            assert math.isclose(s["V"], 1 / (1 / c).real, rel_tol=1e-12)
            assert math.isclose(s["A"], (1 / c).imag, rel_tol=1e-12)
            assert math.isclose(s["Q"], -complex(c2).real / complex(c2).imag, rel_tol=1e-12)
            r = s["r"][[0, 2]]
            assert np.allclose(r, [0.0, 1.0] if j == 0 else [1.0, 0.0], atol=1e-12)
    _resolve(g, [a], [("qP", 0, 37), ("qSV", 0, 52)])
