"""Pins of the FP64 cache oracle against facts that do not come from the oracle:
Thomsen's forward definitions, closed forms (isotropic, elastic VTI group
velocity, viscoelastic qSH ellipse), limits, symmetries and the paper's printed
values.  CPU only."""
import math
import os

import numpy as np
import pytest

from oracle import cache_oracle as co
from paper_2609_26108_b300 import inputs

DEG = math.pi / 180.0
H = 0.01 * DEG       # coarser scan step keeps these tests fast
K = 3000             # still the [-30, 30] deg bracket
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_table2():
    rows = np.loadtxt(os.path.join(GOLDEN, "table2_layers.txt"))
    return rows[:, 1:6] * 1e6, rows[:, 6:11]


def test_thomsen_roundtrip_forward_definitions():
    # Thomsen (1986): eps = (c11-c33)/(2c33), gamma = (c66-c44)/(2c44),
    # delta = ((c13+c44)^2 - (c33-c44)^2) / (2 c33 (c33-c44)).
    for vp0, vs0, eps, delta, gamma in [(3000, 1500, 0.2, 0.1, 0.1), (2500, 1300, 0.05, -0.1, 0.0),
                                        (4400, 2300, 0.3, 0.2, 0.2)]:
        a = co.moduli_from_thomsen(vp0, vs0, eps, delta, gamma, 60.0, 30.0).real
        a11, a13, a33, a44, a66 = a
        assert a33 == pytest.approx(vp0 ** 2, rel=1e-15)
        assert a44 == pytest.approx(vs0 ** 2, rel=1e-15)
        assert (a11 - a33) / (2 * a33) == pytest.approx(eps, rel=1e-13)
        assert (a66 - a44) / (2 * a44) == pytest.approx(gamma, abs=1e-13)
        d = ((a13 + a44) ** 2 - (a33 - a44) ** 2) / (2 * a33 * (a33 - a44))
        assert d == pytest.approx(delta, abs=1e-12)


def test_thomsen_quality_factor_mapping():
    a = co.moduli_from_thomsen(3000, 1500, 0.2, 0.1, 0.1, 60.0, 30.0)
    q = a.real / (-a.imag)
    assert np.allclose(q, [60, 60, 60, 30, 30], rtol=1e-14)


def test_table2_golden_matches_inputs_module():
    aR, q = _load_table2()
    layers = inputs.table2_layers()
    assert len(layers) == 4
    for i, L in enumerate(layers):
        assert np.allclose(L.aR, aR[i], rtol=1e-15)
        assert np.allclose(L.q, q[i], rtol=1e-15)
    a = co.moduli_from_table(aR[0], q[0])
    assert np.allclose(-a.imag * q[0], aR[0], rtol=1e-15)


def test_stiffness_tensor_symmetries():
    aR, q = _load_table2()
    A = co.stiffness_tensor(co.moduli_from_table(aR[0], q[0]))
    assert np.allclose(A, A.transpose(1, 0, 2, 3))
    assert np.allclose(A, A.transpose(0, 1, 3, 2))
    assert np.allclose(A, A.transpose(2, 3, 0, 1))
    # VTI: rotation about z leaves the tensor invariant
    phi = 0.7
    R = np.array([[math.cos(phi), -math.sin(phi), 0], [math.sin(phi), math.cos(phi), 0], [0, 0, 1]])
    Ar = np.einsum("ia,jb,kc,ld,abcd->ijkl", R, R, R, R, A)
    assert np.allclose(Ar, A, rtol=1e-13, atol=1e-3)


def _isotropic(M, mu, Qp, Qs):
    a11 = M * (1 - 1j / Qp)
    a44 = mu * (1 - 1j / Qs)
    return np.array([a11, a11 - 2 * a44, a11, a44, a44])


@pytest.mark.parametrize("kernel", ["OEV", "MEV"])
@pytest.mark.parametrize("mode", ["qP", "qSV", "qSH"])
def test_isotropic_viscoelastic_closed_form(kernel, mode):
    """Homogeneous wave: vartheta* = 0, r = n, V = 1/Re(1/c), A = Im(1/c)."""
    a = _isotropic(9.0e6, 2.25e6 * 1.0, 60.0, 30.0)
    A = co.stiffness_tensor(a)
    c = np.sqrt(a[0] if mode == "qP" else a[3])
    for th in [0.0, 0.2, 0.7, 1.1, math.pi / 2]:
        s = co.solve_direction(A, th, mode, kernel, H, K)
        assert s["flag"] == 0
        assert abs(s["vartheta"]) < 1e-10
        assert s["V"] == pytest.approx(1.0 / (1.0 / c).real, rel=1e-12)
        assert s["A"] == pytest.approx((1.0 / c).imag, rel=1e-9)
        assert np.allclose(s["r"], [math.sin(th), 0.0, math.cos(th)], atol=1e-12)


def _tsvankin_phase_velocity(a, th, mode):
    """Exact VTI phase velocity (Tsvankin 2001), analytic in theta."""
    a11, a13, a33, a44, a66 = a
    s2, c2 = np.sin(th) ** 2, np.cos(th) ** 2
    if mode == "qSH":
        return np.sqrt(a66 * s2 + a44 * c2)
    root = np.sqrt(((a11 - a44) * s2 - (a33 - a44) * c2) ** 2 + 4 * (a13 + a44) ** 2 * s2 * c2)
    sign = 1.0 if mode == "qP" else -1.0
    return np.sqrt(0.5 * ((a11 + a44) * s2 + (a33 + a44) * c2 + sign * root))


@pytest.mark.parametrize("kernel", ["OEV", "MEV"])
@pytest.mark.parametrize("mode", ["qP", "qSV", "qSH"])
def test_elastic_vti_group_velocity(kernel, mode):
    """Q -> infinity: vartheta* = 0, A = 0, and (V, ray angle) equal the textbook
    group velocity V_g = sqrt(V^2 + V'^2) at psi = theta + atan(V'/V)."""
    aR, _ = _load_table2()
    a = aR[0].astype(np.complex128)          # elastic Table 2 layer 1
    A = co.stiffness_tensor(a)
    for th in [0.1, 0.45, 0.8, 1.3]:
        hstep = 1e-30
        Vc = _tsvankin_phase_velocity(aR[0], th + 1j * hstep, mode)
        V, dV = Vc.real, Vc.imag / hstep      # complex-step derivative
        Vg = math.sqrt(V * V + dV * dV)
        psi = th + math.atan2(dV, V)
        s = co.solve_direction(A, th, mode, kernel, H, K)
        assert s["flag"] == 0
        assert abs(s["vartheta"]) < 1e-10
        assert abs(s["A"]) < 1e-15
        assert s["V"] == pytest.approx(Vg, rel=1e-11)
        assert s["r"][0] == pytest.approx(math.sin(psi), abs=1e-11)
        assert s["r"][2] == pytest.approx(math.cos(psi), abs=1e-11)


@pytest.mark.parametrize("kernel", ["OEV", "MEV"])
def test_viscoelastic_qsh_ellipse_closed_form(kernel):
    """qSH in visco-VTI with Q44 != Q66 (Table 2 layer 1): along the oracle's
    ray direction psi, the complex ray velocity s obeys
    1/s^2 = sin^2(psi)/a66 + cos^2(psi)/a44, so V = 1/Re(1/s), A = Im(1/s)."""
    aR, q = _load_table2()
    a = co.moduli_from_table(aR[0], q[0])
    A = co.stiffness_tensor(a)
    a44, a66 = a[3], a[4]
    for th in [0.15, 0.5, 0.9, 1.4]:
        s = co.solve_direction(A, th, "qSH", kernel, H, K)
        assert s["flag"] == 0 and abs(s["vartheta"]) > 1e-4      # not a trivial root
        psi = math.atan2(s["r"][0], s["r"][2])
        inv_s = np.sqrt(math.sin(psi) ** 2 / a66 + math.cos(psi) ** 2 / a44)
        assert s["V"] == pytest.approx(1.0 / inv_s.real, rel=1e-11)
        assert s["A"] == pytest.approx(inv_s.imag, rel=1e-9)


def test_attenuation_vanishes_linearly_as_q_grows():
    aR, q = _load_table2()
    out = []
    for scale in [1e2, 1e3, 1e4]:
        A = co.stiffness_tensor(co.moduli_from_table(aR[0], q[0] * scale))
        s = co.solve_direction(A, 0.6, "qP", "MEV", H, K)
        out.append(s["A"] * scale)
    # A * Q converges: successive ratios approach 1 at rate 1/Q
    assert abs(out[1] / out[0] - 1) < 2e-2
    assert abs(out[2] / out[1] - 1) < 2e-3


def test_mev_equals_oev_for_real_polarisation():
    """With a real polarisation (elastic or qSH) the g* correction vanishes."""
    aR, q = _load_table2()
    n = co.slowness_direction(np.array([0.3, 0.9]), np.array([0.01, -0.02]))
    A = co.stiffness_tensor(co.moduli_from_table(aR[0], q[0]))
    for mode in ["qSH"]:
        assert np.allclose(co.energy_velocity(A, n, mode, "MEV"), co.energy_velocity(A, n, mode, "OEV"),
                           rtol=1e-13, atol=1e-9)
    Ae = co.stiffness_tensor(aR[0].astype(complex))
    n0 = co.slowness_direction(np.array([0.3, 0.9]), np.zeros(2))
    for mode in ["qP", "qSV"]:
        assert np.allclose(co.energy_velocity(Ae, n0, mode, "MEV"), co.energy_velocity(Ae, n0, mode, "OEV"),
                           rtol=1e-12, atol=1e-6)


def test_oev_satisfies_slowness_normalisation():
    """OEV velocity obeys p.v = 1 (Euler relation of the degree-2 Hamiltonian)."""
    aR, q = _load_table2()
    A = co.stiffness_tensor(co.moduli_from_table(aR[0], q[0]))
    th = np.array([0.2, 0.7, 1.2]); vt = np.array([0.01, -0.03, 0.02])
    n = co.slowness_direction(th, vt)
    for mode in ["qP", "qSV", "qSH"]:
        G = co.christoffel(A, n)
        w, V = np.linalg.eig(G)
        v = co.energy_velocity(A, n, mode, "OEV")
        # p = n/c with c^2 the mode eigenvalue: recover c from v via p.v = 1
        lam = np.array([w[i][co._mode_column(w[i:i+1], V[i:i+1], mode)[0]] for i in range(3)])
        p = n / np.sqrt(lam)[:, None]
        assert np.allclose(np.sum(p * v, axis=1), 1.0, rtol=1e-12)


def test_cache_fold_matches_direct_solves():
    """The cache solves at the angle folded into [0, 90] deg; a direct solve in
    every quadrant must give the same V, A and the mirrored ray (VTI symmetry)."""
    aR, q = _load_table2()
    a = co.moduli_from_table(aR[1], q[1])
    M = 6
    cache = co.build_cache([a], [0.0], ["qP", "qSH"], M, "MEV", H, K)
    A = co.stiffness_tensor(a)
    for mi, mode in enumerate(["qP", "qSH"]):
        for d in [1, 7, 9, 14, 20, 23]:
            th = (math.pi / 2) * d / M
            s = co.solve_direction(A, th, mode, "MEV", H, K)
            assert cache["V"][mi, 0, d] == pytest.approx(s["V"], rel=1e-12)
            assert cache["A"][mi, 0, d] == pytest.approx(s["A"], rel=1e-9)
            assert cache["rx"][mi, 0, d] == pytest.approx(s["r"][0], abs=1e-12)
            assert cache["rz"][mi, 0, d] == pytest.approx(s["r"][2], abs=1e-12)
            assert cache["vartheta"][mi, 0, d] == pytest.approx(s["vartheta"], abs=1e-12)


def test_tilt_rotates_ray_directions():
    """Eq. 36: a tilted class is the untilted one rotated by theta_0."""
    aR, q = _load_table2()
    a = co.moduli_from_table(aR[0], q[0])
    M, tilt = 4, 0.4
    c0 = co.build_cache([a], [0.0], ["qP"], M, "MEV", H, K)
    c1 = co.build_cache([a], [tilt], ["qP"], M, "MEV", H, K)
    ang0 = np.arctan2(c0["rx"], c0["rz"])
    ang1 = np.arctan2(c1["rx"], c1["rz"])
    diff = np.angle(np.exp(1j * (ang1 - ang0 - tilt)))
    assert np.max(np.abs(diff)) < 1e-12
    assert np.allclose(c1["V"], c0["V"], rtol=1e-14)
    assert np.allclose(c1["theta"] - c0["theta"], tilt)


@pytest.mark.parametrize("kernel", ["OEV", "MEV"])
def test_paper_kernel_benchmark_qp_range(kernel):
    """Paper, local kernel benchmark (Table 2 layer 1): the imaginary slowness
    angle stays in [-2 deg, 0.5 deg]; qP is smooth and attenuating."""
    lo, hi = np.loadtxt(os.path.join(GOLDEN, "kernel_benchmark_range.txt"))
    aR, q = _load_table2()
    A = co.stiffness_tensor(co.moduli_from_table(aR[0], q[0]))
    vts, Vs = [], []
    for thd in range(0, 91, 10):
        s = co.solve_direction(A, thd * DEG, "qP", kernel, H, K)
        assert s["flag"] == 0 and s["A"] > 0
        vts.append(s["vartheta"] / DEG)
        Vs.append(s["V"])
    assert min(vts) >= lo and max(vts) <= hi
    # smooth and monotone from the symmetry axis (a11 > a33 in layer 1)
    assert np.all(np.diff(Vs) > 0)


def test_scan_bracket_and_tie_rule():
    """Selection takes the least |vartheta| acceptable root; a larger grid step
    that still brackets the same root gives the same answer."""
    aR, q = _load_table2()
    A = co.stiffness_tensor(co.moduli_from_table(aR[0], q[0]))
    s1 = co.solve_direction(A, 0.5, "qP", "MEV", 0.01 * DEG, 3000)
    s2 = co.solve_direction(A, 0.5, "qP", "MEV", 0.05 * DEG, 600)
    assert s1["vartheta"] == pytest.approx(s2["vartheta"], abs=2e-14)
    assert abs(s1["vartheta"]) <= min(abs(r) for r in s1["roots"]) + 1e-15
