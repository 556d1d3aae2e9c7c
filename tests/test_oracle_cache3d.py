"""Pins of the oracle's 3D cache (Eq. 35) against facts that do not come from
its own 3D code: the 2D TTI cache (Eq. 36, a separate mirroring and rotation
path) in the plane that holds the symmetry axis, rotation about the vertical,
azimuthal isotropy of VTI, and the isotropic closed form.  CPU only."""
import math

import numpy as np
import pytest

from oracle import cache_oracle as co

DEG = math.pi / 180.0
H = 0.05 * DEG
K = 600
MOD = co.moduli_from_thomsen(3000.0, 1600.0, 0.2, 0.08, 0.12, 60.0, 30.0)


@pytest.mark.parametrize("mode", ["qP", "qSV", "qSH"])
def test_axis_plane_matches_2d_tti_cache(mode):
    """phi_0 = 0: the directions of azimuth 0 and 180 deg lie in the x-z plane,
    where the 2D TTI cache holds the same entries (ray with ry = 0)."""
    theta0 = 15 * DEG
    n_az, n_pol = 8, 6                      # polar 15, 45, ..., 165 deg
    c3 = co.build_cache_3d([MOD], [theta0], [0.0], [mode], n_az, n_pol, "MEV", H, K)
    c2 = co.build_cache([MOD], [theta0], [mode], 3, "MEV", H, K)   # local angles every 30 deg
    for i in range(n_pol):
        th = (i + 0.5) * 180.0 / n_pol
        for j, glob in ((0, th), (n_az // 2, -th)):          # 2D angle from +z toward +x
            d3 = i * n_az + j
            d2 = int(round(((glob - 15.0) % 360.0) / 30.0)) % 12
            assert c3["flag"][0, 0, d3] == c2["flag"][0, 0, d2]
            if c2["flag"][0, 0, d2]:
                continue
            for key in ("V", "A", "Q"):
                assert c3[key][0, 0, d3] == pytest.approx(c2[key][0, 0, d2], rel=1e-12)
            assert c3["rx"][0, 0, d3] == pytest.approx(c2["rx"][0, 0, d2], abs=1e-12)
            assert c3["rz"][0, 0, d3] == pytest.approx(c2["rz"][0, 0, d2], abs=1e-12)
            assert abs(c3["ry"][0, 0, d3]) < 1e-12


def test_rotation_about_vertical():
    """Turning the symmetry axis by 90 deg about z turns every entry with it."""
    n_az, n_pol = 8, 4
    a = co.build_cache_3d([MOD], [35 * DEG], [0.0], ["qP", "qSV"], n_az, n_pol, "MEV", H, K)
    b = co.build_cache_3d([MOD], [35 * DEG], [90 * DEG], ["qP", "qSV"], n_az, n_pol, "MEV", H, K)
    for i in range(n_pol):
        for j in range(n_az):
            da, db = i * n_az + j, i * n_az + (j + n_az // 4) % n_az
            for key in ("V", "A", "flag"):
                assert np.allclose(a[key][:, 0, da], b[key][:, 0, db], rtol=1e-12, equal_nan=True)
            ok = a["flag"][:, 0, da] == 0
            assert np.allclose(-a["ry"][ok, 0, da], b["rx"][ok, 0, db], atol=1e-12)
            assert np.allclose(a["rx"][ok, 0, da], b["ry"][ok, 0, db], atol=1e-12)
            assert np.allclose(a["rz"][ok, 0, da], b["rz"][ok, 0, db], atol=1e-12)


def test_vti_is_azimuthally_isotropic():
    n_az, n_pol = 6, 4
    c = co.build_cache_3d([MOD], [0.0], [0.0], ["qP", "qSH"], n_az, n_pol, "MEV", H, K)
    for i in range(n_pol):
        row = slice(i * n_az, (i + 1) * n_az)
        for key in ("V", "A"):
            assert np.allclose(c[key][:, 0, row], c[key][:, 0, row][:, :1], rtol=1e-12)
        phi = np.arctan2(c["ry"][:, 0, row], c["rx"][:, 0, row])
        want = np.arange(n_az) * 2 * math.pi / n_az
        assert np.allclose(np.angle(np.exp(1j * (phi - want[None]))), 0.0, atol=1e-12)


def test_isotropic_rays_follow_slowness():
    a33, a44 = 9.0e6 * (1 - 1j / 50), 2.25e6 * (1 - 1j / 30)
    iso = np.array([a33, a33 - 2 * a44, a33, a44, a44])
    n_az, n_pol = 5, 3
    c = co.build_cache_3d([iso], [0.7], [1.1], ["qP", "qSV"], n_az, n_pol, "OEV", H, K)
    for d in range(n_az * n_pol):
        th, ph = c["theta"][0, 0, d], c["phi"][0, 0, d]
        n = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        for mi, a in enumerate([a33, a44]):
            r = np.array([c["rx"][mi, 0, d], c["ry"][mi, 0, d], c["rz"][mi, 0, d]])
            assert np.allclose(r, n, atol=1e-10)
            assert c["V"][mi, 0, d] == pytest.approx(1 / (1 / np.sqrt(a)).real, rel=1e-10)
