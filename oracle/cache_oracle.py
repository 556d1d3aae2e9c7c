"""FP64 oracle of the directional cache C(m, k, theta) -- TEST INFRASTRUCTURE ONLY.

Only tests, the smoke check and the benchmark's CPU-baseline leg may call this.
It is a plain restatement of the paper's local kernel, written for reading
against the equations, not for speed:

* Eq. 2        complex density-normalised moduli a = a^R - i a^I, with the
               per-component reading a^I_pq = a^R_pq / Q_pq (Table 2 lists a
               quality factor beside each modulus).
* Eq. 4-7      Christoffel matrix of the complex slowness direction
               n = (sin(theta + i vartheta), 0, cos(theta + i vartheta)), built
               from the full 4th-order tensor and diagonalised with
               numpy.linalg.eig (no closed form); in this sagittal plane the
               y-polarised block and the x-z block are solved separately.
* Eq. 12       OEV: v_i = a_ijkl p_l g_j g_k with the bilinear norm g.g = 1.
* Eq. 13-14    MEV, read literally: unsymmetrised Gbar_il = a_ijkl g*_j g_k with
               g^H g = 1, plus 1/2 g^H [Gamma(p) - I] dg/dp where dg/dp comes
               from first-order eigenvector perturbation theory.
* Eq. 9        homogeneity: the residual f = (v^R x v^I)_y / |v^R|^2 vanishes.
               Roots are the sign changes of f on the uniform grid
               vartheta_k = k h, |k| <= K (default h = 0.001 deg, K = 30000, i.e.
               the [-30 deg, 30 deg] bracket the paper gives to fminbnd), plus
               exact zeros on the grid, each polished by bisection to 1e-14 rad.
               The acceptable root is the decaying one (A >= -1e-9 / V) of least
               |vartheta|; a tie goes to the negative root; no acceptable root
               flags the entry.
* Eq. 10-11    ray velocity, attenuation and Q of the homogeneous energy velocity.
* Eq. 26, 36   cache over the slowness angles theta_d = d * (pi/2)/M of the local
               symmetry-axis frame, d < 4M; the solve runs at the angle folded
               into [0, pi/2] (the 0-90 deg TI range) and the ray direction is
               mirrored back, then rotated by the tilt theta_0.
* Eq. 35       3D cache over global slowness directions (polar (i + 1/2) pi/n_pol,
               azimuth j 2 pi/n_az): each direction is expressed in the local
               frame (e_x', e_y', e_z') of the class's symmetry axis (theta_0,
               phi_0); VTI is rotationally symmetric about e_z', so the solve is
               the sagittal-plane one at the local polar angle folded into
               [0, pi/2], and its ray is turned to the local azimuth, mirrored
               back and expressed in the global frame.
"""
from __future__ import annotations

import math

import numpy as np

MODES = ("qP", "qSV", "qSH")
ACCEPT_TOL = 1e-9          # a root is decaying when -v_I / v_R >= -ACCEPT_TOL
POLISH_TOL = 1e-14         # bisection stops at this bracket width (rad)
DEG = math.pi / 180.0


# ----------------------------------------------------------------- moduli (Eq. 2)
def moduli_from_table(aR, q) -> np.ndarray:
    """Eq. 2: a = a^R - i a^R/Q per Voigt component (a11, a13, a33, a44, a66)."""
    aR = np.asarray(aR, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    aI = np.where(np.isinf(q), 0.0, aR / q)
    return aR - 1j * aI


def moduli_from_thomsen(vp0, vs0, eps, delta, gamma, qp, qs) -> np.ndarray:
    """Invert Thomsen's (1986) definitions for a VTI solid, then apply Eq. 2 with
    Q11 = Q13 = Q33 = Qp and Q44 = Q66 = Qs."""
    a33 = vp0 * vp0
    a44 = vs0 * vs0
    a11 = a33 * (1.0 + 2.0 * eps)
    a66 = a44 * (1.0 + 2.0 * gamma)
    radicand = (a33 - a44) * (a33 * (1.0 + 2.0 * delta) - a44)
    if not radicand > 0.0:
        raise ValueError("Thomsen delta gives no real a13")
    a13 = math.sqrt(radicand) - a44
    return moduli_from_table([a11, a13, a33, a44, a66], [qp, qp, qp, qs, qs])


def stiffness_tensor(a5) -> np.ndarray:
    """Full a_ijkl (3x3x3x3, complex) of a VTI solid with its axis along z."""
    a11, a13, a33, a44, a66 = [complex(x) for x in a5]
    C = np.zeros((6, 6), dtype=np.complex128)
    C[0, 0] = C[1, 1] = a11
    C[2, 2] = a33
    C[0, 1] = C[1, 0] = a11 - 2.0 * a66
    C[0, 2] = C[2, 0] = C[1, 2] = C[2, 1] = a13
    C[3, 3] = C[4, 4] = a44
    C[5, 5] = a66
    voigt = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (1, 2): 3, (2, 1): 3,
             (0, 2): 4, (2, 0): 4, (0, 1): 5, (1, 0): 5}
    A = np.zeros((3, 3, 3, 3), dtype=np.complex128)
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    A[i, j, k, l] = C[voigt[(i, j)], voigt[(k, l)]]
    return A


# ------------------------------------------------------------ kernel (Eq. 4-14)
def slowness_direction(theta, vartheta) -> np.ndarray:
    """Eq. 7: n = (sin(theta + i vartheta), 0, cos(theta + i vartheta))."""
    z = np.asarray(theta, dtype=np.float64) + 1j * np.asarray(vartheta, dtype=np.float64)
    return np.stack([np.sin(z), np.zeros_like(z), np.cos(z)], axis=-1)


def christoffel(A, x) -> np.ndarray:
    """Eq. 4: Gamma_jk = a_ijkl x_i x_l for a batch of vectors x[..., 3]."""
    return np.einsum("ijkl,...i,...l->...jk", A, x, x)


def eigenpairs(G):
    """Eigenvalues w[..., 3] and eigenvectors V[..., :, 3] of Christoffel matrices.

    With n_y = 0 (the sagittal plane of Eq. 7) the y row and column of Gamma
    are exactly zero off the diagonal: the y-polarised mode (qSH) decouples from
    the x-z block.  The two blocks are then diagonalised separately, so that
    qSH stays y-polarised even where it is degenerate with qSV (on the
    symmetry axis) and numpy.linalg.eig would mix the two."""
    decoupled = not (np.any(G[..., 0, 1] != 0) or np.any(G[..., 1, 0] != 0)
                     or np.any(G[..., 1, 2] != 0) or np.any(G[..., 2, 1] != 0))
    if not decoupled:
        return np.linalg.eig(G)
    xz = G[..., [0, 2], :][..., :, [0, 2]]
    w2, V2 = np.linalg.eig(xz)
    w = np.concatenate([w2, G[..., 1, 1][..., None]], axis=-1)
    V = np.zeros(G.shape, dtype=np.complex128)
    V[..., 0, :2] = V2[..., 0, :]
    V[..., 2, :2] = V2[..., 1, :]
    V[..., 1, 2] = 1.0
    return w, V


def _mode_column(w, V, mode):
    """Index of the eigenpair of wave mode ``mode`` for each batch element.

    qSH is the y-polarised eigenvector; of the two x-z polarised ones, qP has
    the larger real eigenvalue and qSV the smaller."""
    ypol = np.abs(V[..., 1, :])                       # [..., 3]
    sh = np.argmax(ypol, axis=-1)
    if mode == "qSH":
        return sh
    wr = np.where(np.arange(3) == sh[..., None], np.nan, w.real)
    hi = np.nanargmax(wr, axis=-1)
    lo = np.nanargmin(wr, axis=-1)
    return hi if mode == "qP" else lo


def energy_velocity(A, n, mode, kernel) -> np.ndarray:
    """Complex energy velocity v[..., 3] for slowness directions n[..., 3].

    OEV is Eq. 12; MEV is the literal form of Eq. 13-14 (module docstring)."""
    G = christoffel(A, n)
    w, V = eigenpairs(G)
    col = _mode_column(w, V, mode)
    take = lambda arr: np.take_along_axis(arr, col[..., None], axis=-1)[..., 0]
    lam = take(w)                                     # eigenvalue c^2
    g = np.take_along_axis(V, col[..., None, None], axis=-1)[..., 0]   # [...,3]
    c = np.sqrt(lam)                                  # principal: Re c >= 0
    p = n / c[..., None]                              # Eq. 5
    if kernel == "OEV":
        gb = g / np.sqrt(np.sum(g * g, axis=-1))[..., None]           # g.g = 1
        return np.einsum("ijkl,...l,...j,...k->...i", A, p, gb, gb)
    if kernel != "MEV":
        raise ValueError(kernel)
    g = g / np.sqrt(np.sum(np.conj(g) * g, axis=-1).real)[..., None]  # g^H g = 1
    gs = np.conj(g)
    Gbar = np.einsum("ijkl,...j,...k->...il", A, gs, g)
    v = np.einsum("...il,...l->...i", Gbar, p)
    Gp_minus_I = christoffel(A, p) - np.eye(3)
    dG = (np.einsum("ijkl,...l->...ijk", A, p)
          + np.einsum("mjki,...m->...ijk", A, p))     # dGamma_jk / dp_i
    for q in range(3):
        other = col != q
        h = V[..., :, q]
        mu = w[..., q] / lam                          # eigenvalue of Gamma(p)
        hTh = np.sum(h * h, axis=-1)
        s = np.einsum("...j,...ijk,...k->...i", h, dG, g)          # h^T dGamma_i g
        t = np.einsum("...j,...jk,...k->...", gs, Gp_minus_I, h)   # g^H (Gamma-I) h
        with np.errstate(divide="ignore", invalid="ignore"):
            term = 0.5 * (t / ((1.0 - mu) * hTh))[..., None] * s
        # (Gamma(p) - I) h = (mu - 1) h, so the term carries the factor g^H h:
        # a mode orthogonal to g (qSH against the x-z modes in the sagittal
        # plane) or one that dGamma does not couple to g adds exactly nothing,
        # even where it is degenerate with g and the quotient reads 0/0
        coupled = np.any(s != 0, axis=-1) & (np.sum(gs * h, axis=-1) != 0)
        v = v + np.where((other & coupled)[..., None], term, 0.0)
    return v


def residual(v) -> np.ndarray:
    """Homogeneity residual (Eq. 9): f = (v^R_x v^I_z - v^R_z v^I_x) / |v^R|^2."""
    vR, vI = v.real, v.imag
    return (vR[..., 0] * vI[..., 2] - vR[..., 2] * vI[..., 0]) / np.sum(vR * vR, axis=-1)


def ray_quantities(v):
    """Eq. 10-11 for a homogeneous v: ray direction r = v^R/|v^R|,
    v_R = |v^R|, v_I = v^I . r, V = (v_R^2+v_I^2)/v_R, A = -v_I/(v_R^2+v_I^2),
    Q = -Re(v^2)/Im(v^2) with v = v_R + i v_I (Q = inf when v_I = 0)."""
    vR, vI = v.real, v.imag
    vr = np.sqrt(np.sum(vR * vR, axis=-1))
    r = vR / vr[..., None]
    vi = np.sum(vI * r, axis=-1)
    mag2 = vr * vr + vi * vi
    V = mag2 / vr
    A = -vi / mag2
    with np.errstate(divide="ignore"):
        Q = np.where(vi == 0.0, np.inf, -(vr * vr - vi * vi) / (2.0 * vr * vi))
    return V, A, Q, r, vr, vi


def solve_direction(A, theta, mode, kernel, h=0.001 * DEG, K=30000):
    """Homogeneity search at one real slowness angle ``theta`` (Eq. 9).

    Returns a dict with vartheta, V, A, Q, r (3,), flag (0 ok / 1 no acceptable
    root) and the list of all polished roots."""
    vts = np.arange(-K, K + 1, dtype=np.float64) * h
    fk = residual(energy_velocity(A, slowness_direction(theta, vts), mode, kernel))

    def f_at(x):
        return residual(energy_velocity(A, slowness_direction(theta, x), mode, kernel))

    brk = np.nonzero(fk[:-1] * fk[1:] < 0.0)[0]
    lo, hi, flo = vts[brk].copy(), vts[brk + 1].copy(), fk[brk].copy()
    active = np.ones(lo.shape, dtype=bool)
    while active.any():                               # bisection polish
        mid = 0.5 * (lo + hi)
        done = (hi - lo <= POLISH_TOL) | (mid == lo) | (mid == hi)
        active &= ~done
        if not active.any():
            break
        fm = f_at(mid[active])
        same = np.signbit(fm) == np.signbit(flo[active])
        idx = np.nonzero(active)[0]
        lo[idx[same]] = mid[active][same]
        flo[idx[same]] = fm[same]
        hi[idx[~same]] = mid[active][~same]
    roots = np.concatenate([0.5 * (lo + hi), vts[fk == 0.0]])
    if roots.size == 0:
        return dict(vartheta=np.nan, V=np.nan, A=np.nan, Q=np.nan, r=np.full(3, np.nan),
                    flag=1, roots=roots)
    v = energy_velocity(A, slowness_direction(theta, roots), mode, kernel)
    V, Aatt, Q, r, vr, vi = ray_quantities(v)
    ok = (-vi / vr) >= -ACCEPT_TOL
    if not ok.any():
        return dict(vartheta=np.nan, V=np.nan, A=np.nan, Q=np.nan, r=np.full(3, np.nan),
                    flag=1, roots=roots)
    cand = np.nonzero(ok)[0]
    # least |vartheta|; on an exact tie the negative root wins
    best = min(cand, key=lambda i: (abs(roots[i]), 0 if roots[i] < 0 else 1))
    return dict(vartheta=roots[best], V=V[best], A=max(Aatt[best], 0.0), Q=Q[best],
                r=r[best], flag=0, roots=roots)


# --------------------------------------------------------------- cache (Eq. 26)
def folded_solves(A, mode, M, kernel="MEV", h=0.001 * DEG, K=30000):
    """The M+1 solves of one (mode, class) at the folded slowness angles
    theta_j = j*(pi/2)/M, j = 0..M (the 0-90 deg TI range of Eq. 26)."""
    return [solve_direction(A, (math.pi / 2) * j / M, mode, kernel, h, K) for j in range(M + 1)]


def assemble_cache(folded, tilts, M):
    """Cache arrays [n_modes, n_classes, 4M] from folded solves.

    folded[mi][k] is the list of M+1 solve dicts of mode slot mi and class k
    (keys V, A, Q, r, vartheta, flag).  Direction d of the local frame is the
    slowness angle theta_d = d*(pi/2)/M; it takes the solve at its folded
    angle, with the ray direction mirrored into the quadrant of theta_d and
    rotated by the tilt theta_0 (Eq. 36).  Returns V, A, Q, rx, rz, theta
    (global slowness angle, from +z toward +x), vartheta (signed as seen from
    that direction) and flag."""
    tilts = np.asarray(tilts, dtype=np.float64).reshape(-1)
    nm, nk, nd = len(folded), len(folded[0]), 4 * M
    out = {key: np.zeros((nm, nk, nd)) for key in ("V", "A", "Q", "rx", "rz", "theta", "vartheta")}
    out["flag"] = np.zeros((nm, nk, nd), dtype=np.uint8)
    signs = [(1.0, 1.0), (1.0, -1.0), (-1.0, -1.0), (-1.0, 1.0)]
    for mi in range(nm):
        for k in range(nk):
            ct, st = math.cos(tilts[k]), math.sin(tilts[k])
            for d in range(nd):
                quad, rem = divmod(d, M)
                j = rem if quad in (0, 2) else M - rem
                sx, sz = signs[quad]
                s = folded[mi][k][j]
                lx, lz = sx * s["r"][0], sz * s["r"][2]
                out["rx"][mi, k, d] = lx * ct + lz * st          # Eq. 36
                out["rz"][mi, k, d] = -lx * st + lz * ct
                out["V"][mi, k, d] = s["V"]
                out["A"][mi, k, d] = s["A"]
                out["Q"][mi, k, d] = s["Q"]
                out["vartheta"][mi, k, d] = s["vartheta"] * sx * sz
                out["theta"][mi, k, d] = (math.pi / 2) * d / M + tilts[k]
                out["flag"][mi, k, d] = s["flag"]
    return out


def build_cache(moduli, tilts, modes, M, kernel="MEV", h=0.001 * DEG, K=30000):
    """Directional cache for classes ``moduli`` [n_classes, 5] (complex) with
    tilts theta_0 [n_classes] (rad), wave modes ``modes`` (names from MODES) and
    M slowness angles per quadrant: the folded solves of every (mode, class),
    assembled by ``assemble_cache`` (arrays shaped [n_modes, n_classes, 4M])."""
    moduli = np.asarray(moduli, dtype=np.complex128).reshape(-1, 5)
    folded = [[folded_solves(stiffness_tensor(moduli[k]), mode, M, kernel, h, K) for k in range(moduli.shape[0])]
              for mode in modes]
    return assemble_cache(folded, tilts, M)


def local_basis(theta0, phi0):
    """Rows e_x', e_y', e_z' of the local symmetry-axis frame (Eq. 35)."""
    ct, st, cp, sp = math.cos(theta0), math.sin(theta0), math.cos(phi0), math.sin(phi0)
    return np.array([[ct * cp, ct * sp, -st],
                     [-sp, cp, 0.0],
                     [st * cp, st * sp, ct]])


def solve_direction_3d(A, theta0, phi0, th, ph, mode, kernel="MEV", h=0.001 * DEG, K=30000):
    """One 3D entry: the global slowness direction of polar angle ``th`` and
    azimuth ``ph``, for the class with stiffness ``A`` and symmetry axis
    (theta0, phi0).  Returns (solve dict, global ray (3,), z mirror sign)."""
    E = local_basis(theta0, phi0)
    n = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    nl = E @ n                                   # components along e_x', e_y', e_z'
    th_l = math.acos(min(1.0, max(-1.0, nl[2])))
    ph_l = math.atan2(nl[1], nl[0])
    sz = 1.0 if th_l <= math.pi / 2 else -1.0
    th_f = th_l if sz > 0 else math.pi - th_l
    s = solve_direction(A, th_f, mode, kernel, h, K)
    rs, rzl = s["r"][0], s["r"][2]
    rl = np.array([rs * math.cos(ph_l), rs * math.sin(ph_l), sz * rzl])
    return s, E.T @ rl, sz


def build_cache_3d(moduli, tilts, azims, modes, n_az, n_pol, kernel="MEV", h=0.001 * DEG, K=30000):
    """3D directional cache for classes ``moduli`` [n_classes, 5] with symmetry
    axes (tilts theta_0, azims phi_0).  Entry d = i*n_az + j is the global
    slowness direction of polar angle (i + 1/2) pi/n_pol and azimuth j 2 pi/n_az.

    Returns arrays [n_modes, n_classes, n_pol*n_az]: V, A, Q, rx, ry, rz,
    theta (polar), phi (azimuth), vartheta (as solved, times the z mirror sign),
    flag."""
    moduli = np.asarray(moduli, dtype=np.complex128).reshape(-1, 5)
    tilts = np.asarray(tilts, dtype=np.float64).reshape(-1)
    azims = np.asarray(azims, dtype=np.float64).reshape(-1)
    nm, nk, nd = len(modes), moduli.shape[0], n_az * n_pol
    out = {key: np.zeros((nm, nk, nd)) for key in ("V", "A", "Q", "rx", "ry", "rz", "theta", "phi", "vartheta")}
    out["flag"] = np.zeros((nm, nk, nd), dtype=np.uint8)
    for mi, mode in enumerate(modes):
        for k in range(nk):
            A = stiffness_tensor(moduli[k])
            for i in range(n_pol):
                th = (i + 0.5) * math.pi / n_pol
                for j in range(n_az):
                    ph = j * 2.0 * math.pi / n_az
                    d = i * n_az + j
                    s, r, sz = solve_direction_3d(A, tilts[k], azims[k], th, ph, mode, kernel, h, K)
                    out["rx"][mi, k, d], out["ry"][mi, k, d], out["rz"][mi, k, d] = r
                    out["V"][mi, k, d] = s["V"]
                    out["A"][mi, k, d] = s["A"]
                    out["Q"][mi, k, d] = s["Q"]
                    out["vartheta"][mi, k, d] = s["vartheta"] * sz
                    out["theta"][mi, k, d] = th
                    out["phi"][mi, k, d] = ph
                    out["flag"][mi, k, d] = s["flag"]
    return out
