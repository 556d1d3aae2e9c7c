"""Pins of the angular-coverage oracle (oracle/coverage_oracle.py): closed
forms and hand-built caches whose coverage, branch and missing-angle counts
are known without running the oracle's own arithmetic."""
import math

import numpy as np

from oracle import coverage_oracle as cov
from paper_2609_26108_b300 import inputs

from helpers import golden_cache, load_cache_golden

DEG = math.pi / 180


def synthetic(psi_deg, V, valid=None):
    """A one-mode, one-class cache whose entries have ray angles psi (deg,
    measured from +z toward +x) and velocities V."""
    psi = np.radians(np.asarray(psi_deg, np.float64))
    n = len(psi)
    c = {"rx": np.sin(psi)[None, None], "rz": np.cos(psi)[None, None],
         "V": np.asarray(V, np.float64)[None, None], "A": np.full((1, 1, n), 1e-5)}
    c["flag"] = (np.zeros((1, 1, n), np.uint8) if valid is None
                 else (~np.asarray(valid, bool)).astype(np.uint8)[None, None])
    return c


def isotropic(M):
    """Ray = slowness direction at theta_e = e (pi/2) / M, e = 0..4M-1."""
    return synthetic(np.arange(4 * M) * 90.0 / M, np.full(4 * M, 3000.0))


def test_isotropic_cache_covers_every_stencil_direction():
    off = inputs.stencil_2d(5)
    for M in (2, 6, 90):          # M = 1: adjacent rays 90 deg apart bracket nothing
        covd, mis, miss = cov.coverage_counts(isotropic(M), off)
        assert covd[0, 0] == len(off) and mis[0, 0] == 0 and miss[0, 0] == 0
        covd32, mis32, _ = cov.coverage_counts(isotropic(M), off, dtype=np.float32)
        assert covd32[0, 0] == len(off) and mis32[0, 0] == 0


def test_invalid_entry_leaves_its_direction_uncovered():
    """M = 90: entry 90 is the ray along +x.  With it invalid, no adjacent
    valid pair holds the direction (1, 0): exactly that one stencil
    direction of the 80 is uncovered; a hole between two stencil directions
    uncovers none."""
    M = 90
    off = inputs.stencil_2d(5)
    c = isotropic(M)
    c["flag"][0, 0, M] = 1
    covd, mis, _ = cov.coverage_counts(c, off)
    assert covd[0, 0] == len(off) - 1 and mis[0, 0] == 0
    c = isotropic(M)
    c["flag"][0, 0, 50] = 1              # 50 deg: between the stencil's 45 deg and 51.3 deg
    covd, _, _ = cov.coverage_counts(c, off)
    assert covd[0, 0] == len(off)
    # two adjacent valid entries more than 90 degrees apart bracket nothing
    c = synthetic([0.0, 100.0, 200.0, 300.0], [1.0] * 4)
    covd, _, _ = cov.coverage_counts(c, np.array([[1, 0, 1]]))
    assert covd[0, 0] == 0


# Ray angles of a folded (triplicated) branch around the stencil direction
# (3, 4): atan2(3, 4) = 36.87 deg.  Entries 5-6, 6-7 and 9-10 bracket it:
# branch A (36.0 -> 36.9), the backward branch B (36.9 -> 33.0) and branch
# C (36.5 -> 38.0).
FOLD_PSI = [0.0, 10.0, 20.0, 30.0, 35.0, 36.0, 36.9, 33.0, 34.0, 36.5, 38.0, 45.0, 90.0, 135.0, 180.0,
            225.0, 270.0, 315.0, 330.0, 345.0]


def test_fold_branch_mismatch():
    off = np.array([[3, 0, 4]])
    # C fastest: the lookup's nearest entry is 6 (36.9 deg), on A/B -> mismatch
    V = [1.0] * len(FOLD_PSI)
    V[9] = V[10] = 1.2
    V[7] = 0.9
    covd, mis, _ = cov.coverage_counts(synthetic(FOLD_PSI, V), off)
    assert covd[0, 0] == 1 and mis[0, 0] == 1
    # A fastest: entry 6 ends the first-arrival bracket -> no mismatch
    V = [1.0] * len(FOLD_PSI)
    V[5] = V[6] = 1.3
    covd, mis, _ = cov.coverage_counts(synthetic(FOLD_PSI, V), off)
    assert covd[0, 0] == 1 and mis[0, 0] == 0
    # brackets listed in order with their interpolated velocity at d
    d = (0.6, 0.8)
    psi = np.radians(FOLD_PSI)
    br = cov.brackets(np.sin(psi), np.cos(psi), np.array(V, float), np.ones(len(psi), bool), *d)
    assert [e for e, _ in br] == [5, 6, 9]
    assert br[0][1] == 1.3 and br[2][1] == 1.0
    assert 1.0 < br[1][1] < 1.3                  # between V[6] = 1.3 and V[7] = 1.0


def test_missing_angles_against_a_reference():
    c = isotropic(6)
    truth = c["flag"].copy()
    c["flag"][0, 0, [3, 4, 17]] = 1
    truth[0, 0, 17] = 1                          # also invalid in the reference: not missing
    _, _, miss = cov.coverage_counts(c, inputs.stencil_2d(2), truth_flag=truth)
    assert miss[0, 0] == 2


def test_layered_tti_qp_qsh_full_coverage_no_mismatch():
    """The oracle's cache of the layered visco-TTI model at 1 deg
    (tests/golden): qP and qSH ray surfaces are convex, so every stencil
    direction is covered, with no fold to pick a wrong branch from."""
    g = load_cache_golden("layered_tti_cache_M90.txt")
    c = golden_cache(g, ["qP", "qSH"], 8, g["tilts"])
    off = inputs.stencil_2d(5)
    covd, mis, _ = cov.coverage_counts(c, off)
    assert np.all(covd == len(off)) and np.all(mis == 0)
