"""The library's FP64 set-up arithmetic (host only, no GPU) against the oracle.

The two compute the same definitions by different routes: the library uses
closed forms (K[k,l] = 1 - 2[l < k, k + l odd], Mhat = diag(1/(2k+1))),
Gauss-Jordan inversion, and exact polynomial algebra for the transfer
matrices (up to p_t = 10; at p_t = 20 the three-term recurrence in the
Legendre basis); the oracle uses long-double quadrature of the definitions and
Gaussian elimination.  Tolerances are a few ulps of the entries: cond(A) <= 21
at p_t <= 10 and <= 41 at p_t = 20 for every z >= 0.
"""
import numpy as np
import pytest

import oracle as O
from paper_1409_5254_gb300 import tmg

PS = [0, 1, 2, 3, 4, 5, 10, 20]
ZS = [0.0, 1e-6, 1e-3, 0.7, 3.0, 50.0, 1e4]
EPS = np.finfo(float).eps


@pytest.mark.parametrize("p", PS)
@pytest.mark.parametrize("z", ZS)
def test_level_constants_match_the_oracle(p, z):
    L = tmg.level_constants(p, z)
    K, M, a, b = O.blocks(p)
    A = K + z * M
    d = p + 1
    # A: z/(2k+1) is one rounding in the library, two in the oracle
    assert np.abs(L["A"] - A).max() <= 4 * EPS * np.abs(A).max()
    assert np.abs(L["Ainv"] @ A - np.eye(d)).max() <= 64 * EPS
    g = np.linalg.solve(A, a)
    c = np.linalg.solve(A.T, b)
    assert np.abs(L["g"] - g).max() <= 64 * EPS * np.abs(g).max()
    assert np.abs(L["c"] - c).max() <= 64 * EPS * np.abs(c).max()
    # alpha = b^T A^{-1} a: the oracle's (Lemma chap4_theorem2), a difference of O(1) terms
    assert L["alpha"] == pytest.approx(O.alpha(p, z), rel=1e-13, abs=64 * EPS)
    assert L["omega"] == pytest.approx(O.omega_star(p, z), rel=1e-13)


@pytest.mark.parametrize("omega", [0.5, 1.0, 1.5])
def test_user_damping_overrides_omega_star(omega):
    assert tmg.level_constants(1, 0.3, omega)["omega"] == omega


@pytest.mark.parametrize("p", PS)
def test_transfer_matrices_match_the_oracle(p):
    P1, P2 = tmg.transfer_matrices(p)
    Q1, Q2 = O.transfer(p)
    assert np.abs(P1 - Q1).max() <= 4 * EPS and np.abs(P2 - Q2).max() <= 4 * EPS


def test_unbuilt_and_invalid_degrees():
    for p in (6, 9, 11, 19):
        with pytest.raises(tmg.TmgError) as e:
            tmg.transfer_matrices(p)
        assert e.value.status == tmg.TMG_EUNSUPPORTED
    for p, z in ((21, 1.0), (-1, 1.0), (1, -1.0), (1, float("nan"))):
        with pytest.raises(tmg.TmgError) as e:
            tmg.level_constants(p, z)
        assert e.value.status == tmg.TMG_EINVAL
