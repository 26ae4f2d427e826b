"""The host polytope-distance solver of the core-set certificates
(pdscp_polytope_distance, Eq. PD of Sec. 4.2) against the oracle's brute
force over supports and its MDM solver, closed forms and the optimality
condition of Eq. PD (CPU only: the solver runs on the host)."""

import ctypes

import numpy as np
import pytest

from oracle import exact
from paper_2405_09157_gb300 import _ffi, api


def _check_weights(P, Q, dist, mu, ga):
    assert np.all(mu >= -1e-12) and np.all(ga >= -1e-12)
    assert abs(mu.sum() - 1.0) < 1e-9 and abs(ga.sum() - 1.0) < 1e-9
    z = P.T @ mu - Q.T @ ga
    assert abs(np.linalg.norm(z) - dist) <= 1e-9 * max(1.0, dist)
    return z


@pytest.mark.parametrize("seed", range(12))
def test_matches_bruteforce_on_tiny_sets(seed):
    rng = np.random.default_rng(seed)
    d = int(rng.integers(1, 4))
    P = rng.standard_normal((int(rng.integers(1, 6)), d)) + rng.uniform(0, 3)
    Q = rng.standard_normal((int(rng.integers(1, 6)), d)) - rng.uniform(0, 3)
    dist, mu, ga = api.polytope_distance(P, Q, tol=1e-14)
    ref = exact.pd_bruteforce(P, Q)
    assert abs(dist - ref[0]) <= 1e-9 * max(1.0, ref[0]), (dist, ref[0])
    _check_weights(P, Q, dist, mu, ga)


@pytest.mark.parametrize("nP,nQ,d,gap", [(300, 250, 16, 2.5), (600, 600, 128, 2.5), (40, 1000, 3, 4.0)])
def test_matches_mdm_and_is_optimal(nP, nQ, d, gap):
    rng = np.random.default_rng(nP + nQ + d)
    shift = np.zeros(d)
    shift[0] = gap
    P = rng.standard_normal((nP, d)) + shift
    Q = rng.standard_normal((nQ, d)) - shift
    dist, mu, ga = api.polytope_distance(P, Q, tol=1e-13)
    ref = exact.pd_mdm(P, Q, tol=1e-13)
    assert abs(dist - ref[0]) <= 1e-7 * ref[0], (dist, ref[0])
    z = _check_weights(P, Q, dist, mu, ga)
    # Eq. PD's optimality: the margin of z over the sets equals ||z||
    margin = (np.min(P @ z) - np.max(Q @ z)) / dist
    assert abs(margin - dist) <= 1e-6 * dist, (margin, dist)


def test_closed_forms():
    # one point each: the distance of the two points
    p, q = np.array([[1.0, 2.0, 3.0]]), np.array([[-1.0, 0.5, 2.0]])
    dist, mu, ga = api.polytope_distance(p, q)
    assert abs(dist - np.linalg.norm(p - q)) < 1e-12 and mu[0] == 1.0 and ga[0] == 1.0
    # one dimension: min P - max Q when the sets are apart
    rng = np.random.default_rng(5)
    P = rng.uniform(3.0, 5.0, (50, 1))
    Q = rng.uniform(-2.0, 1.0, (70, 1))
    dist, _, _ = api.polytope_distance(P, Q)
    assert abs(dist - (P.min() - Q.max())) < 1e-12
    # a point against a segment: distance to the segment (perpendicular foot inside)
    dist, _, ga = api.polytope_distance([[0.0, 3.0]], [[-2.0, 0.0], [2.0, 0.0]])
    assert abs(dist - 3.0) < 1e-12 and np.allclose(ga, [0.5, 0.5])
    # duplicated points do not change the distance
    P2 = np.vstack([P, P[:5]])
    dist2, _, _ = api.polytope_distance(P2, Q)
    assert abs(dist2 - (P.min() - Q.max())) < 1e-12


def test_intersecting_hulls_give_zero():
    rng = np.random.default_rng(9)
    P = rng.standard_normal((80, 4))
    Q = rng.standard_normal((90, 4))
    dist, mu, ga = api.polytope_distance(P, Q, tol=1e-12, max_iter=5000)
    assert dist < 1e-6
    _check_weights(P, Q, dist, mu, ga)


def test_rejects_bad_arguments():
    lib = _ffi.load()
    buf = (ctypes.c_double * 8)()
    out = ctypes.c_double()
    p = ctypes.cast(buf, ctypes.c_void_p)
    assert lib.pdscp_polytope_distance(None, 1, p, 1, 1, 0.0, 10, p, p, ctypes.byref(out)) == 1
    assert lib.pdscp_polytope_distance(p, 0, p, 1, 1, 0.0, 10, p, p, ctypes.byref(out)) == 1
    assert lib.pdscp_polytope_distance(p, 1, p, 1, 0, 0.0, 10, p, p, ctypes.byref(out)) == 1
    assert lib.pdscp_polytope_distance(p, 1, p, 1, 1, -1.0, 10, p, p, ctypes.byref(out)) == 1
    assert lib.pdscp_polytope_distance(p, 1, p, 1, 1, 0.0, 0, p, p, ctypes.byref(out)) == 1
    with pytest.raises(ValueError):
        api.polytope_distance(np.ones((2, 3)), np.ones((2, 4)))
