"""Core-set certificates for SES (oracle.ses.ses_coreset_bounds): the
Frank-Wolfe weights on the K farthest points give a lower bound and the ball
at their barycentre an upper bound on the minimum enclosing ball's radius,
checked against exact solvers (Welzl's algorithm in the plane, support-set
enumeration in d = 3) and against the closed forms of a regular simplex and
two points."""

import math

import numpy as np
import pytest

from oracle import exact, ses as oses


@pytest.mark.parametrize("seed", range(4))
def test_bounds_bracket_welzl_in_the_plane(seed):
    rng = np.random.default_rng(seed)
    V = rng.random((300, 2))
    opt = exact.mec_2d(V)[1]
    for K in (8, 64, 300):
        lb, ub, c = oses.ses_coreset_bounds(V, V[0], K=K, tol=1e-6)
        assert lb <= opt * (1 + 1e-12) and ub >= opt * (1 - 1e-12), (K, lb, opt, ub)
        assert math.isclose(ub, float(np.linalg.norm(V - c, axis=1).max()), rel_tol=1e-12)
    # the whole set as the core set: the gap closes to the tolerance
    lb, ub, _ = oses.ses_coreset_bounds(V, V.mean(0), K=300, tol=1e-6)
    assert ub <= (1 + 2e-6) * lb


def test_bounds_bracket_support_enumeration_in_3d():
    rng = np.random.default_rng(7)
    V = rng.normal(size=(12, 3))
    opt = exact.meb_bruteforce(V)[1]
    lb, ub, _ = oses.ses_coreset_bounds(V, V[0], K=12, tol=1e-9)
    assert lb <= opt * (1 + 1e-9) and ub >= opt * (1 - 1e-9)
    assert ub <= (1 + 1e-8) * lb


def test_closed_forms():
    # two points: radius half their distance, centre the midpoint
    V = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0]])
    lb, ub, c = oses.ses_coreset_bounds(V, V[0], K=2, tol=1e-12)
    assert math.isclose(lb, 1.0, rel_tol=1e-12) and math.isclose(ub, 1.0, rel_tol=1e-12)
    assert np.allclose(c, [1.0, 0.0, 0.0])
    # regular simplex of d + 1 unit vectors' vertices e_1..e_{d+1} in R^{d+1}:
    # circumradius sqrt(d / (d + 1))
    d = 5
    V = np.eye(d + 1)
    lb, ub, _ = oses.ses_coreset_bounds(V, V[0], K=d + 1, tol=1e-12)
    r = math.sqrt(d / (d + 1))
    assert math.isclose(lb, r, rel_tol=1e-10) and math.isclose(ub, r, rel_tol=1e-10)


def test_pick_is_the_farthest():
    rng = np.random.default_rng(3)
    V = rng.normal(size=(500, 4))
    c = rng.normal(size=4)
    idx = oses.ses_coreset_pick(V, c, 20)
    d = np.linalg.norm(V - c, axis=1)
    assert len(idx) == 20 and np.all(np.diff(idx) > 0)
    assert d[idx].min() >= np.sort(d)[-20]
