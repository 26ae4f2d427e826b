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


def test_rounds_only_tighten():
    rng = np.random.default_rng(9)
    V = rng.normal(size=(2000, 6))
    c = V[0] + 0.3
    lb1, ub1, _ = oses.ses_coreset_bounds(V, c, K=16, tol=1e-6)
    lb4, ub4, _ = oses.ses_coreset_bounds(V, c, K=16, tol=1e-6, rounds=4)
    opt_lb, opt_ub, _ = oses.ses_coreset_bounds(V, V.mean(0), K=2000, tol=1e-9)
    assert lb4 >= lb1 * (1 - 1e-12) and ub4 <= ub1 * (1 + 1e-12)
    assert lb4 <= opt_ub * (1 + 1e-12) and ub4 >= opt_lb * (1 - 1e-12)


@pytest.mark.parametrize("n,seed", [(400, 0), (1500, 1)])
def test_coreset_search_brackets_welzl(n, seed):
    """The search in CORESET mode (points in the plane, eps = 1e-3) brackets
    Welzl's radius, closes within eps, returns an enclosing ball, and needs
    no more iterations than the MWU-only CERTIFIED search."""
    rng = np.random.default_rng(seed)
    V = rng.random((n, 2))
    opt = exact.mec_2d(V)[1]
    res = oses.ses_solve(V, eps=1e-3, mode=oses.MODE_CORESET, max_iters=20_000)
    assert res["lower_bound"] <= opt * (1 + 1e-12) and res["upper_bound"] >= opt * (1 - 1e-12), (res, opt)
    assert res["upper_bound"] <= (1 + 1e-3) * res["lower_bound"]
    assert float(np.linalg.norm(V - res["center"], axis=1).max()) <= res["upper_bound"] * (1 + 1e-12)
    plain = oses.ses_solve(V, eps=1e-3, mode=oses.MODE_CERTIFIED, max_iters=20_000)
    assert res["iters"] <= plain["iters"]
