"""Pins for the exact tiny-input solvers against closed forms and each other."""

import math

import numpy as np

from oracle import exact


def test_mec_closed_forms():
    tri = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, math.sqrt(3) / 2]])
    c, r = exact.mec_2d(tri)
    assert math.isclose(r, 1 / math.sqrt(3), rel_tol=1e-12)          # circumradius
    assert np.allclose(c, [0.5, math.sqrt(3) / 6])
    obtuse = np.array([[0.0, 0.0], [4.0, 0.0], [2.0, 0.3]])          # diameter circle
    c, r = exact.mec_2d(obtuse)
    assert math.isclose(r, 2.0, rel_tol=1e-12) and np.allclose(c, [2.0, 0.0])


def test_mec_matches_support_set_enumeration():
    rng = np.random.default_rng(0)
    for _ in range(20):
        P = rng.standard_normal((int(rng.integers(2, 9)), 2))
        _, r1 = exact.mec_2d(P, seed=int(rng.integers(1000)))
        _, r2 = exact.meb_bruteforce(P)
        assert math.isclose(r1, r2, rel_tol=1e-9)


def test_meb_3d_encloses_and_is_tight():
    rng = np.random.default_rng(1)
    P = rng.standard_normal((7, 3))
    c, r = exact.meb_bruteforce(P)
    dist = np.linalg.norm(P - c, axis=1)
    assert np.all(dist <= r * (1 + 1e-9))
    assert np.sum(np.isclose(dist, r, rtol=1e-9)) >= 2
    # regular simplex vertices e_1..e_4 in R^4: centre (1/4,..), radius sqrt(3/4)
    c, r = exact.meb_bruteforce(np.eye(4))
    assert math.isclose(r, math.sqrt(0.75), rel_tol=1e-12)


def test_pd_closed_forms_and_scipy_agreement():
    # point to segment: distance from (0, 1) to segment [(-1,0),(1,0)] is 1
    dist, mu, ga = exact.pd_bruteforce(np.array([[0.0, 1.0]]), np.array([[-1.0, 0.0], [1.0, 0.0]]))
    assert math.isclose(dist, 1.0, rel_tol=1e-12)
    assert math.isclose(float(mu.sum()), 1.0) and math.isclose(float(ga.sum()), 1.0)
    # against scipy's SLSQP on the QP form (eq. svm_qp) of random tiny sets
    from scipy.optimize import minimize
    rng = np.random.default_rng(2)
    for _ in range(5):
        P = rng.standard_normal((4, 2)) + 3.0
        Q = rng.standard_normal((4, 2)) - 3.0
        dist, _, _ = exact.pd_bruteforce(P, Q)

        def f(z):
            return float(np.sum((z[:4] @ P - z[4:] @ Q) ** 2))
        cons = [{"type": "eq", "fun": lambda z: z[:4].sum() - 1},
                {"type": "eq", "fun": lambda z: z[4:].sum() - 1}]
        sol = minimize(f, np.full(8, 0.25), bounds=[(0, None)] * 8, constraints=cons,
                       method="SLSQP", options={"ftol": 1e-14, "maxiter": 500})
        assert math.isclose(dist, math.sqrt(sol.fun), rel_tol=1e-5)
