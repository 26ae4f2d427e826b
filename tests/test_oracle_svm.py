"""Pins for the SVM oracle (Sec. 3 minimisation variant, Sec. 4.2, Sec. 5).

Checked against: brute force over feasible ORACLE points, the unsimplified
ORACLE program, Claim 8, weak duality against exact polytope distance,
the regret bound of Theorem 1 on R^n_+ and the guarantee of Theorem 3.
"""

import math

import numpy as np
import pytest

from oracle import eja, exact, svm
from paper_2405_09157_gb300 import datagen


def _inst(n1=6, n2=5, d=2, seed=0):
    X, y = datagen.svm_clusters(n1, n2, d, mu_norm=3.0, band=0.5, seed=seed)
    return X.astype(np.float64), y


def test_oracle_closed_form_beats_random_feasible_points():
    X, y = _inst(20, 25, 3, 1)
    D = svm.svm_D(X)
    rng = np.random.default_rng(1)
    p = svm.svm_weights(X, y, rng.standard_normal(3), 0.3, 0.2, k=2.0)
    for alpha in (0.5 * D, 1.3 * D):
        w, s1, s2, value, _, _, _ = svm.svm_oracle(X, y, p, alpha, D)
        assert math.isclose(value, svm.svm_program_value(X, y, p, w, s1, s2), rel_tol=1e-11, abs_tol=1e-12)
        assert np.linalg.norm(w) <= 1 + 1e-12 and s1 <= D + 1e-12 and s2 <= D + 1e-12
        assert s1 + s2 >= alpha - 1e-12
        for _ in range(3000):
            wd = rng.standard_normal(3)
            wd *= rng.random() ** (1 / 3) / np.linalg.norm(wd)
            a = rng.uniform(alpha - D, D)
            b = rng.uniform(alpha - a, D) if alpha - a <= D else None
            if b is None:
                continue
            assert svm.svm_program_value(X, y, p, wd, a, b) <= value + 1e-12


def test_weights_sum_to_one_and_init_uniform():
    X, y = _inst(7, 9, 4, 2)
    p0 = svm.svm_weights(X, y, np.zeros(4), 0.0, 0.0, k=0.0)
    assert np.allclose(p0, 1.0 / 16)  # p^1 = e/r with r = n
    p = svm.svm_weights(X, y, np.ones(4), 0.5, -0.2, k=30.0)
    assert math.isclose(float(np.sum(p)), 1.0, rel_tol=1e-13) and np.all(p > 0)


def test_claim8_and_pd_upper_bound_against_bruteforce():
    X, y = _inst(5, 4, 2, 3)
    P, Q = X[y > 0], X[y < 0]
    opt, _, _ = exact.pd_bruteforce(P, Q)
    D = svm.svm_D(X)
    rng = np.random.default_rng(3)
    for _ in range(40):
        p = svm.svm_weights(X, y, rng.standard_normal(2), rng.normal(), rng.normal(), k=rng.uniform(0, 30))
        ub = svm.svm_pd_value(X, y, p)
        assert ub >= opt * (1 - 1e-12)               # PD-feasible, so >= OPT
        for alpha in np.linspace(0.1, 2 * D, 15):
            value = svm.svm_oracle(X, y, p, alpha, D)[3]
            if value < 0:
                assert ub < alpha                      # Claim 8


def test_margin_is_a_lower_bound_and_single_pair_closed_form():
    X, y = _inst(6, 6, 3, 4)
    P, Q = X[y > 0], X[y < 0]
    opt, _, _ = exact.pd_bruteforce(P, Q)
    rng = np.random.default_rng(4)
    for _ in range(50):
        assert svm.svm_margin(X, y, rng.standard_normal(3)) <= opt * (1 + 1e-12)
    # one point per class: OPT = ||u - v|| with w = (u - v)/||u - v||
    X2 = np.array([[1.0, 2.0], [-2.0, -2.0]])
    y2 = np.array([1, -1], dtype=np.int8)
    res = svm.svm_solve(X2, y2, eps=1e-3, max_iters=20000, eta=1.0)
    assert res["lower_bound"] <= 5.0 * (1 + 1e-12) <= res["upper_bound"] * (1 + 1e-12)
    assert math.isclose(svm.svm_pd_value(X2, y2, np.array([0.5, 0.5])), 5.0)
    assert res["margin"] >= 0.99 * 5.0


def test_regret_bound_on_the_orthant():
    X, y = _inst(8, 7, 2, 5)
    n = X.shape[0]
    D = svm.svm_D(X)
    rho = svm.svm_width(D)
    eta, T, alpha = 0.4, 200, 0.5
    wbar, s1b, s2b = np.zeros(2), 0.0, 0.0
    msum = np.zeros(n)
    lhs = 0.0
    for t in range(T):
        rec = svm.svm_step(X, y, wbar, s1b, s2b, t, alpha, eta, rho, D)
        assert not rec["failed"]
        p_def, _, _ = eja.scmwu_orthant(-eta * msum)   # Eq. (SCMWU) with summed losses
        p_imp = svm.svm_weights(X, y, wbar, s1b, s2b, eta * t / rho)
        assert np.allclose(p_def, p_imp, rtol=1e-9)
        slack = np.where(y > 0, X @ rec["w"] - rec["s1"], -(X @ rec["w"]) - rec["s2"])
        m = slack / rho
        assert np.max(np.abs(m)) <= 1 + 1e-12          # width rho <= 2D
        loss = float(m @ p_def)
        assert loss >= -1e-12
        lhs += loss
        msum += m
        wbar, s1b, s2b = rec["wbar_next"], rec["s1bar_next"], rec["s2bar_next"]
    assert lhs <= float(np.min(msum)) + eta * T + math.log(n) / eta + 1e-9


@pytest.mark.parametrize("rel", [0.85, 1.25])
def test_theorem3_guarantee_small_instance(rel):
    X, y = _inst(4, 4, 2, 6)
    P, Q = X[y > 0], X[y < 0]
    opt, _, _ = exact.pd_bruteforce(P, Q)
    D = svm.svm_D(X)
    alpha, eps = rel * opt, 0.9
    T = svm.svm_T(D, X.shape[0], eps, alpha)
    eta = math.sqrt(math.log(X.shape[0]) / T)
    res = svm.svm_ftp(X, y, alpha, eta, svm.svm_width(D), T, D, mode=svm.MODE_THEORY)
    if res["outcome"] == svm.OUT_SEPARATED:
        assert opt < alpha
    else:
        assert res["iters"] == T
        # dual repair (Theorem 3): (wbar; s1bar - eps alpha/R; s2bar - eps alpha/R) is
        # feasible for (SVM) with value >= (1 - eps) alpha
        d = eps * alpha / svm.SVM_R
        w = res["wbar"]
        assert np.linalg.norm(w) <= 1 + 1e-12
        assert np.all(P @ w >= res["s1bar"] - d - 1e-9)
        assert np.all(-(Q @ w) >= res["s2bar"] - d - 1e-9)
        assert res["s1bar"] + res["s2bar"] - 2 * d >= (1 - eps) * alpha - 1e-9
    if rel > 1:
        assert res["outcome"] == svm.OUT_SEPARATED


def test_solve_brackets_exact_polytope_distance():
    X, y = _inst(6, 6, 2, 7)
    P, Q = X[y > 0], X[y < 0]
    opt, _, _ = exact.pd_bruteforce(P, Q)
    for eta in (None, 1.0):
        res = svm.svm_solve(X, y, eps=1e-2, max_iters=20000, eta=eta)
        assert res["lower_bound"] <= opt * (1 + 1e-9)
        assert res["upper_bound"] >= opt * (1 - 1e-9)
        assert math.isclose(exact.svm_margin_of(P, Q, res["w"]), res["margin"], rel_tol=1e-9)
    assert res["margin"] >= 0.98 * opt


@pytest.mark.parametrize("seed", range(6))
def test_mdm_matches_bruteforce_polytope_distance(seed):
    rng = np.random.default_rng(100 + seed)
    d = int(rng.integers(2, 5))
    P = rng.standard_normal((int(rng.integers(1, 7)), d)) + 1.5
    Q = rng.standard_normal((int(rng.integers(1, 7)), d)) - 1.5
    opt, _, _ = exact.pd_bruteforce(P, Q)
    dist, mu, ga, gap, _ = exact.pd_mdm(P, Q, tol=1e-14)
    assert abs(dist - opt) <= 1e-9 * max(opt, 1.0)
    assert np.all(mu >= 0) and np.all(ga >= 0) and abs(mu.sum() - 1) < 1e-12 and abs(ga.sum() - 1) < 1e-12
    z = P.T @ mu - Q.T @ ga
    assert abs(math.sqrt(float(z @ z)) - dist) <= 1e-12 * max(dist, 1.0)
    # the direction's margin never exceeds the distance (weak duality, Sec. 4.2)
    assert exact.svm_margin_of(P, Q, z) <= dist * (1 + 1e-12)


def test_coreset_bounds_bracket_the_optimum():
    X, y = _inst(7, 6, 3, 8)
    P, Q = X[y > 0], X[y < 0]
    opt, _, _ = exact.pd_bruteforce(P, Q)
    w0 = P.mean(axis=0) - Q.mean(axis=0)
    # a core set holding every point: the bounds are the optimum itself
    lb, ub, w = svm.svm_coreset_bounds(X, y, w0, eps=1e-9, K=100, rounds=1)
    assert abs(ub - opt) <= 1e-8 * opt and abs(lb - opt) <= 1e-6 * opt
    assert math.isclose(exact.svm_margin_of(P, Q, w), lb, rel_tol=1e-9)
    # core sets of two points per class from a poor direction: still bounds
    lb, ub, w = svm.svm_coreset_bounds(X, y, np.array([1.0, 0.0, 0.0]), eps=1e-3, K=2)
    assert lb <= opt * (1 + 1e-9) <= ub * (1 + 2e-9)


def test_coreset_pick_takes_the_points_nearest_the_hyperplane():
    X = np.array([[3.0, 0], [1.0, 5], [2.0, -1], [-1.0, 0], [-4.0, 2], [-2.5, 1]])
    y = np.array([1, 1, 1, -1, -1, -1], dtype=np.int8)
    pick = svm.svm_coreset_pick(X, y, np.array([1.0, 0.0]), 2)
    # y x^T w: P 3, 1, 2 -> 1, 2; Q 1, 4, 2.5 -> 1, 2.5
    assert pick.tolist() == [False, True, True, True, False, True]


def test_coreset_search_certifies_and_brackets():
    for (n1, n2, d, seed) in [(6, 6, 2, 7), (5, 7, 3, 9)]:
        X, y = _inst(n1, n2, d, seed)
        P, Q = X[y > 0], X[y < 0]
        opt, _, _ = exact.pd_bruteforce(P, Q)
        res = svm.svm_solve(X, y, eps=1e-3, mode=svm.MODE_CORESET, max_iters=20000)
        assert res["lower_bound"] <= opt * (1 + 1e-9) and res["upper_bound"] >= opt * (1 - 1e-9)
        assert res["upper_bound"] <= (1 + 1e-3) * res["lower_bound"]
        assert math.isclose(exact.svm_margin_of(P, Q, res["w"]), res["margin"], rel_tol=1e-9)
