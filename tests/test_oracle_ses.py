"""Pins for the SES oracle (Sec. 3, Sec. 4.1, Sec. 5).

Each test checks the oracle against something other than itself: the
unsimplified program it solves, brute force over feasible points, the SCMWU
definition with explicitly accumulated losses, the regret bound of Theorem 1,
the guarantee of Theorem 2, weak duality against exact solvers (Welzl,
support-set enumeration) and closed forms.
"""

import math

import numpy as np
import pytest

from oracle import eja, exact, ses
from paper_2405_09157_gb300 import datagen


def _inst(n=40, d=2, seed=0, radii=False):
    rng = np.random.default_rng(seed)
    V = rng.standard_normal((n, d))
    g = 0.3 * rng.random(n) if radii else None
    return V, g


def test_first_weights_are_e_over_r():
    V, _ = _inst(9, 3)
    P = ses.ses_weights(V, None, V[0], alpha=1.0, k=0.0)
    # p^1 = e/r with e = (0; sqrt2) per cone and r = 2(n-1)
    assert np.allclose(P[:, :-1], 0.0)
    assert np.allclose(P[:, -1], math.sqrt(2) / (2 * 8))


@pytest.mark.parametrize("radii", [False, True])
def test_weights_trace_one_and_in_cone(radii):
    V, g = _inst(50, 4, 1, radii)
    rng = np.random.default_rng(1)
    ubar = rng.standard_normal(4)
    P = ses.ses_weights(V, g, ubar, alpha=2.0, k=7.5)
    assert math.isclose(float(np.sum(P[:, -1])), 1 / math.sqrt(2), rel_tol=1e-13)  # sum s_i = 1/sqrt2
    assert np.all(np.linalg.norm(P[:, :-1], axis=1) <= P[:, -1] * (1 + 1e-13))


@pytest.mark.parametrize("radii", [False, True])
def test_oracle_closed_form_beats_random_feasible_points(radii):
    V, g = _inst(30, 3, 2, radii)
    gm = np.zeros(30) if g is None else g
    rng = np.random.default_rng(2)
    alpha = 1.7 * ses.ses_D(V, g) / 2
    P = ses.ses_weights(V, g, rng.standard_normal(3), alpha, k=3.0)
    u, value, _ = ses.ses_oracle(V, g, P, alpha)
    # the simplified objective equals the program's objective at the maximiser
    assert math.isclose(value, ses.ses_program_value(V, g, P, u, alpha), rel_tol=1e-11, abs_tol=1e-12)
    # u is feasible: ||u - v_1|| <= alpha - gamma_1
    assert np.linalg.norm(u - V[0]) <= alpha - gm[0] + 1e-12
    # no feasible (u', gamma') with gamma' <= alpha does better
    for _ in range(3000):
        gam = alpha - abs(rng.standard_normal()) * 0.3
        if gam < gm[0]:
            continue
        dirn = rng.standard_normal(3)
        dirn /= np.linalg.norm(dirn)
        up = V[0] + (gam - gm[0]) * rng.random() ** (1 / 3) * dirn
        assert ses.ses_program_value(V, g, P, up, gam) <= value + 1e-12


def test_oracle_failure_iff_alpha_below_primal_lb():
    V, g = _inst(25, 2, 3, True)
    rng = np.random.default_rng(3)
    P = ses.ses_weights(V, g, rng.standard_normal(2), 1.0, k=5.0)
    lb = ses.ses_primal_lb(V, g, P)
    for a in np.linspace(0.3 * lb, 3 * lb, 41):
        _, value, _ = ses.ses_oracle(V, g, P, a)
        if abs(a - lb) > 1e-9 * lb:
            assert (value < 0) == (a < lb)


def test_primal_lb_is_weakly_dual_to_exact_radius():
    V = datagen.ses_uniform(60, 2, seed=4).astype(np.float64)
    _, opt = exact.mec_2d(V)
    rng = np.random.default_rng(4)
    for _ in range(30):
        P = ses.ses_weights(V, None, rng.random(2), rng.uniform(0.2, 1.0), k=rng.uniform(0, 80))
        assert ses.ses_primal_lb(V, None, P) <= opt * (1 + 1e-12)


def _run(V, g, alpha, eta, rho, T):
    ubar = V[0].copy()
    recs = []
    for t in range(T):
        rec = ses.ses_step(V, g, ubar, t, alpha, eta, rho)
        recs.append(rec)
        if rec["failed"]:
            break
        ubar = rec["ubar_next"]
    return recs


def test_running_mean_form_equals_scmwu_definition_and_regret_bound():
    # Eq. (implement) rebuilds the exponent from t * ybar; Eq. (SCMWU) sums the
    # losses m^tau = (1/rho)(sum_j a_j y^tau_j - c). Both must give the same p,
    # and the losses must satisfy ||m||_inf <= 1 and Theorem 1's regret bound.
    V, g = _inst(12, 2, 5, True)
    gm = g
    D = ses.ses_D(V, g)
    rho = ses.ses_width(D)
    alpha = 0.9 * D
    eta, T = 0.3, 150
    recs = _run(V, g, alpha, eta, rho, T)
    assert not any(r["failed"] for r in recs)
    msum = np.zeros((11, 3))
    lhs = 0.0
    for rec in recs:
        P_def, _, _ = eja.scmwu_soc(-eta * msum)
        P_imp = ses.ses_weights(V, g, recs[rec["t"] - 1]["ubar_next"] if rec["t"] > 0 else V[0],
                                alpha, eta * rec["t"] / rho)
        assert np.allclose(P_def, P_imp, rtol=1e-9, atol=1e-15)
        m = np.empty((11, 3))
        m[:, :-1] = rec["u"][None, :] - V[1:]
        m[:, -1] = alpha - gm[1:]
        m /= rho
        assert eja.soc_inf_norm(m) <= 1.0 + 1e-12
        loss = float(np.sum(eja.soc_inner(m, P_def)))
        assert loss >= -1e-12          # m^t . p^t >= 0 when the ORACLE succeeds
        lhs += loss
        msum += m
    lam_min = float(np.min(eja.soc_lambda_min(msum)))
    r = ses.ses_rank(12)
    assert lhs <= lam_min + eta * len(recs) + math.log(r) / eta + 1e-9


@pytest.mark.parametrize("rel", [1.15, 0.8])
def test_theorem2_guarantee_small_instance(rel):
    V = datagen.ses_uniform(6, 2, seed=6).astype(np.float64)
    _, opt = exact.mec_2d(V)
    D = ses.ses_D(V)
    alpha, eps = rel * opt, 0.5
    T = ses.ses_T(D, 6, eps, alpha)
    eta = ses.theorem_eta(ses.ses_rank(6), T)
    res = ses.ses_ftp(V, None, alpha, eta, ses.ses_width(D), T, mode=ses.MODE_THEORY)
    if res["outcome"] == ses.OUT_SEPARATED:
        assert alpha < opt
    else:
        assert res["iters"] == T
        # dual repair: ball at ubar^T with radius (1+eps) alpha encloses everything
        assert ses.ses_objective(V, None, res["ubar"]) <= (1 + eps) * alpha + 1e-12
        assert opt <= (1 + eps) * alpha
    if rel < 1:
        assert res["outcome"] == ses.OUT_SEPARATED


def test_solve_brackets_welzl_on_1000_uniform_points():
    V = datagen.ses_uniform(1000, 2, seed=0).astype(np.float64)
    c, opt = exact.mec_2d(V)
    res = ses.ses_solve(V, eps=1e-2, max_iters=6000)
    assert res["lower_bound"] <= opt * (1 + 1e-12)
    assert res["radius"] >= opt * (1 - 1e-12)
    assert ses.ses_objective(V, None, res["center"]) <= res["radius"] * (1 + 1e-12)
    assert res["radius"] <= 1.01 * opt


def test_two_points_and_square():
    # n = 2, alpha = OPT = 1: u^1 = v_1 (g = 0 at t = 0), then every ORACLE
    # answer is the midpoint, so ubar^T = (T-1)/T * midpoint exactly.
    V = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0]])
    T = 50
    res = ses.ses_ftp(V, None, 1.0, 1.0, ses.ses_width(2.0), T, mode=ses.MODE_FIXED)
    assert np.allclose(res["ubar"], [(T - 1) / T, 0.0, 0.0], rtol=1e-14)
    assert math.isclose(res["f_best"], 1.0 + 1.0 / T, rel_tol=1e-13)
    # unit square (+ centre): OPT = sqrt(1/2) at (1/2, 1/2). The paper's
    # practical rule stops within its reported error band (Sec. 5 tables,
    # errors up to ~1e-2), with the theorem's eta or a fixed eta = 1.
    sq = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0], [0.5, 0.5]])
    opt = math.sqrt(0.5)
    res = ses.ses_solve(sq, eps=1e-3, mode=ses.MODE_PRACTICAL, max_iters=20000)
    assert opt * (1 - 1e-12) <= res["radius"] <= 1.01 * opt
    assert res["lower_bound"] <= opt + 1e-12
    res = ses.ses_solve(sq, eps=1e-3, mode=ses.MODE_PRACTICAL, max_iters=20000, eta=1.0)
    assert opt * (1 - 1e-12) <= res["radius"] <= 1.01 * opt
    assert res["lower_bound"] <= opt + 1e-12


def test_spheres_with_radii_against_enclosing_definition():
    # three unit-free spheres on a line: centres 0, 4, 10 with radii 1, 0.5, 2;
    # the smallest enclosing sphere spans [-1, 12]: centre 5.5, radius 6.5.
    V = np.array([[0.0], [4.0], [10.0]])
    g = np.array([1.0, 0.5, 2.0])
    res = ses.ses_solve(V, g, eps=1e-3, max_iters=30000)
    assert res["lower_bound"] <= 6.5 + 1e-9
    assert 6.5 - 1e-9 <= res["radius"] <= 6.5 * 1.01
    res = ses.ses_solve(V, g, eps=1e-3, max_iters=30000, eta=1.0)
    assert 6.5 - 1e-9 <= res["radius"] <= 6.5 * 1.01


def test_bruteforce_meb_3d_bounds():
    V = datagen.ses_gaussian(9, 3, seed=7).astype(np.float64)
    _, opt = exact.meb_bruteforce(V)
    # the budget ends inside a slow separation step: bounds stay valid
    res = ses.ses_solve(V, eps=1e-2, max_iters=8000)
    assert res["lower_bound"] <= opt * (1 + 1e-9)
    assert opt * (1 - 1e-12) <= res["radius"]
    res = ses.ses_solve(V, eps=1e-2, max_iters=8000, eta=1.0)
    assert res["lower_bound"] <= opt * (1 + 1e-9)
    assert opt * (1 - 1e-12) <= res["radius"] <= 1.02 * opt
