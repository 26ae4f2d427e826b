"""Pins for the averaged-weight certificates and the CERTIFIED search of the
oracle (oracle/ses.py, oracle/svm.py).

SES: the weights kappa_i read off the SOC exponential reproduce the ORACLE's g;
the incremental averaged bound equals the QP objective of Sec. 5 (Eq. ses_qp)
evaluated, in absolute coordinates, at the explicitly averaged weight vector;
a symmetric configuration where the bound equals OPT in closed form; every
bound stays below the exact optimum (Welzl in the plane, support-set
enumeration in 3-D); the certified search brackets the exact optimum within
eps. SVM: the averaged Claim 8 value equals |P mubar - Q gammabar| for the
explicitly averaged class-normalised weights; one point per class gives the
closed form |u - v|; bounds against the brute-force polytope distance; the
certified search brackets it.
"""

import math

import numpy as np
import pytest

from oracle import exact
from oracle import ses as oses
from oracle import svm as osvm
from paper_2405_09157_gb300 import datagen


def _ses_run(V, alpha_rel, eta, T):
    """T iterations of the SES alpha-FTP keeping each iterate's weights."""
    D = oses.ses_D(V)
    rho = oses.ses_width(D)
    alpha = alpha_rel * D
    ubar = V[0].copy()
    avg = oses.ses_dual_state(V.shape[1])
    recs, weights = [], []
    for t in range(T):
        k = eta * t / rho
        P = oses.ses_weights(V, None, ubar, alpha, k)
        rec = oses.ses_step(V, None, ubar, t, alpha, eta, rho, avg=avg)
        recs.append(rec)
        weights.append((t, P, ubar.copy(), k))
        if rec["failed"]:
            break
        ubar = rec["ubar_next"]
    return recs, weights, D


def test_kappa_reproduces_g():
    V = datagen.ses_gaussian(200, 5, 3).astype(np.float64)
    _, weights, _ = _ses_run(V, 0.8, 0.5, 12)
    for t, P, ubar, k in weights[1:]:
        kap = oses.ses_qp_weights(V, None, ubar, P, k)
        assert np.all(kap >= 0.0)
        g = np.sum(P[:, :-1], axis=0)
        assert np.allclose(kap @ (V[1:] - ubar), g, rtol=0, atol=1e-14 * max(1.0, np.abs(g).max()))


@pytest.mark.parametrize("n,d,seed", [(60, 3, 1), (150, 8, 2), (40, 2, 5)])
def test_averaged_bound_is_the_qp_value_of_the_averaged_weights(n, d, seed):
    V = datagen.ses_gaussian(n, d, seed).astype(np.float64) + 3.0  # away from the origin
    recs, weights, D = _ses_run(V, 0.9, 0.7, 30)
    num, den = np.zeros(n - 1), 0.0
    for (t, P, ubar, k), rec in zip(weights, recs):
        kap = oses.ses_qp_weights(V, None, ubar, P, k)
        if t >= 1 and kap.sum() > 0:
            num += t * t * kap / kap.sum()
            den += t * t
            mu = num / den
            y = mu @ V[1:]
            qp = float(y @ y) - float(mu @ np.sum(V[1:] * V[1:], axis=1))  # Eq. ses_qp objective at x = mu
            assert rec["dual_bound"] == pytest.approx(math.sqrt(max(-qp, 0.0)), rel=1e-10, abs=1e-12 * D)
        else:
            assert rec["dual_bound"] == 0.0


def test_symmetric_points_give_opt():
    # v_1 at the centre, v_2, v_3 opposite: g = 0 keeps ubar = v_1, mu = (1/2, 1/2) and the bound is 1 = OPT
    V = np.array([[0.0, 0.0], [-1.0, 0.0], [1.0, 0.0]])
    recs, _, _ = _ses_run(V, 0.8, 0.5, 8)
    for rec in recs[1:]:
        assert rec["dual_bound"] == pytest.approx(1.0, abs=1e-15)


def test_ses_bounds_below_exact_optimum():
    V2 = datagen.ses_uniform(300, 2, 4).astype(np.float64)
    _, opt2 = exact.mec_2d(V2)
    V3 = datagen.ses_gaussian(14, 3, 6).astype(np.float64)
    _, opt3 = exact.meb_bruteforce(V3)
    for V, opt in ((V2, opt2), (V3, opt3)):
        for alpha_rel, eta in ((0.6, 1.0), (0.9, 0.3)):
            recs, _, _ = _ses_run(V, alpha_rel, eta, 200)
            for rec in recs:
                assert rec["dual_bound"] <= opt * (1 + 1e-12)
                assert rec["lower_bound"] <= opt * (1 + 1e-12)


def test_ses_certified_search_brackets_welzl():
    V = datagen.ses_uniform(1000, 2, 0).astype(np.float64)
    _, opt = exact.mec_2d(V)
    r = oses.ses_solve(V, eps=1e-3, mode="certified", max_iters=60_000, poll_every=64)
    assert r["lower_bound"] <= opt * (1 + 1e-12) <= r["radius"] * (1 + 1e-12)
    assert r["radius"] <= (1 + 1e-3) * r["lower_bound"]
    assert oses.ses_objective(V, None, r["center"]) == pytest.approx(r["radius"], rel=1e-12)
    # only proven conclusions move the range: every step ended on separation, f < alpha, the
    # certificates, or as stuck (which moves nothing and halves eta)
    allowed = {oses.OUT_SEPARATED, oses.OUT_BELOW_ALPHA, oses.OUT_CERTIFIED, oses.OUT_STUCK}
    assert {s["outcome"] for s in r["steps"]} <= allowed
    for a, b in zip(r["steps"], r["steps"][1:]):
        if a["outcome"] == oses.OUT_STUCK:
            assert b["eta"] == 0.5 * a["eta"]


def test_ses_certified_search_3d_bruteforce():
    V = datagen.ses_gaussian(12, 3, 9).astype(np.float64)
    _, opt = exact.meb_bruteforce(V)
    r = oses.ses_solve(V, eps=1e-3, mode="certified", max_iters=60_000, poll_every=64)
    assert r["lower_bound"] <= opt * (1 + 1e-12) <= r["radius"] * (1 + 1e-12)
    assert r["radius"] <= (1 + 1e-3) * r["lower_bound"]


def test_certified_and_practical_certificates_agree():
    # both searches keep valid certificates, so each one's lower bound is below the other's ball
    V = datagen.ses_gaussian(300, 16, 0).astype(np.float64)
    rc = oses.ses_solve(V, eps=1e-2, mode="certified", max_iters=40_000, poll_every=64)
    rp = oses.ses_solve(V, eps=1e-2, max_iters=40_000)
    assert rc["radius"] <= (1 + 1e-2) * rc["lower_bound"]
    assert rc["L"] <= rc["radius"] and rc["lower_bound"] <= rp["radius"]
    assert rp["lower_bound"] <= rc["radius"]


# --- SVM -----------------------------------------------------------------


def _svm_run(X, y, alpha_rel, eta, T):
    D = osvm.svm_D(X)
    rho = osvm.svm_width(D)
    alpha = alpha_rel * D
    d = X.shape[1]
    wbar, s1, s2 = np.zeros(d), 0.0, 0.0
    avg = osvm.svm_dual_state(d)
    recs, ps = [], []
    for t in range(T):
        p = osvm.svm_weights(X, y, wbar, s1, s2, eta * t / rho)
        rec = osvm.svm_step(X, y, wbar, s1, s2, t, alpha, eta, rho, D, avg=avg)
        recs.append(rec)
        ps.append((t, p))
        if rec["failed"]:
            break
        wbar, s1, s2 = rec["wbar_next"], rec["s1bar_next"], rec["s2bar_next"]
    return recs, ps


def test_svm_averaged_bound_is_the_pd_value_of_the_averaged_weights():
    X, y = datagen.svm_clusters(40, 30, 4, mu_norm=3.0, band=0.5, seed=2)
    X = X.astype(np.float64)
    recs, ps = _svm_run(X, y, 0.3, 0.8, 40)
    P, Q = X[y > 0], X[y < 0]
    mu_acc, ga_acc, den = np.zeros(len(P)), np.zeros(len(Q)), 0.0
    for (t, p), rec in zip(ps, recs):
        if t == 0:
            assert math.isinf(rec["dual_bound"])
            continue
        mu, ga = p[y > 0], p[y < 0]
        mu_acc += t * t * mu / mu.sum()
        ga_acc += t * t * ga / ga.sum()
        den += t * t
        diff = P.T @ (mu_acc / den) - Q.T @ (ga_acc / den)
        assert rec["dual_bound"] == pytest.approx(float(np.linalg.norm(diff)), rel=1e-12)


def test_svm_one_point_per_class_closed_form():
    X = np.array([[1.0, 2.0, 0.5], [-1.0, 0.0, 1.5]])
    y = np.array([1, -1], dtype=np.int8)
    recs, _ = _svm_run(X, y, 0.5, 0.5, 6)
    for rec in recs[1:]:
        assert rec["dual_bound"] == pytest.approx(float(np.linalg.norm(X[0] - X[1])), rel=1e-15)


def test_svm_bounds_and_certified_search_against_bruteforce():
    X, y = datagen.svm_clusters(5, 5, 2, band=0.5, seed=7)
    X = X.astype(np.float64)
    opt, _, _ = exact.pd_bruteforce(X[y > 0], X[y < 0])
    recs, _ = _svm_run(X, y, 0.5, 1.0, 300)
    for rec in recs[1:]:
        assert rec["dual_bound"] >= opt * (1 - 1e-12)
        assert rec["objective"] <= opt * (1 + 1e-12)
    r = osvm.svm_solve(X, y, eps=1e-3, mode="certified", max_iters=100_000, poll_every=64)
    assert r["lower_bound"] <= opt * (1 + 1e-12) <= r["upper_bound"] * (1 + 1e-12)
    assert r["upper_bound"] <= (1 + 1e-3) * r["lower_bound"]
    assert exact.svm_margin_of(X[y > 0], X[y < 0], r["w"]) == pytest.approx(r["margin"], rel=1e-9)
    assert {s["outcome"] for s in r["steps"]} <= {osvm.OUT_SEPARATED, osvm.OUT_ABOVE_ALPHA, osvm.OUT_CERTIFIED,
                                                  osvm.OUT_STUCK}
