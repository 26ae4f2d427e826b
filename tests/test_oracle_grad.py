"""Pins for the FP64 gradient oracles of the unrolled alpha-FTPs
(oracle/ses_grad.py, oracle/svm_grad.py).

SES: the independent numpy forward of oracle/ses.py (value and central finite
differences), the closed form at T = 1 (ubar^1 = v_1), and the closed form for
two points, where every ORACLE answer lies on the segment v_1 v_2 and
ubar^T = v_1 + alpha (T-1)/T (v_2 - v_1)/|v_2 - v_1|.
SVM: the numpy forward of oracle/svm.py (value and central finite differences)
and the closed form at T = 1 (wbar^1 = z/|z| from uniform weights).
"""

import numpy as np
import pytest

from oracle import ses as oses
from oracle import ses_grad
from paper_2405_09157_gb300 import datagen


def numpy_forward(V, g, alpha, eta, rho, T):
    """f(ubar^T) from the numpy alpha-FTP (stops at separation, as the oracle)."""
    ubar = V[0].copy()
    for t in range(T):
        rec = oses.ses_step(V, g, ubar, t, alpha, eta, rho)
        if rec["failed"]:
            break
        ubar = rec["ubar_next"]
    return oses.ses_objective(V, g, ubar)


def _case(n, d, seed, rel_alpha=0.9, radii=False):
    V = datagen.ses_gaussian(n, d, seed).astype(np.float64)
    g = 0.1 * np.random.default_rng(seed).random(n) if radii else None
    D = oses.ses_D(V, g)
    return V, g, rel_alpha * D, oses.ses_width(D)


@pytest.mark.parametrize("radii", [False, True])
def test_value_matches_numpy_forward(radii):
    V, g, alpha, rho = _case(40, 4, 1, radii=radii)
    eta = 0.5
    for T in (1, 2, 7, 20):
        L, grad, steps = ses_grad.ses_unrolled_radius_grad(V, g, alpha, eta / rho, T)
        assert abs(L - numpy_forward(V, g, alpha, eta, rho, T)) <= 1e-12 * alpha
        assert steps == T and np.all(np.isfinite(grad))


@pytest.mark.parametrize("n,d,T,radii,seed", [(25, 3, 8, False, 2), (18, 5, 15, True, 3), (30, 2, 25, False, 4)])
def test_gradient_matches_central_differences(n, d, T, radii, seed):
    V, g, alpha, rho = _case(n, d, seed, radii=radii)
    eta = 0.5
    L, grad, steps = ses_grad.ses_unrolled_radius_grad(V, g, alpha, eta / rho, T)
    assert steps == T
    # the maximum in f must be attained by one row with a clear margin (f is smooth there)
    ubar = V[0].copy()
    for t in range(T):
        ubar = oses.ses_step(V, g, ubar, t, alpha, eta, rho)["ubar_next"]
    dist = np.sqrt(np.sum((V - ubar) ** 2, axis=1)) + (0 if g is None else g)
    top = np.sort(dist)[-2:]
    assert top[1] - top[0] > 1e-3
    h = 1e-6
    fd = np.zeros_like(V)
    for i in range(n):
        for j in range(d):
            Vp, Vm = V.copy(), V.copy()
            Vp[i, j] += h
            Vm[i, j] -= h
            fd[i, j] = (numpy_forward(Vp, g, alpha, eta, rho, T) - numpy_forward(Vm, g, alpha, eta, rho, T)) / (2 * h)
    scale = np.max(np.abs(grad))
    assert np.max(np.abs(fd - grad)) <= 1e-6 * scale, np.max(np.abs(fd - grad)) / scale
    assert np.count_nonzero(np.abs(grad[1:]) > 1e-3 * scale) >= 2  # the sweep reaches the cones, not only v_1


def test_one_iteration_closed_form():
    # T = 1: ubar^1 = u^0 = v_1, so L = max_i |v_1 - v_i| and only v_1 and the farthest row move it
    V, g, alpha, rho = _case(12, 3, 5)
    L, grad, _ = ses_grad.ses_unrolled_radius_grad(V, None, alpha, 0.5 / rho, 1)
    dist = np.linalg.norm(V - V[0], axis=1)
    k = int(np.argmax(dist))
    direc = (V[0] - V[k]) / dist[k]
    want = np.zeros_like(V)
    want[0], want[k] = direc, -direc
    assert abs(L - dist[k]) <= 1e-14 * dist[k]
    assert np.allclose(grad, want, rtol=0, atol=1e-14)


@pytest.mark.parametrize("T,rel", [(3, 0.8), (6, 0.8), (6, 0.95)])
def test_two_points_closed_form(T, rel):
    # n = 2: ubar^T = v_1 + r (v_2 - v_1)/l, r = alpha (T-1)/T, l = |v_2 - v_1|;
    # f = max(r, l - r): gradient (v_2 - v_1)/l on v_2, its negative on v_1 when l - r > r, else 0
    V = np.array([[0.3, -1.0, 2.0], [1.7, 0.4, -0.5]])
    l = float(np.linalg.norm(V[1] - V[0]))
    alpha = rel * l
    rho = oses.ses_width(oses.ses_D(V))
    L, grad, steps = ses_grad.ses_unrolled_radius_grad(V, None, alpha, 0.7 / rho, T)
    assert steps == T
    r = alpha * (T - 1) / T
    assert abs(L - max(r, l - r)) <= 1e-13 * l
    unit = (V[1] - V[0]) / l
    if l - r > r:
        want = np.stack([-unit, unit])
    else:
        want = np.zeros_like(V)
    assert np.allclose(grad, want, rtol=0, atol=1e-12)


# --- SVM: margin of the minimisation alpha-FTP (oracle/svm_grad.py) ----------

from oracle import svm as osvm  # noqa: E402
from oracle import svm_grad  # noqa: E402


def svm_numpy_forward(X, y, alpha, eta, rho, D, T):
    wbar, s1, s2 = np.zeros(X.shape[1]), 0.0, 0.0
    for t in range(T):
        rec = osvm.svm_step(X, y, wbar, s1, s2, t, alpha, eta, rho, D)
        if rec["failed"]:
            break
        wbar, s1, s2 = rec["wbar_next"], rec["s1bar_next"], rec["s2bar_next"]
    return osvm.svm_margin(X, y, wbar)


def _svm_case(n1, n2, d, seed):
    X, y = datagen.svm_clusters(n1, n2, d, mu_norm=3.0, band=0.5, seed=seed)
    X = X.astype(np.float64)
    D = osvm.svm_D(X)
    return X, y, D, osvm.svm_width(D)


def test_svm_value_matches_numpy_forward():
    X, y, D, rho = _svm_case(15, 12, 3, 1)
    for T in (1, 3, 10, 30):
        L, grad, steps = svm_grad.svm_unrolled_margin_grad(X, y, 0.2 * D, 0.5 / rho, D, T)
        assert steps == T and np.all(np.isfinite(grad))
        assert abs(L - svm_numpy_forward(X, y, 0.2 * D, 0.5, rho, D, T)) <= 1e-12 * D


@pytest.mark.parametrize("n1,n2,d,T,seed", [(10, 9, 2, 6, 2), (8, 12, 4, 15, 3), (14, 11, 3, 25, 4)])
def test_svm_gradient_matches_central_differences(n1, n2, d, T, seed):
    X, y, D, rho = _svm_case(n1, n2, d, seed)
    alpha, eta = 0.2 * D, 0.5
    L, grad, steps = svm_grad.svm_unrolled_margin_grad(X, y, alpha, eta / rho, D, T)
    assert steps == T and L > 0
    h = 1e-6
    fd = np.zeros_like(X)
    for i in range(X.shape[0]):
        for j in range(d):
            Xp, Xm = X.copy(), X.copy()
            Xp[i, j] += h
            Xm[i, j] -= h
            fd[i, j] = (svm_numpy_forward(Xp, y, alpha, eta, rho, D, T) -
                        svm_numpy_forward(Xm, y, alpha, eta, rho, D, T)) / (2 * h)
    scale = np.max(np.abs(grad))
    assert np.max(np.abs(fd - grad)) <= 1e-6 * scale, np.max(np.abs(fd - grad)) / scale
    # beyond the two rows attaining the margin, the sweep reaches the other points through z
    assert np.count_nonzero(np.abs(grad) > 1e-3 * scale) > 2 * d


def test_svm_one_iteration_closed_form():
    # T = 1: wbar^1 = w^0 = z/|z| with z = (sum_P x - sum_Q x)/n (p^1 = e/r), |wbar^1| = 1, so
    # L = x_iP.w - x_iQ.w and dL/dx_i = [i = iP] w - [i = iQ] w + (y_i/n)(I - w w^T)(x_iP - x_iQ)/|z|
    X, y, D, rho = _svm_case(9, 11, 3, 5)
    n = X.shape[0]
    L, grad, _ = svm_grad.svm_unrolled_margin_grad(X, y, 0.1 * D, 0.5 / rho, D, 1)
    z = (X[y > 0].sum(axis=0) - X[y < 0].sum(axis=0)) / n
    w = z / np.linalg.norm(z)
    s = X @ w
    iP = np.flatnonzero(y > 0)[np.argmin(s[y > 0])]
    iQ = np.flatnonzero(y < 0)[np.argmax(s[y < 0])]
    assert abs(L - (s[iP] - s[iQ])) <= 1e-13 * D
    proj = (np.eye(3) - np.outer(w, w)) @ (X[iP] - X[iQ]) / np.linalg.norm(z)
    want = np.outer(y.astype(np.float64) / n, proj)
    want[iP] += w
    want[iQ] -= w
    assert np.allclose(grad, want, rtol=0, atol=1e-13)


# --- the unrolled gradient against the envelope-theorem gradient -------------


def _envelope_gradient(V, c, r):
    """dr*/dv_i = mu_i (v_i - c*)/r* with mu the optimal dual weights on the
    support (points at distance r* from c*; c* = sum mu_i v_i, sum mu_i = 1,
    mu >= 0, solved by non-negative least squares)."""
    from scipy.optimize import nnls
    dist = np.linalg.norm(V - c, axis=1)
    S = np.flatnonzero(np.abs(dist - r) <= 1e-9 * r)
    A = np.vstack([(V[S] - c).T, np.ones(len(S))])
    mu, res = nnls(A, np.concatenate([np.zeros(V.shape[1]), [1.0]]))
    assert res <= 1e-9
    G = np.zeros_like(V)
    G[S] = mu[:, None] * (V[S] - c) / r
    return G


def test_unrolled_gradient_is_not_the_envelope_gradient():
    # The unrolled gradient is the derivative of the T-step computation, not of the optimal radius r*:
    # near the equilibrium g -> 0 and u = v_1 + alpha g/|g| turns with O(1/|g|) sensitivity, so the
    # derivative of ubar^T grows quickly with T. Measured on a 40-point planar instance at alpha = 1.02 r*:
    # relative distance to the envelope gradient ~1.9 for T <= 10, then > 10 by T = 20 and > 100 by T = 50.
    from oracle import exact
    V = datagen.ses_gaussian(40, 2, 1).astype(np.float64)
    c, r = exact.mec_2d(V)
    Ge = _envelope_gradient(V, c, r)
    assert np.allclose(Ge.sum(axis=0), 0.0, atol=1e-12)  # translation invariance of r*
    rho = oses.ses_width(oses.ses_D(V))
    errs = {}
    for T in (5, 20, 50):
        _, G, steps = ses_grad.ses_unrolled_radius_grad(V, None, 1.02 * r, 0.5 / rho, T)
        assert steps == T and np.allclose(G.sum(axis=0), 0.0, atol=1e-9 * np.abs(G).max())
        errs[T] = np.linalg.norm(G - Ge) / np.linalg.norm(Ge)
    assert 1.0 < errs[5] < 3.0 and errs[20] > 10.0 and errs[50] > 100.0, errs
