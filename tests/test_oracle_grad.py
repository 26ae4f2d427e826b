"""Pins for the FP64 gradient oracle of the unrolled SES alpha-FTP (oracle/ses_grad.py).

Checked against: the independent numpy forward of oracle/ses.py (value and
central finite differences), the closed form at T = 1 (ubar^1 = v_1), and the
closed form for two points, where every ORACLE answer lies on the segment
v_1 v_2 and ubar^T = v_1 + alpha (T-1)/T (v_2 - v_1)/|v_2 - v_1|.
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
