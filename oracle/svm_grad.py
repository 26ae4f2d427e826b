"""Gradient of the SVM alpha-FTP's final margin with respect to the points, FP64.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline may import this package; the library never does.

The function differentiated is the minimisation alpha-FTP of Sec. 3
(Theorem 3) for the hard-margin SVM (Sec. 4.2) at a fixed alpha, a fixed
eta/rho and a fixed D (Lemma 6), run for T iterations from t = 0 (wbar = 0,
sbar = 0), followed by the margin of Sec. 5 at the final mean:

    L(X) = f(wbar^T) = max{(min_P x^T wbar - max_Q x^T wbar)/|wbar|, 0}.

Each iteration is written in the paper's order with plain PyTorch CPU ops in
float64: the exponent -(eta t/rho)(y_i x_i^T wbar - sbar_class(i)) of Eq.
(min_implement) over R^n_+, the normalised weights p = exp(x)/Tr exp(x) (Eq.
SCMWU, largest exponent subtracted first as in eja.scmwu_orthant), the
closed-form ORACLE of Eq. (svm_oracle): z = P mu - Q gamma, w = z/|z|,
s_1 = D if Tr mu <= Tr gamma else alpha - D, s_2 = alpha - s_1, its value,
and the running means. Reverse-mode automatic differentiation (a library
primitive) gives dL/dX. The choice of s_1 is piecewise constant in X (no
gradient flows through it); the rows attaining the minimum over P and the
maximum over Q (smallest index on ties) carry the margin's subgradient; a
clipped margin (f = 0) has gradient 0.

Pinned in tests/test_oracle_grad.py against central finite differences of
the independent numpy forward (svm.svm_step), the forward's value, and the
closed form at T = 1.
"""

import math

import numpy as np
import torch


def svm_unrolled_margin(X, y, alpha, eta_over_rho, D, T):
    """L = f(wbar^T) as a differentiable function of X ((n, d) float64 tensor).

    Returns (L, wbar^T, steps); stops early, as svm.svm_ftp does, when the
    ORACLE value is negative (separation).
    """
    n, d = X.shape
    yt = torch.as_tensor(np.asarray(y, dtype=np.float64))
    pos, neg = yt > 0, yt < 0
    wbar = torch.zeros(d, dtype=torch.float64)
    s1b, s2b = 0.0, 0.0
    steps = 0
    for t in range(T):
        k = eta_over_rho * t
        sbar = torch.where(pos, torch.tensor(s1b, dtype=torch.float64), torch.tensor(s2b, dtype=torch.float64))
        e = -k * (yt * (X @ wbar) - sbar)                    # Eq. (min_implement)
        e = e - torch.max(e).detach()
        ex = torch.exp(e)
        p = ex / torch.sum(ex)                               # Eq. (SCMWU) over R^n_+
        mu = torch.where(pos, p, torch.zeros_like(p))
        ga = torch.where(neg, p, torch.zeros_like(p))
        z = X.T @ mu - X.T @ ga                              # Eq. (svm_oracle)
        nz = torch.sqrt(torch.sum(z * z))
        w = z / nz if float(nz.detach()) > 0.0 else torch.zeros_like(z)
        tr_mu, tr_ga = float(torch.sum(mu).detach()), float(torch.sum(ga).detach())
        s1 = D if tr_mu <= tr_ga else alpha - D
        s2 = alpha - s1
        value = torch.dot(z, w) - torch.sum(mu) * s1 - torch.sum(ga) * s2
        if float(value.detach()) < 0.0:
            break
        wbar = wbar + (w - wbar) / (t + 1)
        s1b = s1b + (s1 - s1b) / (t + 1)
        s2b = s2b + (s2 - s2b) / (t + 1)
        steps += 1
    nw = torch.sqrt(torch.sum(wbar * wbar))
    if float(nw.detach()) == 0.0:
        return torch.sum(X) * 0.0, wbar, steps
    with torch.no_grad():
        s = (X @ wbar).numpy()
        yn = np.asarray(y)
        iP = int(np.flatnonzero(yn > 0)[np.argmin(s[yn > 0])])
        iQ = int(np.flatnonzero(yn < 0)[np.argmax(s[yn < 0])])
    m = (torch.dot(X[iP], wbar) - torch.dot(X[iQ], wbar)) / nw
    if float(m.detach()) <= 0.0:
        return m * 0.0, wbar, steps
    return m, wbar, steps


def svm_unrolled_margin_grad(X, y, alpha, eta_over_rho, D, T):
    """(L, dL/dX as an (n, d) float64 numpy array, steps taken)."""
    Xt = torch.tensor(np.asarray(X, dtype=np.float64), requires_grad=True)
    L, _, steps = svm_unrolled_margin(Xt, y, alpha, eta_over_rho, D, T)
    L.backward()
    g = Xt.grad
    return float(L.detach()), (np.zeros(Xt.shape) if g is None else g.numpy().copy()), steps
