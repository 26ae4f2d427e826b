"""Gradient of the SES alpha-FTP's final radius with respect to the points, FP64.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline may import this package; the library never does.

The function differentiated is the alpha-FTP of Sec. 3 (Theorem 2) for SES
(Sec. 4.1) at a fixed alpha and a fixed eta/rho, run for T iterations from
t = 0, followed by the radius of Sec. 5 at the final running mean:

    L(V) = f(ubar^T),   f(c) = max_i ||c - v_i|| + gamma_i.

Each iteration is written in the paper's order with plain PyTorch CPU ops in
float64: the accumulated exponent X_i = -(eta t/rho)(ubar - v_i; alpha -
gamma_i) of Eq. (implement), its SOC spectral decomposition and Loewner
exponential (Sec. 2.1), the normalisation p = exp(X)/Tr exp(X) (Eq. SCMWU),
the ORACLE's maximiser u = v_1 + (alpha - gamma_1) g/||g|| with g = sum_i w_i
(Eq. ses_oracle; u = v_1 when g = 0, the reading taken in ses.py), and the
running mean ubar^{t+1} = ubar^t + (u - ubar^t)/(t+1). Reverse-mode automatic
differentiation of that program (a library primitive, like a matmul) gives
dL/dV. The largest eigenvalue is subtracted before exponentiating, as in
eja.scmwu_soc; the shift cancels in p.

Pinned in tests/test_oracle_grad.py against: central finite differences of
the independent numpy forward (ses.ses_step), the closed forms at T = 1 and at
n = 2, and the value of the forward itself.
"""

import math

import numpy as np
import torch

SQRT2 = math.sqrt(2.0)


def ses_unrolled_radius(V, gamma, alpha, eta_over_rho, T):
    """L = f(ubar^T) as a differentiable function of V ((n, d) float64 tensor).

    Returns (L, ubar^T, steps): the iterations stop early, as ses.ses_ftp does,
    when the ORACLE value is negative (separation); steps counts those taken.
    """
    n, d = V.shape
    gm = torch.zeros(n, dtype=torch.float64) if gamma is None else torch.as_tensor(gamma, dtype=torch.float64)
    v1, cones = V[0], V[1:]
    a = alpha - gm[1:]
    ubar = v1
    steps = 0
    for t in range(T):
        k = eta_over_rho * t
        # exponent of Eq. (implement): vector part -k (ubar - v_i), scalar part -k (alpha - gamma_i)
        xv = -k * (ubar[None, :] - cones)
        x0 = -k * a
        # spectral decomposition (Sec. 2.1): lambda_{1,2} = (x0 +- ||xv||)/sqrt2
        if t == 0:
            # X = 0: exp(X) = e, p = e/r, g = 0 and the ORACLE returns u = v_1
            w = torch.zeros_like(cones)
            s = torch.full((n - 1,), 1.0 / (SQRT2 * (n - 1)), dtype=torch.float64)
        else:
            nx = torch.sqrt(torch.sum(xv * xv, dim=1))
            lam1 = (x0 + nx) / SQRT2
            lam2 = (x0 - nx) / SQRT2
            M = torch.max(lam1).detach()
            e1, e2 = torch.exp(lam1 - M), torch.exp(lam2 - M)
            # exp(X_i) = e1 q1 + e2 q2, q_{1,2} = (1/sqrt2)(+-xv/||xv||; 1)
            xhat = xv / nx[:, None]
            ev = (e1 - e2)[:, None] * xhat / SQRT2
            e0 = (e1 + e2) / SQRT2
            C = torch.sum(SQRT2 * e0)  # Tr exp(X) summed over the cones
            w, s = ev / C, e0 / C
        g = torch.sum(w, dim=0)
        ng = torch.sqrt(torch.sum(g * g))
        u = v1 if t == 0 or float(ng.detach()) == 0.0 else v1 + (alpha - gm[0]) * g / ng
        # ORACLE value of Eq. (ses_oracle): g^T u + gamma/sqrt2 - sum v_i^T w_i - sum gamma_i s_i
        value = torch.dot(g, u) + alpha / SQRT2 - torch.sum(cones * w) - torch.sum(gm[1:] * s)
        if float(value.detach()) < 0.0:
            break
        ubar = ubar + (u - ubar) / (t + 1)
        steps += 1
    # f = max_i; its (sub)gradient flows through the row attaining the maximum
    # (the smallest index on ties)
    with torch.no_grad():
        dist = torch.sqrt(torch.sum((ubar[None, :] - V) ** 2, dim=1)) + gm
        top = int(np.argmax(dist.numpy()))
    L = torch.sqrt(torch.sum((ubar - V[top]) ** 2)) + gm[top]
    return L, ubar, steps


def ses_unrolled_radius_grad(V, gamma, alpha, eta_over_rho, T):
    """(L, dL/dV as an (n, d) float64 numpy array, steps taken)."""
    Vt = torch.tensor(np.asarray(V, dtype=np.float64), requires_grad=True)
    L, _, steps = ses_unrolled_radius(Vt, gamma, alpha, eta_over_rho, T)
    L.backward()
    return float(L.detach()), Vt.grad.numpy().copy(), steps
