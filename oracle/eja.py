"""Euclidean Jordan algebra primitives (Sec. 2.1), FP64.

Layout. An element (u; u0) of the second-order-cone algebra R^{d+1} is stored
as a float64 array whose LAST entry is the scalar part u0 and whose first d
entries are the vector part u. A product of m such algebras (Sec. 2.1,
"Product cones") is an (m, d+1) array, one row per component.

Second-order cone Q^{d+1} (Sec. 2.1):
  product   (u; u0) o (v; v0) = (1/sqrt2) (v0 u + u0 v ; u^T v + u0 v0)
  identity  e = (0; sqrt2), rank 2
  spectrum  lambda_{1,2} = (u0 +- ||u||) / sqrt2,
            q_{1,2} = (1/sqrt2) (+-u/||u|| ; 1)   (any unit vector if u = 0)
  trace     Tr(u; u0) = sqrt2 u0 = lambda_1 + lambda_2
  inner     x . y = Tr(x o y)
Non-negative orthant R^n_+ (Sec. 2.1): componentwise product, e = 1, trace =
sum, spectral decomposition x = sum_i x_i e_i.
Loewner extension of exp (Sec. 2.1): exp(sum lambda_i q_i) = sum e^{lambda_i} q_i.
"""

import numpy as np

SQRT2 = np.sqrt(2.0)


# ----------------------------------------------------------------- SOC algebra
def soc_identity(d):
    """Identity element e = (0; sqrt2) of the SOC algebra R^{d+1} (Sec. 2.1)."""
    e = np.zeros(d + 1)
    e[-1] = SQRT2
    return e


def soc_product(x, y):
    """Jordan product of SOC elements, row-wise for (m, d+1) arrays (Sec. 2.1)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    u, u0 = x[..., :-1], x[..., -1:]
    v, v0 = y[..., :-1], y[..., -1:]
    vec = (v0 * u + u0 * v) / SQRT2
    sca = (np.sum(u * v, axis=-1, keepdims=True) + u0 * v0) / SQRT2
    return np.concatenate([vec, sca], axis=-1)


def soc_trace(x):
    """Tr(u; u0) = sqrt2 * u0 (Sec. 2.1)."""
    return SQRT2 * np.asarray(x, dtype=np.float64)[..., -1]


def soc_inner(x, y):
    """EJA inner product x . y = Tr(x o y) (Sec. 2.1)."""
    return soc_trace(soc_product(x, y))


def soc_spectral(x):
    """Spectral decomposition of SOC elements (Sec. 2.1).

    Returns (lam1, lam2, q1, q2) with lam_{1,2} = (u0 +- ||u||)/sqrt2 and
    q_{1,2} = (1/sqrt2)(+-u/||u||; 1). Where u = 0 the unit vector is taken to
    be the first standard basis vector (the paper allows any unit vector).
    Works row-wise on (m, d+1) arrays.
    """
    x = np.asarray(x, dtype=np.float64)
    u, u0 = x[..., :-1], x[..., -1]
    nu = np.sqrt(np.sum(u * u, axis=-1))
    lam1 = (u0 + nu) / SQRT2
    lam2 = (u0 - nu) / SQRT2
    vhat = np.zeros_like(u)
    nz = nu > 0
    vhat[nz] = u[nz] / nu[nz][..., None]
    vhat[~nz, 0] = 1.0
    ones = np.ones(u.shape[:-1] + (1,))
    q1 = np.concatenate([vhat, ones], axis=-1) / SQRT2
    q2 = np.concatenate([-vhat, ones], axis=-1) / SQRT2
    return lam1, lam2, q1, q2


def soc_exp(x):
    """Loewner exponential exp(x) = e^{lam1} q1 + e^{lam2} q2 (Sec. 2.1)."""
    lam1, lam2, q1, q2 = soc_spectral(x)
    return np.exp(lam1)[..., None] * q1 + np.exp(lam2)[..., None] * q2


def soc_in_cone(x, tol=0.0):
    """Membership in Q^{d+1} = {(u; u0): ||u|| <= u0} (Sec. 2.1), row-wise."""
    x = np.asarray(x, dtype=np.float64)
    return np.sqrt(np.sum(x[..., :-1] ** 2, axis=-1)) <= x[..., -1] + tol


def soc_lambda_min(x):
    """Smallest eigenvalue (u0 - ||u||)/sqrt2 of each SOC component (Sec. 2.1)."""
    return soc_spectral(x)[1]


def soc_inf_norm(x):
    """||x||_inf = max_i |lambda_i| over all components (Sec. 2.1)."""
    lam1, lam2, _, _ = soc_spectral(x)
    return float(np.max(np.maximum(np.abs(lam1), np.abs(lam2))))


# ------------------------------------------------------- SCMWU on product cones
def scmwu_soc(X):
    """SCMWU normalisation p = exp(X) / Tr(exp(X)) over a product of SOCs.

    ``X`` is the (m, d+1) array of the accumulated, already scaled exponent
    -eta * sum_tau m^tau (Eq. SCMWU; with the running-mean form of Eq.
    (implement)). The exponential is taken per component from its spectral
    decomposition (Sec. 2.1, product cones) and the trace of the product is the
    sum of the components' traces.

    Before exponentiating, every eigenvalue is shifted by the largest one, M:
    exp(X - M e) = e^{-M} exp(X) because e commutes with everything, so the
    normalised result is unchanged in exact arithmetic and no term overflows.
    Returns (P, C_shifted, M) with P the (m, d+1) trace-one weights.
    """
    lam1, lam2, q1, q2 = soc_spectral(X)
    M = max(float(np.max(lam1)), float(np.max(lam2)))
    e1 = np.exp(lam1 - M)
    e2 = np.exp(lam2 - M)
    W = e1[:, None] * q1 + e2[:, None] * q2
    C = float(np.sum(soc_trace(W)))
    return W / C, C, M


def scmwu_orthant(x):
    """SCMWU normalisation over R^n_+: p = exp(x)/sum(exp(x)) (Sec. 2.1, 2.3).

    Same exact max-shift as :func:`scmwu_soc`. Returns (p, C_shifted, M).
    """
    x = np.asarray(x, dtype=np.float64)
    M = float(np.max(x))
    w = np.exp(x - M)
    C = float(np.sum(w))
    return w / C, C, M
