"""Exact solvers for tiny inputs, used only to pin the MWU oracle.

None of these is the paper's method. They are textbook algorithms that the
paper names as the exact alternatives (Sec. 4.1 cites Welzl's randomised
algorithm among the exact SES methods; Sec. 4.2 relates hard-margin SVM to the
polytope-distance problem PD), written out plainly in FP64.

  mec_2d            minimum enclosing circle of points in the plane by the
                    randomised incremental algorithm of Welzl (1991).
  meb_bruteforce    minimum enclosing ball in any dimension by enumerating
                    support sets of at most d+1 points (Carathéodory: the
                    optimal ball is the circumscribed ball of such a set,
                    centred in its affine hull).
  pd_bruteforce     polytope distance min ||P mu - Q gamma|| over the two
                    simplices by enumerating pairs of supports (at most d+1
                    points in total) and solving each affine least-distance
                    problem from its KKT system.
  pd_mdm            the same problem for sets of any size by the
                    Mitchell-Dem'yanov-Malozemov descent (1974), which the
                    paper names among the geometric PD methods (Sec. 4.2):
                    the core-set certificates of the SVM search solve it on a core set.
"""

import itertools
import math

import numpy as np


def _circle2(a, b):
    c = (a + b) / 2.0
    return c, float(np.linalg.norm(a - c))


def _circle3(a, b, c):
    # circumcircle of three points; collinear -> the widest two-point circle
    ax, ay = a
    bx, by = b
    cx, cy = c
    den = 2.0 * (ax * (by - cy) + bx * (cy - ay) + cx * (ay - by))
    if abs(den) < 1e-300:
        best = None
        for p, q in ((a, b), (a, c), (b, c)):
            cc, rr = _circle2(p, q)
            if best is None or rr > best[1]:
                best = (cc, rr)
        return best
    a2, b2, c2 = ax * ax + ay * ay, bx * bx + by * by, cx * cx + cy * cy
    ux = (a2 * (by - cy) + b2 * (cy - ay) + c2 * (ay - by)) / den
    uy = (a2 * (cx - bx) + b2 * (ax - cx) + c2 * (bx - ax)) / den
    ctr = np.array([ux, uy])
    return ctr, float(np.linalg.norm(a - ctr))


def mec_2d(points, seed=0, rel_tol=1e-12):
    """Minimum enclosing circle (centre, radius) by Welzl's randomised
    incremental algorithm, expected O(n)."""
    P = np.array(points, dtype=np.float64)
    if P.ndim != 2 or P.shape[1] != 2 or P.shape[0] == 0:
        raise ValueError("mec_2d needs an (n, 2) array")
    P = P[np.random.default_rng(seed).permutation(P.shape[0])]
    n = P.shape[0]

    def outside(p, c, r):
        return np.linalg.norm(p - c) > r * (1.0 + rel_tol) + 1e-300

    c, r = P[0].copy(), 0.0
    for i in range(1, n):
        if outside(P[i], c, r):
            c, r = P[i].copy(), 0.0
            for j in range(i):
                if outside(P[j], c, r):
                    c, r = _circle2(P[i], P[j])
                    for k in range(j):
                        if outside(P[k], c, r):
                            c, r = _circle3(P[i], P[j], P[k])
    return c, r


def _circumball(S):
    """Ball through all points of S with centre in their affine hull, or None."""
    p0 = S[0]
    if len(S) == 1:
        return p0.copy(), 0.0
    A = S[1:] - p0                       # (m, d)
    G = A @ A.T                           # Gram matrix
    rhs = 0.5 * np.sum(A * A, axis=1)
    try:
        lam = np.linalg.solve(G, rhs)
    except np.linalg.LinAlgError:
        return None
    c = p0 + lam @ A
    return c, float(np.linalg.norm(S[0] - c))


def meb_bruteforce(points, rel_tol=1e-9):
    """Minimum enclosing ball (centre, radius) of a small point set in R^d."""
    P = np.asarray(points, dtype=np.float64)
    n, d = P.shape
    best = None
    for m in range(1, min(n, d + 1) + 1):
        for idx in itertools.combinations(range(n), m):
            cb = _circumball(P[list(idx)])
            if cb is None:
                continue
            c, r = cb
            if np.all(np.linalg.norm(P - c, axis=1) <= r * (1.0 + rel_tol) + 1e-12):
                if best is None or r < best[1]:
                    best = (c, r)
    return best


def _affine_distance(A, B):
    """min ||A^T a - B^T b|| s.t. sum a = 1, sum b = 1 (no sign constraint).

    KKT of the equality-constrained least squares; returns (a, b, dist) or None.
    """
    ma, mb = A.shape[0], B.shape[0]
    M = np.concatenate([A, -B], axis=0)          # rows: +a_i, -b_j
    H = M @ M.T
    E = np.zeros((2, ma + mb))
    E[0, :ma] = 1.0
    E[1, ma:] = 1.0
    K = np.block([[H, E.T], [E, np.zeros((2, 2))]])
    rhs = np.concatenate([np.zeros(ma + mb), [1.0, 1.0]])
    try:
        sol = np.linalg.solve(K, rhs)
    except np.linalg.LinAlgError:
        sol = np.linalg.lstsq(K, rhs, rcond=None)[0]
    coef = sol[: ma + mb]
    x = coef @ M
    if not np.allclose(K @ sol, rhs, atol=1e-9):
        return None
    return coef[:ma], coef[ma:], float(np.linalg.norm(x))


def pd_bruteforce(P, Q, tol=1e-12):
    """Polytope distance min ||P mu - Q gamma|| over simplices (Eq. PD) for tiny
    inputs; P and Q are (n1, d) and (n2, d). Returns (dist, mu, gamma)."""
    P = np.asarray(P, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    d = P.shape[1]
    best = None
    for k1 in range(1, min(P.shape[0], d + 1) + 1):
        for k2 in range(1, min(Q.shape[0], d + 2 - k1) + 1):
            for I in itertools.combinations(range(P.shape[0]), k1):
                for J in itertools.combinations(range(Q.shape[0]), k2):
                    res = _affine_distance(P[list(I)], Q[list(J)])
                    if res is None:
                        continue
                    a, b, dist = res
                    if np.all(a >= -tol) and np.all(b >= -tol):
                        if best is None or dist < best[0]:
                            mu = np.zeros(P.shape[0])
                            ga = np.zeros(Q.shape[0])
                            mu[list(I)] = a
                            ga[list(J)] = b
                            best = (dist, mu, ga)
    return best


def svm_margin_of(P, Q, w):
    """Margin (min_P x^T w - max_Q x^T w)/||w|| of a direction w (Eq. SVM)."""
    w = np.asarray(w, dtype=np.float64)
    nw = math.sqrt(float(w @ w))
    return (float(np.min(P @ w)) - float(np.max(Q @ w))) / nw


def pd_mdm(P, Q, tol=1e-12, max_iter=1_000_000):
    """Polytope distance min ||P^T mu - Q^T gamma|| over the two simplices
    (Eq. PD; P, Q are (n1, d) and (n2, d) arrays of points) by the descent of
    Mitchell, Dem'yanov and Malozemov.

    With z = P^T mu - Q^T gamma and the projections s_i = p_i . z, t_j =
    q_j . z: z . z = sum mu_i s_i - sum gamma_j t_j >= min_i s_i - max_j t_j,
    with equality at the optimum, so gap = z . z - (min s - max t) >= 0
    certifies the iterate (the margin of z is (min s - max t)/||z|| <= OPT <=
    ||z||). A step moves weight within one simplex, from the support point
    that is worst along z to the point that is best (P: from the largest s to
    the smallest; Q: from the smallest t to the largest), in the set where
    that difference is larger, by the step that minimises ||z|| (at most all
    of the moved point's weight). Stops when gap <= tol z . z.

    Returns (dist, mu, gamma, gap, iterations); dist = ||z|| recomputed from
    the weights."""
    P = np.asarray(P, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    mu = np.zeros(P.shape[0])
    ga = np.zeros(Q.shape[0])
    # start: the pair closest along the difference of the centroids
    c = P.mean(axis=0) - Q.mean(axis=0)
    mu[int(np.argmin(P @ c))] = 1.0
    ga[int(np.argmax(Q @ c))] = 1.0
    z = P.T @ mu - Q.T @ ga
    gap = math.inf
    it = 0
    for it in range(max_iter):
        s, tq = P @ z, Q @ z
        zz = float(z @ z)
        b, e = int(np.argmin(s)), int(np.argmax(tq))
        gap = zz - (s[b] - tq[e])
        if gap <= tol * zz:
            break
        supp = np.nonzero(mu > 0.0)[0]
        a = int(supp[np.argmax(s[supp])])
        suppq = np.nonzero(ga > 0.0)[0]
        cq = int(suppq[np.argmin(tq[suppq])])
        if s[a] - s[b] >= tq[e] - tq[cq]:
            v, lim = P[b] - P[a], mu[a]
        else:
            v, lim = Q[cq] - Q[e], ga[cq]
        vv = float(v @ v)
        lam = min(lim, max(0.0, -float(z @ v) / vv)) if vv > 0.0 else 0.0
        if lam <= 0.0:
            break
        if s[a] - s[b] >= tq[e] - tq[cq]:
            mu[a] -= lam
            mu[b] += lam
        else:
            ga[cq] -= lam
            ga[e] += lam
        z = z + lam * v
    mu = np.maximum(mu, 0.0)
    ga = np.maximum(ga, 0.0)
    mu /= mu.sum()
    ga /= ga.sum()
    z = P.T @ mu - Q.T @ ga
    return math.sqrt(float(z @ z)), mu, ga, gap, it
