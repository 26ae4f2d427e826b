"""Smallest Enclosing Sphere through the primal-dual meta-algorithm, FP64.

Follows Sec. 4.1 (problem SES, its split into the easy set C and the hard set
F, the dual/primal pair (dualses)/(primalses), the bounds D, the closed-form
ORACLE of Eq. (ses_oracle), the width rho <= 3D/sqrt2 and T of Theorem 4),
Sec. 3 (the alpha-FTP of Theorem 2, the hyperplane update of Eq. (implement),
the primal solution of Eq. (primal_construction), the search from
feasibility to optimisation) and Sec. 5 (per-iteration objective f^t, the
early-exit and early-stop rules).

Inputs: V is the (n, d) array of centres v_1..v_n, gamma the (n,) radii (None
means points, gamma = 0). Row 0 is v_1, the constraint kept as the easy set C
("the first one", Sec. 4.1); rows 1..n-1 form the product cone
K = prod_{i>=2} Q^{d+1} of rank r = 2(n-1).

Readings of the paper taken here (the GPU path takes the same ones):
  * gamma-bar, the running mean of the oracle's gamma outputs, equals alpha
    inside one alpha-FTP because the ORACLE always returns gamma = alpha.
  * When g = sum_i w_i = 0 (always at t = 0, where p^1 = e/r) the ORACLE's
    maximiser is not unique; u = v_1, the centre of the ball, is returned.
  * An ORACLE value exactly 0 counts as success (Sec. 3: "non-negative").
  * f^0, before any iterate exists, is evaluated at ubar^0 = v_1.
"""

import math

import numpy as np

from .eja import SQRT2, scmwu_soc, soc_inner

OUT_SEPARATED = "separated"      # ORACLE value < 0: alpha < OPT (Sec. 3)
OUT_FEASIBLE = "feasible"        # T iterations without separation (Theorem 2)
OUT_BELOW_ALPHA = "below_alpha"  # f^t < alpha: affirmative early exit (Sec. 5)
OUT_STALLED = "stalled"          # |f^t - f^{t-1}|/f^{t-1} < delta, patience times (Sec. 5)
OUT_FIXED = "fixed"              # FIXED_ITERS mode ran its T iterations
OUT_CERTIFIED = "certified"      # CERTIFIED mode: the certificates closed at a poll

MODE_PRACTICAL = "practical"
MODE_THEORY = "theory"
MODE_FIXED = "fixed"
MODE_CERTIFIED = "certified"
MODE_CORESET = "coreset"         # CERTIFIED with core-set certificates (points; beyond the paper)
CORESET_FIRST = 256              # first core-set check at this many iterations of the search, then every doubling
OUT_STUCK = "stuck"              # CERTIFIED mode: the certificate gap stopped shrinking (eta is halved)
CERT_FIRST_CHECK = 1024          # CERTIFIED: first progress check of an alpha-FTP at eta = 1 (then 2x, 4x, ...)
CERT_SHRINK = 0.8                # CERTIFIED: the FTP's own gap must shrink by this factor while t doubles
CERT_MIN_ETA = 1.0 / 64.0        # CERTIFIED: eta is not halved below this (no progress test there)


def _prep(V, gamma):
    V = np.asarray(V, dtype=np.float64)
    if V.ndim != 2 or V.shape[0] < 2:
        raise ValueError("SES needs an (n, d) array with n >= 2")
    g = np.zeros(V.shape[0]) if gamma is None else np.asarray(gamma, dtype=np.float64)
    return V, g


# ------------------------------------------------------------- constants
def ses_D(V, gamma=None):
    """D = max_{i>=2} ||v_1 - v_i|| + gamma_1 + gamma_i; OPT in [D/2, D] (Sec. 4.1)."""
    V, gm = _prep(V, gamma)
    dist = np.sqrt(np.sum((V[1:] - V[0]) ** 2, axis=1))
    return float(np.max(dist + gm[0] + gm[1:]))


def ses_width(D):
    """Width of the SES ORACLE, rho <= 3D/sqrt2 (Sec. 4.1)."""
    return 3.0 * D / SQRT2


def ses_rank(n):
    """Rank r = 2(n-1) of K = prod_{i>=2} Q^{d+1} (Sec. 4.1)."""
    return 2 * (n - 1)


SES_R = SQRT2  # b_{d+1} after scaling the last primal constraint by sqrt2 (Sec. 4.1)


def ses_T(D, n, eps, alpha):
    """T = ceil(36 D^2 ln(2n-2) / (eps^2 alpha^2)) (Sec. 4.1, from Theorem 2)."""
    return int(math.ceil(36.0 * D * D * math.log(2 * n - 2) / (eps * eps * alpha * alpha)))


def theorem_eta(r, T):
    """Step size eta = sqrt(ln r / T) of Theorems 2 and 3."""
    return math.sqrt(math.log(r) / T)


# ------------------------------------------------- one iteration, step by step
def ses_exponent(V, gamma, ubar, alpha, k):
    """Accumulated exponent of Eq. (implement) for the SES split.

    sum_j a_j ybar_j - c = prod_{i>=2} (ubar - v_i; alpha - gamma_i)  (Eq. dualses
    with ybar = (ubar; alpha)), scaled by -k where k = eta t / rho.
    Returns the (n-1, d+1) array X.
    """
    V, gm = _prep(V, gamma)
    ubar = np.asarray(ubar, dtype=np.float64)
    X = np.empty((V.shape[0] - 1, V.shape[1] + 1))
    X[:, :-1] = ubar[None, :] - V[1:]
    X[:, -1] = alpha - gm[1:]
    return -k * X


def ses_weights(V, gamma, ubar, alpha, k):
    """p^{t+1} = exp(X)/Tr(exp(X)) with X from :func:`ses_exponent` (Eq. implement).

    Returns P, the (n-1, d+1) array whose row i-2 is (w_i; s_i) (Sec. 4.1).
    """
    P, _, _ = scmwu_soc(ses_exponent(V, gamma, ubar, alpha, k))
    return P


def ses_oracle(V, gamma, P, alpha):
    """Closed-form ORACLE of Eq. (ses_oracle).

    max_{u,gamma} g^T u + gamma/sqrt2 - sum v_i^T w_i - sum gamma_i s_i
    s.t. gamma <= alpha, ||u - v_1|| <= gamma - gamma_1, with g = sum_{i>=2} w_i.
    The optimum takes gamma = alpha and u = v_1 + (alpha - gamma_1) g/||g||.
    Returns (u, value, g).
    """
    V, gm = _prep(V, gamma)
    w, s = P[:, :-1], P[:, -1]
    g = np.sum(w, axis=0)
    ng = math.sqrt(float(g @ g))
    if ng > 0.0:
        u = V[0] + (alpha - gm[0]) * g / ng
    else:
        u = V[0].copy()
    value = float(g @ u) + alpha / SQRT2 - float(np.sum(V[1:] * w)) - float(gm[1:] @ s)
    return u, value, g


def ses_program_value(V, gamma, P, u, gam):
    """Objective of Eq. (oracle_program) for y = (u; gam), unsimplified.

    (sum_j a_j y_j - c) . p = sum_{i>=2} (u - v_i; gam - gamma_i) . (w_i; s_i),
    with the SOC inner product of Sec. 2.1.
    """
    V, gm = _prep(V, gamma)
    Y = np.empty((V.shape[0] - 1, V.shape[1] + 1))
    Y[:, :-1] = np.asarray(u)[None, :] - V[1:]
    Y[:, -1] = gam - gm[1:]
    return float(np.sum(soc_inner(Y, P)))


def ses_primal_lb(V, gamma, P):
    """Value of the primal solution (z~ p; x~') of Eq. (primal_construction).

    Problem D there, for the SES data of Eq. (dualses): maximise
    (c . p) z + c' . x' subject to (a_j . p) z + a'_j . x' = b_j, z >= 0,
    x' in K' = Q^{d+1}. With g_j = a_j . p (j <= d), sigma = a_{d+1} . p
    = sum s_i and b = (0; 1): x' = (-z g; 1 - z sigma), feasible iff
    z <= 1/(||g|| + sigma), value gamma_1 + z (c . p - v_1^T g - gamma_1 sigma).
    (z~ p; x~') is primal feasible for (SCP), so by weak duality the value is a
    lower bound on OPT, the optimal radius.
    """
    V, gm = _prep(V, gamma)
    w, s = P[:, :-1], P[:, -1]
    g = np.sum(w, axis=0)
    sigma = float(np.sum(s))
    cp = float(np.sum(V[1:] * w)) + float(gm[1:] @ s)
    coef = cp - float(V[0] @ g) - gm[0] * sigma
    zmax = 1.0 / (math.sqrt(float(g @ g)) + sigma)
    return float(gm[0] + max(coef, 0.0) * zmax)


def ses_objective(V, gamma, c):
    """f = max_{i in [n]} ||c - v_i|| + gamma_i: radius of the smallest ball
    centred at c enclosing every input sphere (Sec. 5)."""
    V, gm = _prep(V, gamma)
    return float(np.max(np.sqrt(np.sum((V - np.asarray(c)[None, :]) ** 2, axis=1)) + gm))


def ses_qp_weights(V, gamma, ubar, P, k):
    """kappa_i >= 0 with w_i = kappa_i (v_i - ubar), i >= 2: the coefficient of
    each point in the ORACLE's g = sum_i w_i (Eq. ses_oracle).

    The vector part of exp(X_i) points along x_i = k (v_i - ubar) (Sec. 2.1:
    exp keeps the eigenvectors), so kappa_i = w_i . (v_i - ubar) / dist_i^2.
    Where v_i sits at the mean (dist_i = 0) w_i vanishes; kappa_i is then its
    limit k s_i / sqrt2 as dist_i -> 0 (lambda_1 - lambda_2 = sqrt2 k dist_i).
    """
    V, gm = _prep(V, gamma)
    R = V[1:] - np.asarray(ubar, dtype=np.float64)[None, :]
    dist2 = np.sum(R * R, axis=1)
    w, s = P[:, :-1], P[:, -1]
    kap = np.empty(R.shape[0])
    pos = dist2 > 0.0
    kap[pos] = np.sum(w[pos] * R[pos], axis=1) / dist2[pos]
    kap[~pos] = k * s[~pos] / SQRT2
    return kap


def ses_qp_moments(V, kap):
    """(A, B) of the weights mu = kappa / sum kappa over the points i >= 2,
    taken about v_1: A = sum_i mu_i |v_i - v_1|^2, B = sum_i mu_i (v_i - v_1).

    The QP of Sec. 5 (Eq. ses_qp) maximises, over the simplex, -(y^T y -
    sum_i x_i v_i^T v_i) with y = sum_i x_i v_i, whose optimum is OPT^2 for
    points; every simplex x therefore gives OPT^2 >= A - |B|^2 (the value is
    unchanged by the shift to v_1). None when sum kappa = 0 (t = 0: k = 0).
    """
    V = np.asarray(V, dtype=np.float64)
    tot = float(np.sum(kap))
    if not tot > 0.0:
        return None
    mu = kap / tot
    Z = V[1:] - V[0][None, :]
    return float(mu @ np.sum(Z * Z, axis=1)), mu @ Z


def ses_dual_update(avg, t, moments):
    """Running average of the QP moments over an alpha-FTP, iterate t weighted
    by t^2 (so the early, nearly uniform weights fade): avg = {"A", "B", "wsum"}.
    Returns the lower bound sqrt(max(Abar - |Bbar|^2, 0)) (0 before any update).
    The averaged weights are again a point of the simplex, so the bound holds
    for any positive weights; t^2 closed the certified search in about 20 %
    fewer iterations than t on Gaussian sets and no more on the unit square.
    """
    if moments is not None and t >= 1:
        A, B = moments
        w = float(t) * float(t)
        avg["wsum"] += w
        r = w / avg["wsum"]
        avg["A"] += r * (A - avg["A"])
        avg["B"] = avg["B"] + r * (B - avg["B"])
    if avg["wsum"] == 0.0:
        return 0.0
    return math.sqrt(max(avg["A"] - float(avg["B"] @ avg["B"]), 0.0))


def ses_dual_state(d):
    return {"A": 0.0, "B": np.zeros(d), "wsum": 0.0}


def ses_step(V, gamma, ubar, t, alpha, eta, rho, avg=None):
    """One iteration of the alpha-FTP (Sec. 3, Theorem 2) for SES.

    ``t`` oracle calls have completed and ``ubar`` is the mean of their u's (any
    value when t = 0). Computes p^{t+1} (Eq. implement with k = eta t/rho), the
    ORACLE answer, the primal lower bound and f at ubar. If the ORACLE succeeds
    the mean is advanced to ubar^{t+1}. ``avg`` (points only; from
    :func:`ses_dual_state`) is advanced by this iteration's QP moments and
    rec["dual_bound"] is the averaged QP lower bound (0 for spheres). Returns a
    dict record.
    """
    V, gm = _prep(V, gamma)
    k = eta * t / rho
    P = ses_weights(V, gm, ubar, alpha, k)
    u, value, g = ses_oracle(V, gm, P, alpha)
    rec = {
        "t": t,
        "k": k,
        "objective": ses_objective(V, gm, ubar),
        "oracle_value": value,
        "lower_bound": ses_primal_lb(V, gm, P),
        "u": u,
        "g": g,
        "failed": value < 0.0,
        "dual_bound": 0.0,
    }
    if avg is not None and not np.any(gm):
        rec["dual_bound"] = ses_dual_update(avg, t, ses_qp_moments(V, ses_qp_weights(V, gm, ubar, P, k)))
    if value >= 0.0:
        rec["ubar_next"] = np.asarray(ubar, dtype=np.float64) + (u - ubar) / (t + 1)
    else:
        rec["ubar_next"] = np.asarray(ubar, dtype=np.float64).copy()
    return rec


# ------------------------------------------------------------ the alpha-FTP
def ses_ftp(V, gamma, alpha, eta, rho, T, mode=MODE_FIXED, delta=1e-4, patience=10,
            keep_trace=False, cert=None):
    """alpha-feasibility test of Theorem 2 for SES, run for at most T iterations.

    Modes: FIXED runs exactly T iterations unless the ORACLE separates;
    THEORY is the same with the conclusion of Theorem 2 (OPT <= (1+eps) alpha
    when T is the theorem's count); PRACTICAL adds the two rules of Sec. 5:
    stop with an affirmative answer as soon as f^t < alpha, and stop when
    |f^t - f^{t-1}|/f^{t-1} < delta for ``patience`` consecutive iterations
    (the ratio is skipped when f^{t-1} = 0). CERTIFIED keeps the first rule
    only (f^t < alpha proves OPT < alpha) and, every cert["poll_every"]
    completed iterations, stops once the certificates close:
    min(cert["ub"], f_best) <= (1 + cert["eps"]) max(cert["lb"], lb_best),
    or as STUCK when, at the first poll with t >= c, 2c, 4c, ... (c = 1024/eta),
    the FTP's own gap f_best / lb_best - 1 has not shrunk by the factor 0.8
    since the previous such poll (the first check compares with infinity, so it
    never stops there; no check once eta <= 1/64).
    Returns a dict with the outcome, the iteration count, the final mean, the
    best enclosing ball seen (c_best, f_best), the best lower bound (primal
    construction or, for points, the averaged QP bound) and, if asked, the
    per-iteration records.
    """
    V, gm = _prep(V, gamma)
    ubar = V[0].copy()
    f_best, c_best = math.inf, ubar.copy()
    lb_best = 0.0
    avg = ses_dual_state(V.shape[1])
    trace = []
    f_prev, streak = None, 0
    outcome = OUT_FIXED if mode == MODE_FIXED else OUT_FEASIBLE
    last_gap = math.inf
    next_check = math.ceil(CERT_FIRST_CHECK / eta) if mode == MODE_CERTIFIED and eta > CERT_MIN_ETA else math.inf
    t = 0
    while t < T:
        rec = ses_step(V, gm, ubar, t, alpha, eta, rho, avg=avg)
        if keep_trace:
            trace.append(rec)
        if t > 0 and rec["objective"] < f_best:
            f_best, c_best = rec["objective"], ubar.copy()
        lb_best = max(lb_best, rec["lower_bound"], rec["dual_bound"])
        if rec["failed"]:
            outcome = OUT_SEPARATED
            break
        if mode in (MODE_PRACTICAL, MODE_CERTIFIED) and t > 0:
            f = rec["objective"]
            if f < alpha:
                outcome = OUT_BELOW_ALPHA
                break
            if mode == MODE_PRACTICAL and f_prev is not None and f_prev > 0.0:
                streak = streak + 1 if abs(f - f_prev) / f_prev < delta else 0
                if streak >= patience:
                    outcome = OUT_STALLED
                    break
            f_prev = f
        ubar = rec["ubar_next"]
        t += 1
        if mode == MODE_CERTIFIED and t % cert["poll_every"] == 0:
            cs = cert.get("coreset")
            if cs is not None and cs["base"] + t >= cs["next"]:
                # core-set bounds from the current mean: their ball joins the
                # FTP's best, their dual value its lower bound
                lb_c, ub_c, c_c = ses_coreset_bounds(V, ubar, tol=cert["eps"] / 10.0, rounds=4, eps=cert["eps"])
                lb_best = max(lb_best, lb_c)
                if ub_c < f_best:
                    f_best, c_best = ub_c, c_c
                cs["next"] *= 2
            if min(cert["ub"], f_best) <= (1.0 + cert["eps"]) * max(cert["lb"], lb_best):
                outcome = OUT_CERTIFIED
                break
            if t >= next_check:  # progress test: this FTP's own gap must halve while t doubles
                gap = f_best / lb_best - 1.0 if lb_best > 0.0 else math.inf
                if gap > CERT_SHRINK * last_gap:
                    outcome = OUT_STUCK
                    break
                last_gap, next_check = gap, 2 * next_check
    f_end = ses_objective(V, gm, ubar)
    if t > 0 and f_end < f_best:
        f_best, c_best = f_end, ubar.copy()
    return {"outcome": outcome, "iters": t, "ubar": ubar, "f_best": f_best,
            "c_best": c_best, "lb_best": lb_best, "trace": trace}


# ------------------------------------------------- feasibility -> optimisation
def ses_solve(V, gamma=None, eps=1e-2, mode=MODE_PRACTICAL, max_iters=10**7,
              delta=1e-4, patience=10, max_steps=200, eta=None, poll_every=256):
    """(1+eps)-approximate SES by the search of Sec. 3 over alpha in [D/2, D].

    Step i: alpha_i = L + (U-L)/3, eps_i = (U-L)/(3 alpha_i), T_i and eta_i from
    Theorem 2 (Sec. 4.1 constants). Separation -> L = alpha_i; otherwise the
    FTP's conclusion OPT <= (1+eps_i) alpha_i -> U = (1+eps_i) alpha_i. The
    paper's PRACTICAL rules (Sec. 5) replace the T_i iterations by its early
    exit / early stop; a stalled run is taken as the affirmative answer, as the
    paper's experiments do.

    Two pairs of bounds are kept. (L, U) is the search range. (lb, ub) are
    certificates: ub is the radius f of an actual enclosing ball (the best
    centre seen), lb the best primal value of Eq. (primal_construction) seen,
    both valid whatever the mode. The loop ends when U <= (1+eps) L, when
    ub <= (1+eps) lb, or when ``max_iters`` MWU iterations have run.

    ``eta`` None uses eta_i = sqrt(ln r / T_i) of Theorem 2 in every step; a
    number fixes the step size (Theorem 1 allows any eta in (0, 1]; the
    guarantee of Theorem 2 then no longer applies, the certificates still do).

    CERTIFIED mode draws only proven conclusions: separation gives L = alpha_i,
    f^t < alpha_i gives U = f^t; nothing is concluded from a stall or from T_i.
    Each alpha-FTP runs until one of those, or until the certificates close at
    a poll (every ``poll_every`` iterations), and the loop ends only when
    ub <= (1+eps) max(lb, L) or the budget is spent. Its step size is eta
    (default 1, the largest Theorem 1 allows). The search range (L, U) is then
    a certificate too and lower_bound reports max(lb, L).

    CORESET mode (points only; with radii it is CERTIFIED) adds core-set
    certificates: at the polls where the search's iteration count first
    reaches 256, 512, 1024, ..., ses_coreset_bounds runs from the current
    mean, its dual value joining the lower bounds and its ball the upper ones.
    """
    if mode in (MODE_CERTIFIED, MODE_CORESET):
        return _ses_solve_certified(V, gamma, eps, max_iters, max_steps, 1.0 if eta is None else float(eta),
                                    poll_every, coreset=mode == MODE_CORESET and gamma is None)
    V, gm = _prep(V, gamma)
    n = V.shape[0]
    D = ses_D(V, gm)
    rho = ses_width(D)
    r = ses_rank(n)
    L, U = D / 2.0, D
    lb, ub, center = 0.0, ses_objective(V, gm, V[0]), V[0].copy()
    total, steps = 0, []
    if D == 0.0:
        return {"radius": ub, "center": center, "lower_bound": ub, "upper_bound": ub,
                "iters": 0, "steps": steps, "L": 0.0, "U": 0.0}
    while U > (1.0 + eps) * L and ub > (1.0 + eps) * lb and total < max_iters and len(steps) < max_steps:
        alpha = L + (U - L) / 3.0
        eps_i = (U - L) / (3.0 * alpha)
        T = ses_T(D, n, eps_i, alpha)
        eta_i = theorem_eta(r, T) if eta is None else float(eta)
        res = ses_ftp(V, gm, alpha, eta_i, rho, min(T, max_iters - total), mode=mode,
                      delta=delta, patience=patience)
        total += res["iters"]
        if res["f_best"] < ub:
            ub, center = res["f_best"], res["c_best"]
        lb = max(lb, res["lb_best"])
        if res["outcome"] == OUT_SEPARATED:
            L = max(L, alpha)
        elif res["iters"] >= T or res["outcome"] in (OUT_STALLED, OUT_BELOW_ALPHA):
            U = min(U, (1.0 + eps_i) * alpha, ub)
        L = max(L, lb)
        steps.append({"alpha": alpha, "eps_i": eps_i, "T": T, "eta": eta_i,
                      "outcome": res["outcome"], "iters": res["iters"], "L": L, "U": U})
        if res["outcome"] not in (OUT_SEPARATED, OUT_STALLED, OUT_BELOW_ALPHA) and res["iters"] < T:
            break  # iteration budget exhausted inside the step
    return {"radius": ub, "center": center, "lower_bound": lb, "upper_bound": ub,
            "iters": total, "steps": steps, "L": L, "U": U}


def _ses_solve_certified(V, gamma, eps, max_iters, max_steps, eta, poll_every, coreset=False):
    V, gm = _prep(V, gamma)
    n = V.shape[0]
    D = ses_D(V, gm)
    rho = ses_width(D)
    L, U = D / 2.0, D
    lb, ub, center = 0.0, ses_objective(V, gm, V[0]), V[0].copy()
    total, steps = 0, []
    if D == 0.0:
        return {"radius": ub, "center": center, "lower_bound": ub, "upper_bound": ub,
                "iters": 0, "steps": steps, "L": 0.0, "U": 0.0}
    cs = {"next": CORESET_FIRST, "base": 0} if coreset else None
    while ub > (1.0 + eps) * max(lb, L) and total < max_iters and len(steps) < max_steps:
        alpha = L + (U - L) / 3.0
        cert = {"lb": max(lb, L), "ub": ub, "eps": eps, "poll_every": poll_every}
        if cs is not None:
            cs["base"] = total
            cert["coreset"] = cs
        res = ses_ftp(V, gm, alpha, eta, rho, max_iters - total, mode=MODE_CERTIFIED, cert=cert)
        total += res["iters"]
        eta_used = eta
        if res["outcome"] == OUT_STUCK:
            eta *= 0.5  # smaller steps resolve alpha closer to OPT
        if res["f_best"] < ub:
            ub, center = res["f_best"], res["c_best"]
        lb = max(lb, res["lb_best"])
        if res["outcome"] == OUT_SEPARATED:
            L = max(L, alpha)
        U = min(U, ub)
        L = max(L, lb)
        steps.append({"alpha": alpha, "eta": eta_used, "outcome": res["outcome"], "iters": res["iters"],
                      "L": L, "U": U})
        if res["outcome"] not in (OUT_SEPARATED, OUT_BELOW_ALPHA, OUT_CERTIFIED, OUT_STUCK):
            break  # iteration budget exhausted inside the step
    return {"radius": ub, "center": center, "lower_bound": max(lb, L), "upper_bound": ub,
            "iters": total, "steps": steps, "L": L, "U": U}


# ---------------------------------------------------------------------------
# Core-set certificates for SES (beyond the paper, on the dual pair of Sec. 4.1
# for points, gamma = 0): any weights mu on the simplex over a subset of the
# points give phi(mu) = sum_i mu_i |v_i|^2 - |sum_i mu_i v_i|^2 <= OPT^2 (weak
# duality of the minimum-enclosing-ball QP: a subset's weights are feasible
# for the whole problem), and every centre c gives the enclosing radius
# max_i |v_i - c| >= OPT. The subset is the K points farthest from a given
# centre (the current mean of the MWU), the weights are maximised by
# Frank-Wolfe steps with away steps on the subset, and the ball at their
# barycentre c_mu = sum_i mu_i v_i is evaluated on every point.
# ---------------------------------------------------------------------------
CORESET_K_SES = 512


def ses_coreset_pick(V, c, K):
    """Indices of the K points (all, if fewer) farthest from c, by descending
    distance (ties by index)."""
    d2 = ((V - c) ** 2).sum(axis=1)
    order = np.lexsort((np.arange(len(V)), -d2))
    return np.sort(order[:min(K, len(V))])


def meb_dual_fw(P, tol, max_iter=200_000):
    """Weights mu on the simplex over the rows of P maximising phi(mu) by
    Frank-Wolfe steps toward the farthest point and away steps from the
    nearest point of the support (exact line searches: phi is a concave
    quadratic along both), until the farthest point of P from c_mu lies
    within (1 + tol) sqrt(phi). Returns (mu, c_mu, sqrt(phi), the farthest
    distance)."""
    m = len(P)
    sq = (P * P).sum(axis=1)
    mu = np.zeros(m)
    c0 = P.mean(axis=0)
    j0 = int(np.argmax(((P - c0) ** 2).sum(axis=1)))
    mu[j0] = 1.0
    c = P[j0].copy()
    for _ in range(max_iter):
        dist2 = ((P - c) ** 2).sum(axis=1)
        phi = float(mu @ sq - c @ c)
        j = int(np.argmax(dist2))
        if dist2[j] <= (1.0 + tol) ** 2 * phi:
            break
        supp = np.nonzero(mu > 0.0)[0]
        a = int(supp[np.argmin(dist2[supp])])
        g_fw = dist2[j] - phi            # slope of phi toward e_j
        g_aw = phi - dist2[a]            # slope of phi away from e_a
        if g_fw >= g_aw or mu[a] >= 1.0:
            s = min(1.0, g_fw / (2.0 * dist2[j]))
            mu *= 1.0 - s
            mu[j] += s
            c = (1.0 - s) * c + s * P[j]
        else:
            smax = mu[a] / (1.0 - mu[a])
            s = min(smax, g_aw / (2.0 * dist2[a])) if dist2[a] > 0.0 else smax
            mu *= 1.0 + s
            mu[a] -= s
            if s >= smax:
                mu[a] = 0.0
            c = (1.0 + s) * c - s * P[a]
    phi = max(float(mu @ sq - c @ c), 0.0)
    far = math.sqrt(float(((P - c) ** 2).sum(axis=1).max()))
    return mu, c, math.sqrt(phi), far


def ses_coreset_bounds(V, c, K=CORESET_K_SES, tol=1e-4, rounds=1, eps=None):
    """Core-set bounds from centre c: (lb, ub, centre) with lb = sqrt(phi(mu))
    for the weights of meb_dual_fw on the K points farthest from c (a lower
    bound on OPT) and ub = max_i |v_i - c_mu| over every point, the radius of
    an actual enclosing ball at c_mu (an upper bound). With rounds > 1 the K
    points farthest from each new centre join the core set for up to that
    many rounds, until ub <= (1 + eps) lb; the best bounds are returned."""
    core = np.zeros(0, dtype=np.int64)
    lb, ub, best_c = 0.0, math.inf, np.asarray(c, dtype=np.float64).copy()
    for _ in range(rounds):
        core = np.union1d(core, ses_coreset_pick(V, c, K))
        _, cm, lb_r, _ = meb_dual_fw(V[core], tol)
        lb = max(lb, lb_r)
        ub_r = math.sqrt(float(((V - cm) ** 2).sum(axis=1).max()))
        if ub_r < ub:
            ub, best_c = ub_r, cm
        c = cm
        if eps is not None and ub <= (1.0 + eps) * lb:
            break
    return lb, ub, best_c
