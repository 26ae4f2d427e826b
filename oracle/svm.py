"""Hard-margin SVM / polytope distance through the minimisation variant, FP64.

Follows Sec. 4.2: problem (SVM) and its dual (PD); Lemma 6 (s_1, s_2 <= D
with D the largest point norm); the split into C = {||w|| <= 1, s_1, s_2 <= D}
and F = {P^T w >= s_1 1, -Q^T w >= s_2 1}; the min-form SCP (svm_dual_scp)
with K = R^n_+ (r = n) and R = 2; the closed-form ORACLE of Eq. (svm_oracle)
and its solution; Claim 8 (the normalised weights are PD-feasible); the
width rho <= 2D and T = ceil(64 D^2 ln n / (eps^2 alpha^2)). Sec. 3 supplies
the minimisation variant (Eq. min_implement, Theorem 3). Sec. 5 supplies the
margin f^t and the early rules.

Inputs: X is the (n, d) array of points, y the (n,) labels in {+1, -1}.
P = rows with y = +1, Q = rows with y = -1 (Sec. 4.2). Component i of
K = R^n_+ belongs to row i; the order of components in a product cone does
not matter (Sec. 2.1).

Readings of the paper taken here (the GPU path takes the same ones):
  * f^t (Sec. 5) prints the letters of the two sets swapped; it is read as
    (min over P of x^T wbar - max over Q of x^T wbar)/||wbar||, clipped at 0,
    which is the margin of the hyperplane with normal wbar (Eq. SVM).
  * f^0, and f whenever wbar = 0, is 0.
  * z = P mu - Q gamma = 0 gives w = 0 (the ORACLE's maximiser is then any
    unit vector; its value does not depend on it).
  * The search for the minimisation variant mirrors Sec. 3: alpha_i =
    U - (U-L)/3, eps_i = (U-L)/(3 alpha_i); separation (value < 0, so
    OPT < alpha_i) gives U = alpha_i, the Theorem 3 conclusion gives
    L = (1 - eps_i) alpha_i.
"""

import math

import numpy as np

from .eja import scmwu_orthant

OUT_SEPARATED = "separated"      # ORACLE value < 0: OPT < alpha (Theorem 3)
OUT_FEASIBLE = "feasible"        # T iterations without separation
OUT_ABOVE_ALPHA = "above_alpha"  # margin f^t > alpha: affirmative early exit (Sec. 5)
OUT_STALLED = "stalled"
OUT_FIXED = "fixed"
OUT_CERTIFIED = "certified"      # CERTIFIED mode: the certificates closed at a poll

MODE_PRACTICAL = "practical"
MODE_THEORY = "theory"
MODE_FIXED = "fixed"
MODE_CERTIFIED = "certified"
MODE_CORESET = "coreset"         # CERTIFIED with core-set certificates (beyond the paper)
OUT_STUCK = "stuck"              # CERTIFIED mode: the certificate gap stopped shrinking (eta is halved)
CERT_FIRST_CHECK = 1024          # CERTIFIED: first progress check of an alpha-FTP at eta = 1 (then 2x, 4x, ...)
CERT_SHRINK = 0.8                # CERTIFIED: the FTP's own gap must shrink by this factor while t doubles
CERT_MIN_ETA = 1.0 / 64.0        # CERTIFIED: eta is not halved below this (no progress test there)

SVM_R = 2.0  # Sec. 4.2
CORESET_K = 512        # points per class in a core set
CORESET_FIRST = 256    # first core-set check after this many iterations of the search, then every doubling
CORESET_ROUNDS = 4     # active-set rounds of one check


def _prep(X, y):
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y).astype(np.float64)
    if X.ndim != 2 or y.shape != (X.shape[0],):
        raise ValueError("SVM needs an (n, d) array and (n,) labels")
    if not np.all((y == 1.0) | (y == -1.0)):
        raise ValueError("labels must be +1 or -1")
    if not (np.any(y > 0) and np.any(y < 0)):
        raise ValueError("both classes must be non-empty")
    return X, y


def svm_D(X):
    """D = max point norm over P and Q (Lemma 6)."""
    X = np.asarray(X, dtype=np.float64)
    return float(np.max(np.sqrt(np.sum(X * X, axis=1))))


def svm_width(D):
    """Width of the SVM ORACLE, rho <= 2D (Sec. 4.2)."""
    return 2.0 * D


def svm_T(D, n, eps, alpha):
    """T = ceil(64 D^2 ln n / (eps^2 alpha^2)) (Sec. 4.2, from Theorem 3)."""
    return int(math.ceil(64.0 * D * D * math.log(n) / (eps * eps * alpha * alpha)))


def svm_exponent(X, y, wbar, s1bar, s2bar, k):
    """Exponent of Eq. (min_implement) for the SVM data of Eq. (svm_dual_scp).

    c - sum_j a_j ybar_j = (P^T wbar - s1bar 1; -Q^T wbar - s2bar 1), i.e.
    y_i x_i^T wbar - sbar_{class(i)} for component i, scaled by -k with
    k = eta t / rho. Returns the (n,) array.
    """
    X, y = _prep(X, y)
    sbar = np.where(y > 0, s1bar, s2bar)
    return -k * (y * (X @ np.asarray(wbar, dtype=np.float64)) - sbar)


def svm_weights(X, y, wbar, s1bar, s2bar, k):
    """p^{t+1} = exp(x)/Tr(exp(x)) over R^n_+ (Eq. min_implement). Returns (n,)."""
    p, _, _ = scmwu_orthant(svm_exponent(X, y, wbar, s1bar, s2bar, k))
    return p


def svm_oracle(X, y, p, alpha, D):
    """Closed-form ORACLE of Eq. (svm_oracle) and its analytical solution.

    mu = p on P, gamma = p on Q. z = P mu - Q gamma, w = z/||z||,
    s_1 = D if Tr(mu) <= Tr(gamma) else alpha - D, s_2 = alpha - s_1;
    value = z^T w - Tr(mu) s_1 - Tr(gamma) s_2.
    Returns (w, s1, s2, value, z, tr_mu, tr_gamma).
    """
    X, y = _prep(X, y)
    mu = np.where(y > 0, p, 0.0)
    ga = np.where(y < 0, p, 0.0)
    z = X.T @ mu - X.T @ ga
    nz = math.sqrt(float(z @ z))
    w = z / nz if nz > 0.0 else np.zeros_like(z)
    # correctly rounded traces: two classes carrying equal weight (n1 = n2 at
    # t = 0) tie exactly and take s_1 = D, not a choice left to rounding
    tr_mu, tr_ga = math.fsum(mu), math.fsum(ga)
    s1 = D if tr_mu <= tr_ga else alpha - D
    s2 = alpha - s1
    value = float(z @ w) - tr_mu * s1 - tr_ga * s2
    return w, s1, s2, value, z, tr_mu, tr_ga


def svm_program_value(X, y, p, w, s1, s2):
    """Objective of Eq. (min_oracle) for y = (w; s1; s2), unsimplified:
    (c - sum_j a_j y_j) . p = sum_{i in P} (u_i^T w - s1) mu_i + sum_{i in Q} (-v_i^T w - s2) gamma_i."""
    X, y = _prep(X, y)
    slack = np.where(y > 0, X @ w - s1, -(X @ w) - s2)
    return float(slack @ p)


def svm_pd_vector(X, y, p):
    """P mu/Tr mu - Q gamma/Tr gamma for the weights p (Claim 8)."""
    X, y = _prep(X, y)
    mu = np.where(y > 0, p, 0.0)
    ga = np.where(y < 0, p, 0.0)
    return X.T @ mu / np.sum(mu) - X.T @ ga / np.sum(ga)


def svm_pd_value(X, y, p):
    """Claim 8: (mu/Tr mu; gamma/Tr gamma) is PD-feasible; returns its PD objective
    ||P mu/Tr mu - Q gamma/Tr gamma||, an upper bound on OPT (Eq. PD)."""
    diff = svm_pd_vector(X, y, p)
    return math.sqrt(float(diff @ diff))


def svm_dual_state(d):
    return {"z": np.zeros(d), "wsum": 0.0}


def svm_dual_update(avg, t, z):
    """Running average of the Claim 8 vectors over an alpha-FTP, iterate t
    weighted by t^2 (as the SES bound): zbar is P mubar - Q gammabar for the
    averaged class-normalised weights (each a point of its simplex), so |zbar|
    is again a PD-feasible value, an upper bound on OPT. Returns |zbar| (inf
    before any update)."""
    if t >= 1 and np.all(np.isfinite(z)):
        w = float(t) * float(t)
        avg["wsum"] += w
        avg["z"] = avg["z"] + (w / avg["wsum"]) * (z - avg["z"])
    if avg["wsum"] == 0.0:
        return math.inf
    return math.sqrt(float(avg["z"] @ avg["z"]))


def svm_margin(X, y, wbar):
    """f = max{(min_P x^T wbar - max_Q x^T wbar)/||wbar||, 0} (Sec. 5); 0 if wbar = 0."""
    X, y = _prep(X, y)
    wbar = np.asarray(wbar, dtype=np.float64)
    nw = math.sqrt(float(wbar @ wbar))
    if nw == 0.0:
        return 0.0
    s = X @ wbar
    return max((float(np.min(s[y > 0])) - float(np.max(s[y < 0]))) / nw, 0.0)


def svm_coreset_pick(X, y, w, K):
    """The core set picked by a direction w (core-set certificates, a reading
    beyond the paper built on Eq. (PD) and Sec. 4.2): in each class the K
    points (all, if fewer) with the smallest y_i x_i^T w, the points nearest
    the hyperplane with normal w, which are also the points the MWU weighs
    most in that class (the class-normalised weights fall with y_i x_i^T w).
    Returns a boolean mask over the rows."""
    X, y = _prep(X, y)
    s = y * (X @ np.asarray(w, dtype=np.float64))
    pick = np.zeros(X.shape[0], dtype=bool)
    for cls in (y > 0, y < 0):
        idx = np.nonzero(cls)[0]
        pick[idx[np.argsort(s[idx], kind="stable")[:K]]] = True
    return pick


def svm_coreset_bounds(X, y, w, eps, K=CORESET_K, rounds=CORESET_ROUNDS):
    """Certificates from core sets (beyond the paper): restricting Eq. (PD) to a
    subset of each class can only raise its minimum, so the exact polytope
    distance of a core set C (the points svm_coreset_pick takes from w) is an
    upper bound on OPT; the direction z_C of that solution is a separating
    direction of all the points only if no point outside C lies closer, and
    its margin over all the points (Sec. 5's f) is a lower bound on OPT. Each
    round adds the core set picked by z_C to C (an active set) until the
    bounds are within 1 + eps or `rounds` rounds have run. The core-set
    problem is solved by exact.pd_mdm to a gap of eps/10 of its value.
    Returns (lb, ub, w_lb): the margin of the best direction found, the
    smallest core-set distance, that direction."""
    from .exact import pd_mdm
    X, y = _prep(X, y)
    C = np.zeros(X.shape[0], dtype=bool)
    lb, ub, w_lb = 0.0, math.inf, None
    w = np.asarray(w, dtype=np.float64)
    for _ in range(rounds):
        C |= svm_coreset_pick(X, y, w, K)
        P, Q = X[C & (y > 0)], X[C & (y < 0)]
        dist, mu, ga, _, _ = pd_mdm(P, Q, tol=eps / 10.0)
        z = P.T @ mu - Q.T @ ga
        ub = min(ub, dist)
        m = svm_margin(X, y, z)
        if m > lb:
            lb, w_lb = m, z / math.sqrt(float(z @ z))
        if ub <= (1.0 + eps) * lb:
            break
        w = z
    return lb, ub, w_lb


def svm_step(X, y, wbar, s1bar, s2bar, t, alpha, eta, rho, D, avg=None):
    """One iteration of the minimisation alpha-FTP (Sec. 3, Theorem 3) for SVM.

    Computes p^{t+1} (k = eta t/rho), the ORACLE answer, the Claim 8 upper
    bound and the margin f at wbar; advances the means when the ORACLE succeeds.
    ``avg`` (from :func:`svm_dual_state`) is advanced by this iteration's Claim 8
    vector and rec["dual_bound"] is the averaged upper bound (inf without it).
    """
    X, y = _prep(X, y)
    k = eta * t / rho
    p = svm_weights(X, y, wbar, s1bar, s2bar, k)
    w, s1, s2, value, z, tr_mu, tr_ga = svm_oracle(X, y, p, alpha, D)
    pd = svm_pd_vector(X, y, p)
    rec = {
        "t": t, "k": k,
        "objective": svm_margin(X, y, wbar),
        "oracle_value": value,
        "upper_bound": math.sqrt(float(pd @ pd)),
        "w": w, "s1": s1, "s2": s2, "z": z, "tr_mu": tr_mu, "tr_gamma": tr_ga,
        "failed": value < 0.0,
        "dual_bound": math.inf,
    }
    if avg is not None:
        rec["dual_bound"] = svm_dual_update(avg, t, pd)
    wbar = np.asarray(wbar, dtype=np.float64)
    if value >= 0.0:
        rec["wbar_next"] = wbar + (w - wbar) / (t + 1)
        rec["s1bar_next"] = s1bar + (s1 - s1bar) / (t + 1)
        rec["s2bar_next"] = s2bar + (s2 - s2bar) / (t + 1)
    else:
        rec["wbar_next"], rec["s1bar_next"], rec["s2bar_next"] = wbar.copy(), s1bar, s2bar
    return rec


def svm_ftp(X, y, alpha, eta, rho, T, D, mode=MODE_FIXED, delta=1e-4, patience=10,
            keep_trace=False, cert=None):
    """Minimisation alpha-FTP of Theorem 3 for SVM, at most T iterations.

    Same modes as the SES test. PRACTICAL stops affirmatively once the margin
    f^t exceeds alpha and on the delta/patience rule of Sec. 5. CERTIFIED keeps
    the first rule only (f^t > alpha proves OPT > alpha) and, every
    cert["poll_every"] completed iterations, stops once
    min(cert["ub"], ub_best) <= (1 + cert["eps"]) max(cert["lb"], f_best),
    or as STUCK when, at the first poll with t >= c, 2c, 4c, ... (c = 1024/eta),
    the FTP's own gap ub_best / f_best - 1 has not shrunk by the factor 0.8
    since the previous such poll (no check once eta <= 1/64). ub_best is the
    best of the per-iteration and the averaged Claim 8 values.

    With cert["coreset"] (mode "coreset" of the search), a poll at
    which the search's iteration count cert["coreset"]["base"] + t has reached
    cert["coreset"]["next"] also runs svm_coreset_bounds from the FTP's best
    direction (wbar when no direction separates yet), folds its bounds into
    f_best / w_best and ub_best, and doubles "next", before the test above.
    """
    X, y = _prep(X, y)
    d = X.shape[1]
    wbar, s1bar, s2bar = np.zeros(d), 0.0, 0.0
    f_best, w_best = 0.0, np.zeros(d)
    ub_best = math.inf
    avg = svm_dual_state(d)
    trace = []
    f_prev, streak = None, 0
    outcome = OUT_FIXED if mode == MODE_FIXED else OUT_FEASIBLE
    last_gap = math.inf
    next_check = math.ceil(CERT_FIRST_CHECK / eta) if mode == MODE_CERTIFIED and eta > CERT_MIN_ETA else math.inf
    t = 0
    while t < T:
        rec = svm_step(X, y, wbar, s1bar, s2bar, t, alpha, eta, rho, D, avg=avg)
        if keep_trace:
            trace.append(rec)
        if rec["objective"] > f_best:
            f_best, w_best = rec["objective"], wbar.copy()
        ub_best = min(ub_best, rec["upper_bound"], rec["dual_bound"])
        if rec["failed"]:
            outcome = OUT_SEPARATED
            break
        if mode in (MODE_PRACTICAL, MODE_CERTIFIED) and t > 0:
            f = rec["objective"]
            if f > alpha:
                outcome = OUT_ABOVE_ALPHA
                break
            if mode == MODE_PRACTICAL and f_prev is not None and f_prev > 0.0:
                streak = streak + 1 if abs(f - f_prev) / f_prev < delta else 0
                if streak >= patience:
                    outcome = OUT_STALLED
                    break
            f_prev = f
        wbar, s1bar, s2bar = rec["wbar_next"], rec["s1bar_next"], rec["s2bar_next"]
        t += 1
        if mode == MODE_CERTIFIED and t % cert["poll_every"] == 0:
            cs = cert.get("coreset")
            if cs is not None and cs["base"] + t >= cs["next"]:
                lb_c, ub_c, w_c = svm_coreset_bounds(X, y, w_best if f_best > 0.0 else wbar, cert["eps"])
                if lb_c > f_best:
                    f_best, w_best = lb_c, w_c
                ub_best = min(ub_best, ub_c)
                cs["next"] *= 2
            if min(cert["ub"], ub_best) <= (1.0 + cert["eps"]) * max(cert["lb"], f_best):
                outcome = OUT_CERTIFIED
                break
            if t >= next_check:  # progress test: this FTP's own gap must halve while t doubles
                gap = ub_best / f_best - 1.0 if f_best > 0.0 else math.inf
                if gap > CERT_SHRINK * last_gap:
                    outcome = OUT_STUCK
                    break
                last_gap, next_check = gap, 2 * next_check
    f_end = svm_margin(X, y, wbar)
    if f_end > f_best:
        f_best, w_best = f_end, wbar.copy()
    return {"outcome": outcome, "iters": t, "wbar": wbar, "s1bar": s1bar, "s2bar": s2bar,
            "f_best": f_best, "w_best": w_best, "ub_best": ub_best, "trace": trace}


def svm_solve(X, y, eps=1e-2, mode=MODE_PRACTICAL, max_iters=10**7, delta=1e-4,
              patience=10, max_steps=200, eta=None, poll_every=256):
    """(1-eps)-approximate max margin by the search over alpha in (0, 2D] (Sec. 4.2).

    Certificates: lb = best margin f of an actual separating direction, ub =
    best Claim 8 PD value; the loop ends when U <= (1+eps) L, when
    ub <= (1+eps) lb, or when ``max_iters`` iterations have run. ``eta`` as in
    the SES search: None for Theorem 3's eta_i, a number to fix it.

    CERTIFIED mode (as for SES): separation gives U = alpha_i, f^t > alpha_i
    gives L = f^t, nothing else is concluded; each alpha-FTP runs until one of
    those or until the certificates close at a poll, and the loop ends when
    min(ub, U) <= (1+eps) lb or the budget is spent; eta defaults to 1 and
    upper_bound reports min(ub, U).

    CORESET mode is CERTIFIED with core-set certificates (beyond the paper):
    at the polls where the search's iteration count first reaches 256, 512,
    1024, ..., svm_coreset_bounds runs from the running FTP's best direction.
    """
    if mode in (MODE_CERTIFIED, MODE_CORESET):
        return _svm_solve_certified(X, y, eps, max_iters, max_steps, 1.0 if eta is None else float(eta),
                                    poll_every, coreset=mode == MODE_CORESET)
    X, y = _prep(X, y)
    n = X.shape[0]
    D = svm_D(X)
    rho = svm_width(D)
    L, U = 0.0, 2.0 * D
    lb, ub, w_best = 0.0, math.inf, np.zeros(X.shape[1])
    total, steps = 0, []
    while U > (1.0 + eps) * L and ub > (1.0 + eps) * lb and total < max_iters and len(steps) < max_steps:
        alpha = U - (U - L) / 3.0
        eps_i = (U - L) / (3.0 * alpha)
        T = svm_T(D, n, eps_i, alpha)
        eta_i = math.sqrt(math.log(n) / T) if eta is None else float(eta)
        res = svm_ftp(X, y, alpha, eta_i, rho, min(T, max_iters - total), D, mode=mode,
                      delta=delta, patience=patience)
        total += res["iters"]
        if res["f_best"] > lb:
            lb, w_best = res["f_best"], res["w_best"]
        ub = min(ub, res["ub_best"])
        if res["outcome"] == OUT_SEPARATED:
            U = min(U, alpha)
        elif res["iters"] >= T or res["outcome"] in (OUT_STALLED, OUT_ABOVE_ALPHA):
            L = max(L, (1.0 - eps_i) * alpha, lb)
        U = min(U, ub)
        L = max(L, lb)
        steps.append({"alpha": alpha, "eps_i": eps_i, "T": T, "eta": eta_i,
                      "outcome": res["outcome"], "iters": res["iters"], "L": L, "U": U})
        if res["outcome"] not in (OUT_SEPARATED, OUT_STALLED, OUT_ABOVE_ALPHA) and res["iters"] < T:
            break
    return {"margin": lb, "w": w_best, "lower_bound": lb, "upper_bound": ub,
            "iters": total, "steps": steps, "L": L, "U": U}


def _svm_solve_certified(X, y, eps, max_iters, max_steps, eta, poll_every, coreset=False):
    X, y = _prep(X, y)
    D = svm_D(X)
    rho = svm_width(D)
    L, U = 0.0, 2.0 * D
    lb, ub, w_best = 0.0, math.inf, np.zeros(X.shape[1])
    total, steps = 0, []
    cs = {"next": CORESET_FIRST, "base": 0} if coreset else None
    while min(ub, U) > (1.0 + eps) * lb and total < max_iters and len(steps) < max_steps:
        alpha = U - (U - L) / 3.0
        cert = {"lb": lb, "ub": min(ub, U), "eps": eps, "poll_every": poll_every}
        if cs is not None:
            cs["base"] = total
            cert["coreset"] = cs
        res = svm_ftp(X, y, alpha, eta, rho, max_iters - total, D, mode=MODE_CERTIFIED, cert=cert)
        total += res["iters"]
        eta_used = eta
        if res["outcome"] == OUT_STUCK:
            eta *= 0.5
        if res["f_best"] > lb:
            lb, w_best = res["f_best"], res["w_best"]
        ub = min(ub, res["ub_best"])
        if res["outcome"] == OUT_SEPARATED:
            U = min(U, alpha)
        U = min(U, ub)
        L = max(L, lb)
        steps.append({"alpha": alpha, "eta": eta_used, "outcome": res["outcome"], "iters": res["iters"],
                      "L": L, "U": U})
        if res["outcome"] not in (OUT_SEPARATED, OUT_ABOVE_ALPHA, OUT_CERTIFIED, OUT_STUCK):
            break
    return {"margin": lb, "w": w_best, "lower_bound": lb, "upper_bound": min(ub, U),
            "iters": total, "steps": steps, "L": L, "U": U}
