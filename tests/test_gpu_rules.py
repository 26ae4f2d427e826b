"""The alpha-FTP's stopping rules on the device against the FP64 oracle.

Sec. 5 (practical rules): an alpha-FTP stops affirmatively once f^t beats
alpha (SES: the radius f^t < alpha; SVM: the margin f^t > alpha) and once
|f^t - f^{t-1}| / f^{t-1} < delta for `patience` consecutive iterations (the
ratio skipped while f^{t-1} = 0); Sec. 3 / Theorem 2 or 3: the ORACLE's
separation ends it with OPT > alpha (SES) or OPT < alpha (SVM). THEORY mode of
the search runs the T_i iterations of Theorems 2/3 per alpha-FTP.

Three kinds of check:
  * replayed trajectories: after every device step the oracle takes the same
    step from the device's own state (t and the FP64 mean read back), applies
    the rules to its own values, and the device's streak counter, stop flag
    and outcome must agree wherever the oracle's quantity is farther from its
    threshold than the FP32 error observed in that step (elsewhere the
    device's decision is adopted and counted; at most two per case);
  * independent trajectories: the device's stop iteration and outcome equal
    those of the oracle's own alpha-FTP in the same mode, on cases where every
    decision of the oracle is at least ten tolerances from its threshold
    (asserted on the oracle first);
  * the THEORY search of ses_solve / svm_solve against the oracle's THEORY
    search on tiny instances, with both searches' certificates bracketing the
    exact optimum.
"""

import math

import numpy as np
import pytest
import torch

from oracle import exact, ses as oses, svm as osvm
from paper_2405_09157_gb300 import _ffi, api, datagen

pytestmark = pytest.mark.gpu
RTOL = 1e-5
OUT = {oses.OUT_SEPARATED: _ffi.OUT_SEPARATED, oses.OUT_BELOW_ALPHA: _ffi.OUT_BEAT_ALPHA,
       oses.OUT_STALLED: _ffi.OUT_STALLED, osvm.OUT_ABOVE_ALPHA: _ffi.OUT_BEAT_ALPHA}

# The device state header (128 bytes), field for field.
HDR = np.dtype([("t", "<i8"), ("stopped", "<i4"), ("outcome", "<i4"), ("status", "<i4"), ("rules", "<i4"),
                ("streak", "<i4"), ("patience", "<i4"), ("delta", "<f8"), ("hint", "<f8"), ("move", "<f8"),
                ("f_prev", "<f8"), ("best_f", "<f8"), ("lb_best", "<f8"), ("ub_best", "<f8"), ("s1bar", "<f8"),
                ("s2bar", "<f8"), ("last_value", "<f8"), ("dual_A", "<f8"), ("dual_w", "<f8")])
assert HDR.itemsize == 128


def read_state(state, d):
    """(header, FP64 running mean) of a device state."""
    torch.cuda.synchronize()
    b = state.cpu().numpy().tobytes()
    return np.frombuffer(b[:128], dtype=HDR)[0], np.frombuffer(b[128:128 + 8 * d], dtype="<f8").copy()


class RuleReplay:
    """The Sec. 5 rules applied to the oracle's values, step by step. A
    decision counts as robust when the oracle's quantity is farther from its
    threshold than 1.5 times the FP32 error actually observed in that step
    (device value against oracle value); otherwise the device's decision is
    adopted and counted."""

    def __init__(self, alpha, delta, patience, beats):
        self.alpha, self.delta, self.patience, self.beats = alpha, delta, patience, beats
        self.f_prev, self.f_prev_dev, self.streak, self.adopted = None, None, 0, 0

    def step(self, t, o, r, dev_hdr):
        """Expected (stopped, outcome) after the step at t (o: oracle record,
        r: device record, dev_hdr: device state header after the step)."""
        f, fd = o["objective"], r["objective"]
        value = o["oracle_value"]
        if abs(value) <= 1.5 * abs(r["oracle_value"] - value):  # the sign is within rounding: follow the device
            self.adopted += 1
            failed = dev_hdr["outcome"] == _ffi.OUT_SEPARATED
        else:
            failed = o["failed"]
        if failed:
            return True, _ffi.OUT_SEPARATED
        if t == 0:
            return False, _ffi.OUT_RUNNING
        beat = self.beats(f)
        if abs(f - self.alpha) <= 1.5 * abs(fd - f):
            self.adopted += 1
            beat = dev_hdr["outcome"] == _ffi.OUT_BEAT_ALPHA
        if beat:
            return True, _ffi.OUT_BEAT_ALPHA
        if self.f_prev is not None and self.f_prev > 0.0:
            ratio = abs(f - self.f_prev) / self.f_prev
            err = (abs(fd - f) + abs(self.f_prev_dev - self.f_prev)) / self.f_prev
            if abs(ratio - self.delta) <= 1.5 * err:
                self.adopted += 1
                self.streak = int(dev_hdr["streak"]) if not dev_hdr["stopped"] else self.patience
            else:
                self.streak = self.streak + 1 if ratio < self.delta else 0
            if self.streak >= self.patience:
                return True, _ffi.OUT_STALLED
        self.f_prev, self.f_prev_dev = f, fd
        return False, _ffi.OUT_RUNNING


def _ses_setup(n, d, seed, rel_alpha):
    V32 = datagen.ses_gaussian(n, d, seed)
    V = V32.astype(np.float64)
    D = oses.ses_D(V)
    return V32, V, D, oses.ses_width(D), rel_alpha * D


@pytest.mark.parametrize("n,d,seed,rel_alpha,eta,delta,outcome", [
    (800, 3, 7, 0.80, 0.5, 5e-3, _ffi.OUT_STALLED),      # the streak fires at t = 43
    (800, 3, 4, 0.85, 0.5, 1e-4, _ffi.OUT_BEAT_ALPHA),   # the paper's delta; f beats alpha at t = 79
    (800, 3, 9, 0.80, 0.5, 1e-4, _ffi.OUT_BEAT_ALPHA),   # at t = 2
    (800, 3, 7, 0.80, 0.5, 1e-4, _ffi.OUT_SEPARATED),    # separation at t = 83 under the practical rules
    (3000, 16, 11, 0.62, 0.5, 2e-3, None),               # whatever ends it first
])
def test_ses_practical_rules_replayed(n, d, seed, rel_alpha, eta, delta, outcome):
    V32, V, D, rho, alpha = _ses_setup(n, d, seed, rel_alpha)
    tol = RTOL * D
    patience = 10
    m = api.MWU(_ffi.SES, torch.from_numpy(V32).cuda(), rules=_ffi.RULES_PRACTICAL, delta=delta, patience=patience)
    rules = RuleReplay(alpha, delta, patience, lambda f: f < alpha)
    out = api.new_steps(1)
    end = None
    for _ in range(400):
        h0, ubar = read_state(m.state, d)
        t = int(h0["t"])
        m.step(alpha, eta / rho, out=out)
        h1, _ = read_state(m.state, d)
        r = api.decode_steps(out)[0]
        o = oses.ses_step(V, None, ubar, t, alpha, eta, rho)
        assert r["status"] == 0
        for key in ("objective", "oracle_value", "lower_bound"):
            assert abs(r[key] - o[key]) <= tol, (t, key, r[key], o[key])
        stopped, oc = rules.step(t, o, r, h1)
        assert bool(h1["stopped"]) == stopped and h1["outcome"] == oc, (t, dict(zip(HDR.names, h1)), stopped, oc)
        assert r["stopped"] == int(stopped) and r["outcome"] == oc
        if not stopped and t > 0 and rules.f_prev is not None:
            assert h1["streak"] == rules.streak, (t, h1["streak"], rules.streak)
        assert h1["t"] == (t if stopped else t + 1)
        if stopped:
            end = (t, oc)
            break
    assert end is not None, "the alpha-FTP did not stop"
    if outcome is not None:
        assert end[1] == outcome, end
    assert rules.adopted <= 2, rules.adopted
    # a stopped alpha-FTP is left alone by further steps
    m.step(alpha, eta / rho, out=out)
    h2, _ = read_state(m.state, d)
    assert h2["t"] == h1["t"] and h2["stopped"] == 1 and h2["outcome"] == end[1]


@pytest.mark.parametrize("n,d,seed,rel_alpha,eta,delta", [
    (800, 3, 7, 0.80, 0.5, 5e-3),   # stalled at t = 43
    (800, 3, 4, 0.78, 0.5, 5e-3),   # stalled at t = 18
    (800, 3, 9, 0.80, 0.5, 1e-4),   # f beats alpha at t = 2
])
def test_ses_practical_stop_matches_oracle_ftp(n, d, seed, rel_alpha, eta, delta):
    V32, V, D, rho, alpha = _ses_setup(n, d, seed, rel_alpha)
    tol = RTOL * D
    res = oses.ses_ftp(V, None, alpha, eta, rho, 5000, mode=oses.MODE_PRACTICAL, delta=delta, patience=10,
                       keep_trace=True)
    tr = res["trace"]
    f = np.array([x["objective"] for x in tr])
    # every decision of the oracle is at least ten tolerances from its threshold
    assert min(abs(x["oracle_value"]) for x in tr) > 10 * tol
    assert np.min(np.abs(f[1:] - alpha)) > 10 * tol
    if len(f) > 2:
        ratio = np.abs(np.diff(f[1:])) / f[1:-1]
        assert np.min(np.abs(ratio - delta) / (3 * tol / f[1:-1])) > 10
    m = api.MWU(_ffi.SES, torch.from_numpy(V32).cuda(), rules=_ffi.RULES_PRACTICAL, delta=delta, patience=10)
    T = res["iters"] + 5
    out = api.new_steps(T)
    for t in range(T):
        m.step(alpha, eta / rho, out=out[t])
    recs = api.decode_steps(out)
    stop = int(np.argmax(recs["stopped"] == 1))
    assert recs["stopped"][stop] == 1
    assert stop == res["iters"], (stop, res["iters"], res["outcome"])
    assert recs["outcome"][stop] == OUT[res["outcome"]]
    assert np.all(recs["t"][stop + 1:] == 0)  # no record after the stop
    h, mean = read_state(m.state, d)
    assert h["t"] == res["iters"] and h["outcome"] == OUT[res["outcome"]]
    assert np.linalg.norm(mean - res["ubar"]) <= tol


def _svm_setup(n1, n2, d, seed):
    X32, y = datagen.svm_clusters(n1, n2, d, seed=seed)
    X = X32.astype(np.float64)
    D = osvm.svm_D(X)
    return X32, y, X, y.astype(np.float64), D, osvm.svm_width(D)


@pytest.mark.parametrize("n1,n2,d,seed,alpha,eta,delta,outcome", [
    (400, 300, 8, 5, 1.0, 0.5, 5e-3, _ffi.OUT_STALLED),      # the streak fires at t = 12
    (400, 300, 8, 5, 1.0, 0.5, 1e-4, _ffi.OUT_BEAT_ALPHA),   # the margin beats alpha at t = 135
    (400, 300, 8, 5, 0.5, 0.5, 5e-3, _ffi.OUT_BEAT_ALPHA),   # at t = 1
    (1000, 1000, 16, 7, 1.5, 0.5, 1e-4, _ffi.OUT_SEPARATED),  # OPT < alpha: separation at t = 152
])
def test_svm_practical_rules_replayed(n1, n2, d, seed, alpha, eta, delta, outcome):
    X32, y8, X, y, D, rho = _svm_setup(n1, n2, d, seed)
    tol = RTOL * D
    patience = 10
    m = api.MWU(_ffi.SVM, torch.from_numpy(X32).cuda(), labels=torch.from_numpy(y8).cuda(),
                rules=_ffi.RULES_PRACTICAL, delta=delta, patience=patience)
    rules = RuleReplay(alpha, delta, patience, lambda f: f > alpha)
    out = api.new_steps(1)
    end = None
    for _ in range(400):
        h0, wbar = read_state(m.state, d)
        t = int(h0["t"])
        m.step(alpha, eta / rho, out=out, D=D)
        h1, _ = read_state(m.state, d)
        r = api.decode_steps(out)[0]
        o = osvm.svm_step(X, y, wbar, float(h0["s1bar"]), float(h0["s2bar"]), t, alpha, eta, rho, D)
        assert r["status"] == 0
        for key in ("objective", "oracle_value", "upper_bound"):
            assert abs(r[key] - o[key]) <= tol, (t, key, r[key], o[key])
        stopped, oc = rules.step(t, o, r, h1)
        assert bool(h1["stopped"]) == stopped and h1["outcome"] == oc, (t, dict(zip(HDR.names, h1)), stopped, oc)
        if not stopped and t > 0 and rules.f_prev is not None:
            assert h1["streak"] == rules.streak, (t, h1["streak"], rules.streak)
        if stopped:
            end = (t, oc)
            break
    assert end is not None and end[1] == outcome, end
    assert rules.adopted <= 2, rules.adopted


def test_ses_theory_search_matches_oracle():
    """THEORY mode (T_i of Theorem 2 per alpha-FTP, Sec. 4.1 constants): the
    first FTP runs its T_1 iterations (alpha_1 = 2D/3 > OPT: no separation),
    then the range closes; the device reports the same iteration count and
    search steps, and both searches' certificates bracket Welzl's radius."""
    V32 = datagen.ses_gaussian(20, 2, 1)
    V = V32.astype(np.float64)
    eps = 0.1
    o = oses.ses_solve(V, None, eps=eps, mode=oses.MODE_THEORY)
    center, rep = api.ses_solve(torch.from_numpy(V32).cuda(), eps=eps, mode="theory")
    D = oses.ses_D(V)
    opt = exact.mec_2d(V)[1]
    assert rep["status"] == 0
    assert rep["search_steps"] == len(o["steps"]) and rep["iters"] == o["iters"], (rep, o["iters"], o["steps"])
    # the bounds are the best of 4715 iterations, over which the trajectories
    # drift apart by more than one step's rounding (see test_gpu_parity.py);
    # they are compared at ten times the single-step tolerance
    assert abs(rep["upper_bound"] - o["radius"]) <= 10 * RTOL * D
    assert abs(rep["lower_bound"] - o["lower_bound"]) <= 10 * RTOL * D
    for lb, ub in ((rep["lower_bound"], rep["upper_bound"]), (o["lower_bound"], o["radius"])):
        assert lb <= opt * (1 + 1e-9) and ub >= opt * (1 - 1e-9)
    c = center.cpu().numpy().astype(np.float64)
    assert abs(np.max(np.linalg.norm(V - c, axis=1)) - rep["upper_bound"]) <= RTOL * D


def test_svm_theory_search_matches_oracle():
    """THEORY mode for SVM (Theorem 3): every FTP of this instance ends by
    separation, several after thousands of iterations where the ORACLE value
    approaches 0 slowly, so the separating iteration can move by a few steps
    between FP32 and FP64; the search steps, the range and the certificates
    are compared, and both searches bracket the exact polytope distance."""
    X32, y8, X, y, D, rho = _svm_setup(15, 15, 3, 2)
    eps = 0.2
    o = osvm.svm_solve(X, y, eps=eps, mode=osvm.MODE_THEORY)
    w, rep = api.svm_solve(torch.from_numpy(X32).cuda(), torch.from_numpy(y8).cuda(), eps=eps, mode="theory")
    opt = exact.pd_bruteforce(X[y > 0], X[y < 0])[0]
    assert rep["status"] == 0
    assert rep["search_steps"] == len(o["steps"]), (rep, o["steps"])
    assert abs(rep["iters"] - o["iters"]) <= 0.02 * o["iters"], (rep["iters"], o["iters"])
    assert abs(rep["search_U"] - o["U"]) <= 1e-3 * D and abs(rep["search_L"] - o["L"]) <= 1e-3 * D
    for lb, ub in ((rep["lower_bound"], rep["upper_bound"]), (o["lower_bound"], o["upper_bound"])):
        assert lb <= opt * (1 + 1e-6) and ub >= opt * (1 - 1e-6)
    assert rep["lower_bound"] >= (1 - 2 * eps) * opt
