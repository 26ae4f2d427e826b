"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerance. The kernels compute per point in FP32, reduce the per-CTA
partial sums in compensated FP32 (FP64-grade totals), run the O(d) finish of
each iteration in FP32 from those totals and keep the running mean in FP64.
A per-point weight e^{x} carries a relative error of about
k D 2^-24 from its FP32 argument (k = eta t / rho, D the problem scale);
with k D <= 64 (every case below) that is <= 4e-6, and the ORACLE value, f,
the bounds and the next running mean, being weighted averages, inherit it.
The tests require agreement to RTOL = 1e-5 relative to D.

Two kinds of check:
  * single steps from a checkpoint (t, mean) set on both sides (mwu_state_set),
    at k D in {1, 10, 40, 64}: the kernel's arithmetic against the oracle's;
  * trajectories of 25 iterations from t = 0: the state bookkeeping (t,
    means, shift bound). Longer trajectories are not compared: the alpha-FTP
    dynamics amplify any rounding difference (an FP64 re-implementation of
    the kernel's formulas drifts from the FP64 oracle from 1e-16 at t = 50 to
    5e-10 at t = 200), so they would measure that amplification, not the
    kernel.
ORACLE decisions are compared only where the oracle's value is farther than
the tolerance from 0.
"""

import math

import numpy as np
import pytest
import torch

from oracle import exact, ses as oses, svm as osvm
from paper_2405_09157_gb300 import _ffi, api, datagen

pytestmark = pytest.mark.gpu
RTOL = 1e-5


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_ses_traj(V32, g32, alpha, eta_over_rho, T, dtype=torch.float32, rules=_ffi.RULES_NONE, pts=None):
    pts = _cuda(V32).to(dtype) if pts is None else pts
    radii = None if g32 is None else _cuda(g32)
    m = api.MWU(_ffi.SES, pts, radii=radii, rules=rules)
    out = api.new_steps(T)
    for t in range(T):
        m.step(alpha, eta_over_rho, out=out[t])
    torch.cuda.synchronize()
    mean, best = m.read()
    return api.decode_steps(out), mean.cpu().numpy().astype(np.float64)


def oracle_ses_traj(V, g, alpha, eta, rho, T):
    ubar = V[0].copy()
    recs = []
    avg = oses.ses_dual_state(V.shape[1])
    for t in range(T):
        rec = oses.ses_step(V, g, ubar, t, alpha, eta, rho, avg=avg)
        recs.append(rec)
        if rec["failed"]:
            break
        ubar = rec["ubar_next"]
    return recs, ubar


def dual_tol(D, lb):
    """Tolerance for the averaged QP bound sqrt(Abar - |Bbar|^2): the FP32
    moments carry an error of about eta2 = 1e-6 D^2 (a few ulp of D^2, the
    scale of |v_i - v_1|^2), which moves the square root by at most
    min(sqrt(eta2), eta2/lb); that is within RTOL D once lb >= D/10 and
    grows only where the averaged weights sit on nearly one point (lb -> 0)."""
    eta2 = 1e-6 * D * D
    return max(RTOL * D, min(math.sqrt(eta2), eta2 / max(lb, 1e-300)))


def compare_ses(gr, orr, gmean, omean, D):
    tol = RTOL * D
    assert len(orr) <= len(gr)
    for t, o in enumerate(orr):
        g = gr[t]
        assert g["status"] == 0
        assert abs(g["objective"] - o["objective"]) <= tol, (t, g["objective"], o["objective"])
        assert abs(g["oracle_value"] - o["oracle_value"]) <= tol, (t, g["oracle_value"], o["oracle_value"])
        assert abs(g["lower_bound"] - o["lower_bound"]) <= tol, (t, g["lower_bound"], o["lower_bound"])
        assert abs(g["dual_bound"] - o["dual_bound"]) <= dual_tol(D, o["dual_bound"]), (t, g["dual_bound"],
                                                                                        o["dual_bound"])
        if abs(o["oracle_value"]) > tol:
            assert bool(g["failed"]) == o["failed"], t
    assert np.linalg.norm(gmean - omean) <= tol, (gmean[:4], omean[:4])


def run_ses_case(n, d, seed=0, T=25, eta=0.5, rel_alpha=0.8, radii=False, dtype=torch.float32, dist="gauss"):
    V32 = datagen.ses_gaussian(n, d, seed) if dist == "gauss" else datagen.ses_uniform(n, d, seed)
    g32 = (0.1 * np.random.default_rng(seed).random(n)).astype(np.float32) if radii else None
    if dtype == torch.bfloat16:
        V = torch.from_numpy(V32).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    else:
        V = V32.astype(np.float64)
    g = None if g32 is None else g32.astype(np.float64)
    D = oses.ses_D(V, g)
    rho = oses.ses_width(D)
    alpha = rel_alpha * D
    gr, gmean = gpu_ses_traj(V32, g32, alpha, eta / rho, T, dtype)
    orr, omean = oracle_ses_traj(V, g, alpha, eta, rho, T)
    compare_ses(gr, orr, gmean, omean, D)
    return gr, orr


@pytest.mark.parametrize("n,d", [(1000, 2), (4099, 32), (3001, 3), (2500, 7), (1777, 33), (1500, 128),
                                 (600, 64), (900, 16), (513, 1), (257, 200)])
def test_ses_trajectory_matches_oracle(n, d):
    run_ses_case(n, d, seed=n + d)


def test_ses_config1_uniform_square():
    # n = 1000 points U[0,1]^2, seed 0 (the small SES workload)
    run_ses_case(1000, 2, seed=0, dist="uniform", T=25, eta=0.7)


def _load(V32, dtype):
    if dtype == torch.bfloat16:
        return torch.from_numpy(V32).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    return V32.astype(np.float64)


def forced_ses(n, d, seed, kDs, rel_alpha=0.8, radii=False, dtype=torch.float32, eta=0.5):
    """Single steps from checkpoints (t, ubar) chosen so that k D = eta t D / rho hits each kDs."""
    V32 = datagen.ses_gaussian(n, d, seed)
    g32 = (0.2 * np.random.default_rng(seed).random(n)).astype(np.float32) if radii else None
    V = _load(V32, dtype)
    g = None if g32 is None else g32.astype(np.float64)
    D = oses.ses_D(V, g)
    rho = oses.ses_width(D)
    alpha = rel_alpha * D
    pts = _cuda(V32).to(dtype)
    m = api.MWU(_ffi.SES, pts, radii=None if g32 is None else _cuda(g32))
    rng = np.random.default_rng(seed + 1)
    out = api.new_steps(len(kDs))
    ubars = []
    for j, kD in enumerate(kDs):
        t = max(1, int(round(kD * rho / (eta * D))))
        ubar = V.mean(axis=0) + 0.3 * D / math.sqrt(d) * rng.standard_normal(d)
        ubars.append((t, ubar))
        m.set(t, torch.from_numpy(ubar))
        m.step(alpha, eta / rho, out=out[j])
        mean, _ = m.read()
        torch.cuda.synchronize()
        # a checkpoint restarts the averaged bound: this step's weights alone
        o = oses.ses_step(V, g, ubar, t, alpha, eta, rho, avg=oses.ses_dual_state(d))
        r = api.decode_steps(out[j])[0]
        tol = RTOL * D
        assert r["status"] == 0 and r["t"] == (t + 1 if not o["failed"] else t)
        for key in ("objective", "oracle_value", "lower_bound"):
            assert abs(r[key] - o[key]) <= tol, (kD, key, r[key], o[key])
        assert abs(r["dual_bound"] - o["dual_bound"]) <= dual_tol(D, o["dual_bound"]), (kD, r["dual_bound"],
                                                                                         o["dual_bound"])
        assert np.linalg.norm(mean.cpu().numpy().astype(np.float64) - o["ubar_next"]) <= tol, kD


KDS = [1.0, 10.0, 40.0, 64.0]


@pytest.mark.parametrize("n,d", [(1000, 2), (4099, 32), (3001, 3), (2500, 7), (1777, 33), (1500, 128),
                                 (600, 64), (900, 16), (513, 1), (257, 200), (300, 1024)])
def test_ses_single_steps_match_oracle(n, d):
    forced_ses(n, d, seed=n + d, kDs=KDS)


def test_ses_single_steps_radii_and_bf16():
    forced_ses(2000, 8, seed=11, kDs=KDS, radii=True)
    forced_ses(3000, 32, seed=12, kDs=KDS, dtype=torch.bfloat16)
    forced_ses(1000, 12, seed=13, kDs=KDS, dtype=torch.bfloat16)


def test_ses_single_steps_full_size():
    # the benchmarked launch configuration: 1,000,000 points N(0, I_32)
    forced_ses(1_000_000, 32, seed=0, kDs=[10.0, 64.0], rel_alpha=2 / 3)


@pytest.mark.parametrize("n,d,dtype", [(100_000, 64, torch.float32), (100_000, 64, torch.bfloat16),
                                       (300_000, 16, torch.float32), (60_000, 128, torch.float32)])
def test_ses_single_steps_large_grids(n, d, dtype):
    # grids of one CTA per SM whose completion stages every partial row in
    # shared memory next to the kernel's static shared memory
    forced_ses(n, d, seed=d, kDs=[10.0, 64.0], dtype=dtype)


@pytest.mark.parametrize("d,dtype", [(64, torch.float32), (32, torch.bfloat16), (128, torch.float32),
                                     (128, torch.bfloat16)])
def test_svm_single_steps_large_grids(d, dtype):
    # d = 128: rows too wide to stage complete through the fixed-point column
    # accumulators; at k D = 64 from a random direction one class's weight sum
    # falls far below its bound and the completion falls back to the rows
    forced_svm(50_000, 50_000, d, seed=d, kDs=[10.0, 64.0], dtype=dtype)


def test_ses_with_radii():
    run_ses_case(2000, 8, seed=3, radii=True)


def test_ses_bf16_points():
    run_ses_case(3000, 32, seed=4, dtype=torch.bfloat16)
    run_ses_case(1000, 12, seed=5, dtype=torch.bfloat16)   # scalar bf16 path


def test_ses_separation_then_noop():
    # alpha well below OPT: the ORACLE separates; later steps leave the state alone
    gr, orr = run_ses_case(800, 4, seed=6, rel_alpha=0.45, T=40, eta=1.0)  # separates at t = 37
    assert orr[-1]["failed"]
    t_fail = len(orr) - 1
    assert gr[t_fail]["failed"] == 1 and gr[t_fail]["stopped"] == 1
    assert np.all(gr[t_fail + 1:]["t"] == 0)  # no record written after the stop


def test_ses_misaligned_points_take_scalar_path():
    V32 = datagen.ses_gaussian(1001, 8, seed=7)
    flat = torch.zeros(1001 * 8 + 1, dtype=torch.float32, device="cuda")
    flat[1:] = _cuda(V32).reshape(-1)
    mis = flat[1:].view(1001, 8)
    assert mis.data_ptr() % 16 != 0
    V = V32.astype(np.float64)
    D = oses.ses_D(V)
    rho = oses.ses_width(D)
    gr, gmean = gpu_ses_traj(V32, None, 0.8 * D, 0.5 / rho, 40, pts=mis)
    orr, omean = oracle_ses_traj(V, None, 0.8 * D, 0.5, rho, 40)
    compare_ses(gr, orr, gmean, omean, D)


def test_ses_duplicates_and_two_points():
    V32 = np.repeat(datagen.ses_gaussian(5, 3, seed=8), 40, axis=0)  # every point 40 times, incl. v_1
    run_V = V32.astype(np.float64)
    D = oses.ses_D(run_V)
    rho = oses.ses_width(D)
    gr, gmean = gpu_ses_traj(V32, None, 0.9 * D, 0.5 / rho, 40)
    orr, omean = oracle_ses_traj(run_V, None, 0.9 * D, 0.5, rho, 40)
    compare_ses(gr, orr, gmean, omean, D)
    # n = 2 at alpha = 1.01 > OPT = 1: u^1 = v_1, then every ORACLE answer is
    # v_1 + alpha e_1, so ubar^T = (T-1)/T * alpha e_1 exactly. (At alpha = OPT the
    # ORACLE value sqrt2 E2/S tends to 0 and its sign is decided by rounding.)
    two = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0]], dtype=np.float32)
    gr, gmean = gpu_ses_traj(two, None, 1.01, 1.0 / oses.ses_width(2.0), 50)
    assert np.allclose(gmean, [49 / 50 * 1.01, 0, 0], atol=1e-6)
    assert np.all(gr["failed"] == 0) and gr["t"][-1] == 50


def test_ses_completion_fallback_on_large_radii():
    """The fixed-point column totals assume |Wt| <= 2 n (2 |alpha| + 3 H + 2)
    with H bounding dist_i + gamma_i; at t = 0 (H = 0) over spheres whose
    radii far exceed alpha, Wt = sum 2 (alpha - gamma_i) breaks that bound and
    the finishing CTA falls back to reducing the CTAs' FP32 rows. The steps
    must still match the oracle (the first one through the fallback)."""
    rng = np.random.default_rng(41)
    V32 = (10.0 * rng.standard_normal((5000, 4))).astype(np.float32)
    g32 = rng.uniform(0.0, 40.0, 5000).astype(np.float32)
    V, g = V32.astype(np.float64), g32.astype(np.float64)
    D = oses.ses_D(V, g)
    rho = oses.ses_width(D)
    alpha = 0.02 * D
    assert 2.0 * np.sum(g[1:] - alpha) > 2.0 * 5000 * (2.0 * alpha + 2.0)  # beyond the bound at t = 0
    gr, gmean = gpu_ses_traj(V32, g32, alpha, 0.5 / rho, 5)
    orr, omean = oracle_ses_traj(V, g, alpha, 0.5, rho, 5)
    compare_ses(gr, orr, gmean, omean, D)


def test_ses_full_size_trajectory():
    # 1,000,000 points N(0, I_32), the benchmarked launch configuration: a few
    # iterations with the largest step Theorem 1 allows (eta = 1).
    run_ses_case(1_000_000, 32, seed=0, T=6, eta=1.0, rel_alpha=2 / 3)


# ----------------------------------------------------------------------------- SVM
def gpu_svm_traj(X32, y, alpha, eta_over_rho, D, T, dtype=torch.float32):
    pts = _cuda(X32).to(dtype)
    lab = _cuda(y)
    m = api.MWU(_ffi.SVM, pts, labels=lab)
    out = api.new_steps(T)
    for t in range(T):
        m.step(alpha, eta_over_rho, out=out[t], D=D)
    torch.cuda.synchronize()
    mean, _ = m.read()
    return api.decode_steps(out), mean.cpu().numpy().astype(np.float64)


def run_svm_case(n1, n2, d, seed=0, T=100, eta=0.5, rel_alpha=0.5, dtype=torch.float32, band=0.1):
    X32, y = datagen.svm_clusters(n1, n2, d, seed=seed, band=band)
    if dtype == torch.bfloat16:
        X = torch.from_numpy(X32).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    else:
        X = X32.astype(np.float64)
    D = osvm.svm_D(X)
    rho = osvm.svm_width(D)
    alpha = rel_alpha * D
    gr, gmean = gpu_svm_traj(X32, y, alpha, eta / rho, D, T, dtype)
    wbar, s1, s2 = np.zeros(d), 0.0, 0.0
    tol = RTOL * D
    avg = osvm.svm_dual_state(d)
    for t in range(T):
        o = osvm.svm_step(X, y, wbar, s1, s2, t, alpha, eta, rho, D, avg=avg)
        g = gr[t]
        assert g["status"] == 0
        assert abs(g["objective"] - o["objective"]) <= tol, (t, g["objective"], o["objective"])
        assert abs(g["oracle_value"] - o["oracle_value"]) <= tol, (t, g["oracle_value"], o["oracle_value"])
        assert abs(g["upper_bound"] - o["upper_bound"]) <= tol, (t, g["upper_bound"], o["upper_bound"])
        if t == 0:
            assert math.isinf(g["dual_bound"]) and math.isinf(o["dual_bound"])
        else:
            assert abs(g["dual_bound"] - o["dual_bound"]) <= tol, (t, g["dual_bound"], o["dual_bound"])
        if abs(o["oracle_value"]) > tol:
            assert bool(g["failed"]) == o["failed"]
        if o["failed"]:
            break
        wbar, s1, s2 = o["wbar_next"], o["s1bar_next"], o["s2bar_next"]
    assert np.linalg.norm(gmean[:d] - wbar) <= RTOL
    assert abs(gmean[d] - s1) <= tol and abs(gmean[d + 1] - s2) <= tol


def forced_svm(n1, n2, d, seed, kDs, dtype=torch.float32, eta=0.5, rel_alpha=0.5):
    X32, y = datagen.svm_clusters(n1, n2, d, seed=seed)
    X = _load(X32, dtype)
    D = osvm.svm_D(X)
    rho = osvm.svm_width(D)
    alpha = rel_alpha * D
    m = api.MWU(_ffi.SVM, _cuda(X32).to(dtype), labels=_cuda(y))
    rng = np.random.default_rng(seed + 1)
    out = api.new_steps(len(kDs))
    for j, kD in enumerate(kDs):
        t = max(1, int(round(kD * rho / (eta * D))))
        w = rng.standard_normal(d)
        w *= 0.9 / np.linalg.norm(w)
        s1, s2 = rng.uniform(-0.5, 1.0) * D, rng.uniform(-0.5, 1.0) * D
        m.set(t, torch.from_numpy(np.concatenate([w, [s1, s2]])), D=D)
        m.step(alpha, eta / rho, out=out[j], D=D)
        mean, _ = m.read()
        torch.cuda.synchronize()
        o = osvm.svm_step(X, y, w, s1, s2, t, alpha, eta, rho, D, avg=osvm.svm_dual_state(d))
        r = api.decode_steps(out[j])[0]
        tol = RTOL * D
        assert r["status"] == 0
        for key in ("objective", "oracle_value", "upper_bound", "dual_bound"):
            assert abs(r[key] - o[key]) <= tol, (kD, key, r[key], o[key])
        mm = mean.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(mm[:d] - o["wbar_next"]) <= RTOL
        assert abs(mm[d] - o["s1bar_next"]) <= tol and abs(mm[d + 1] - o["s2bar_next"]) <= tol


@pytest.mark.parametrize("n1,n2,d", [(2000, 1500, 16), (1000, 1001, 128), (700, 900, 3), (800, 800, 37),
                                     (300, 200, 1024)])
def test_svm_single_steps_match_oracle(n1, n2, d):
    forced_svm(n1, n2, d, seed=n1 + d, kDs=KDS)


def test_svm_single_steps_bf16_and_full_size():
    forced_svm(1500, 1500, 64, seed=9, kDs=KDS, dtype=torch.bfloat16)
    forced_svm(500_000, 500_000, 128, seed=0, kDs=[10.0, 64.0])


@pytest.mark.parametrize("n1,n2,d", [(2000, 1500, 16), (1000, 1001, 128), (700, 900, 3), (800, 800, 37)])
def test_svm_trajectory_matches_oracle(n1, n2, d):
    run_svm_case(n1, n2, d, seed=n1 + d)


def test_svm_bf16_points():
    run_svm_case(1500, 1500, 64, seed=9, dtype=torch.bfloat16)


def test_svm_full_size_sampled_parity():
    # 1,000,000 points in d = 128 (two clusters, ||mu|| = 3, band 0.1)
    run_svm_case(500_000, 500_000, 128, seed=0, T=4, eta=1.0)


# -------------------------------------------------------------------------- bounds
@pytest.mark.parametrize("n,d", [(1000, 2), (12345, 32), (777, 3), (4000, 128), (99, 1000)])
def test_bounds_match_oracle(n, d):
    V32 = datagen.ses_gaussian(n, d, seed=n)
    pts = _cuda(V32)
    V = V32.astype(np.float64)
    Dg = float(api.bounds(_ffi.SES, pts).item())
    assert math.isclose(Dg, oses.ses_D(V), rel_tol=1e-6)
    Dg = float(api.bounds(_ffi.SVM, pts).item())
    assert math.isclose(Dg, osvm.svm_D(V), rel_tol=1e-6)
    g32 = np.random.default_rng(n).random(n).astype(np.float32)
    Dg = float(api.bounds(_ffi.SES, pts, radii=_cuda(g32)).item())
    assert math.isclose(Dg, oses.ses_D(V, g32.astype(np.float64)), rel_tol=1e-6)


# --------------------------------------------------------------------------- solves
def test_ses_solve_against_welzl_and_oracle():
    V32 = datagen.ses_uniform(1000, 2, seed=0)
    V = V32.astype(np.float64)
    _, opt = exact.mec_2d(V)
    center, rep = api.ses_solve(_cuda(V32), eps=1e-2, max_iters=50_000)
    c = center.cpu().numpy().astype(np.float64)
    assert rep["lower_bound"] <= opt * (1 + 1e-6)
    assert rep["value"] >= opt * (1 - 1e-6)
    assert oses.ses_objective(V, None, c) <= rep["value"] * (1 + 1e-6)
    assert rep["value"] <= 1.01 * opt
    ref = oses.ses_solve(V, eps=1e-2, max_iters=50_000)
    assert abs(rep["value"] - ref["radius"]) <= 1e-2 * opt


def test_ses_solve_identical_points():
    pts = torch.ones((100, 5), dtype=torch.float32, device="cuda")
    center, rep = api.ses_solve(pts, eps=1e-3)
    assert rep["value"] == 0.0 and torch.allclose(center.cpu(), torch.ones(5))


def test_svm_solve_against_bruteforce():
    X32, y = datagen.svm_clusters(5, 5, 2, band=0.5, seed=7)
    X = X32.astype(np.float64)
    opt, _, _ = exact.pd_bruteforce(X[y > 0], X[y < 0])
    w, rep = api.svm_solve(_cuda(X32), _cuda(y), eps=1e-2, max_iters=20_000, eta=1.0)
    assert rep["lower_bound"] <= opt * (1 + 1e-5)
    assert rep["upper_bound"] >= opt * (1 - 1e-5)
    wn = w.cpu().numpy().astype(np.float64)
    assert math.isclose(exact.svm_margin_of(X[y > 0], X[y < 0], wn), rep["value"], rel_tol=1e-4)
    assert rep["value"] >= 0.97 * opt


@pytest.mark.parametrize("problem,n,d,dtype", [("ses", 5000, 32, torch.float32), ("ses", 3001, 5, torch.float32),
                                               ("ses", 4099, 32, torch.bfloat16), ("svm", 3000, 64, torch.float32)])
def test_mwu_run_equals_single_steps_bit_for_bit(problem, n, d, dtype):
    # k iterations launched back to back with dependent-launch overlap give the records and means of k
    # separate mwu_step calls exactly: the overlap changes when a launch starts, not what it computes
    k = 12
    if problem == "ses":
        V32 = datagen.ses_gaussian(n, d, seed=n)
        pts = _cuda(V32).to(dtype)
        D = oses.ses_D(V32.astype(np.float64))
        args = dict(alpha=0.8 * D, eta_over_rho=0.5 / oses.ses_width(D))
        make = lambda: api.MWU(_ffi.SES, pts)
        extra = {}
    else:
        X32, y = datagen.svm_clusters(n // 2, n - n // 2, d, seed=3)
        pts = _cuda(X32).to(dtype)
        D = osvm.svm_D(X32.astype(np.float64))
        args = dict(alpha=0.3 * D, eta_over_rho=0.5 / osvm.svm_width(D))
        lab = _cuda(y)
        make = lambda: api.MWU(_ffi.SVM, pts, labels=lab)
        extra = {"D": D}
    a, b = make(), make()
    out_a, out_b = api.new_steps(k), api.new_steps(k)
    for t in range(k):
        a.step(args["alpha"], args["eta_over_rho"], out=out_a[t], **extra)
    b.run(args["alpha"], args["eta_over_rho"], k, out=out_b, **extra)
    torch.cuda.synchronize()
    assert torch.equal(out_a, out_b)
    ma, ba = a.read()
    mb, bb = b.read()
    assert torch.equal(ma, mb) and torch.equal(ba, bb)
    assert api.decode_steps(out_b)[-1]["t"] == k
