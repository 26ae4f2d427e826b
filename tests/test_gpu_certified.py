"""CERTIFIED solves (ses_solve / svm_solve, mode "certified") on the GPU
against exact optima and the FP64 oracle's certified search.

Both searches draw only proven conclusions, so each one's report brackets
OPT; the GPU's trajectory differs from the oracle's by FP32 rounding (and
its decisions may fall one poll apart), so the two are compared through
what they certify: both brackets contain the exact optimum where one is
known, both close to within eps, and both radii (margins) lie within the
other's certified range.
"""

import math

import numpy as np
import pytest
import torch

from oracle import exact, ses as oses, svm as osvm
from paper_2405_09157_gb300 import api, datagen

pytestmark = pytest.mark.gpu
FP = 1e-5  # FP32 slack on a certified value (relative)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_ses_certified_brackets_welzl():
    V32 = datagen.ses_uniform(1000, 2, seed=0)
    V = V32.astype(np.float64)
    _, opt = exact.mec_2d(V)
    center, rep = api.ses_solve(_cuda(V32), eps=1e-3, mode="certified", max_iters=100_000, poll_every=64)
    assert rep["status"] == 0
    assert rep["lower_bound"] <= opt * (1 + FP) and rep["value"] >= opt * (1 - FP)
    assert rep["value"] <= (1 + 1e-3) * rep["lower_bound"]
    c = center.cpu().numpy().astype(np.float64)
    assert oses.ses_objective(V, None, c) <= rep["value"] * (1 + FP)


@pytest.mark.parametrize("n,d", [(2000, 8), (3000, 32)])
def test_ses_certified_matches_oracle(n, d):
    V32 = datagen.ses_gaussian(n, d, seed=1)
    V = V32.astype(np.float64)
    ref = oses.ses_solve(V, eps=1e-3, mode="certified", max_iters=100_000, poll_every=64)
    center, rep = api.ses_solve(_cuda(V32), eps=1e-3, mode="certified", max_iters=100_000, poll_every=64)
    assert rep["status"] == 0 and ref["radius"] <= (1 + 1e-3) * ref["lower_bound"]
    assert rep["value"] <= (1 + 1e-3) * rep["lower_bound"]
    # each certified interval contains the other's ball radius and lower bound
    assert rep["lower_bound"] <= ref["radius"] * (1 + FP) and ref["lower_bound"] <= rep["value"] * (1 + FP)
    assert abs(rep["value"] - ref["radius"]) <= 1e-3 * ref["radius"]
    c = center.cpu().numpy().astype(np.float64)
    assert oses.ses_objective(V, None, c) <= rep["value"] * (1 + FP)
    # the GPU's iteration count is the oracle's up to the decisions FP32 moves by a poll or a step
    assert rep["iters"] <= 3 * ref["iters"] + 4096


def test_ses_certified_spheres_use_primal_bound_only():
    V32 = datagen.ses_gaussian(1500, 4, seed=3)
    g32 = (0.2 * np.random.default_rng(3).random(1500)).astype(np.float32)
    center, rep = api.ses_solve(_cuda(V32), radii=_cuda(g32), eps=1e-2, mode="certified", max_iters=60_000,
                                poll_every=64)
    V, g = V32.astype(np.float64), g32.astype(np.float64)
    c = center.cpu().numpy().astype(np.float64)
    assert oses.ses_objective(V, g, c) <= rep["value"] * (1 + FP)
    assert rep["lower_bound"] <= rep["value"]
    ref = oses.ses_solve(V, g, eps=1e-2, mode="certified", max_iters=60_000, poll_every=64)
    assert rep["lower_bound"] <= ref["radius"] * (1 + FP) and ref["lower_bound"] <= rep["value"] * (1 + FP)


def test_svm_certified_brackets_bruteforce():
    X32, y = datagen.svm_clusters(5, 5, 2, band=0.5, seed=7)
    X = X32.astype(np.float64)
    opt, _, _ = exact.pd_bruteforce(X[y > 0], X[y < 0])
    w, rep = api.svm_solve(_cuda(X32), _cuda(y), eps=1e-3, mode="certified", max_iters=100_000, poll_every=64)
    assert rep["status"] == 0
    assert rep["lower_bound"] <= opt * (1 + FP) and rep["upper_bound"] >= opt * (1 - FP)
    assert rep["upper_bound"] <= (1 + 1e-3) * rep["lower_bound"]
    wn = w.cpu().numpy().astype(np.float64)
    assert math.isclose(exact.svm_margin_of(X[y > 0], X[y < 0], wn), rep["value"], rel_tol=1e-4)


def test_svm_certified_matches_oracle():
    X32, y = datagen.svm_clusters(300, 300, 16, seed=1)
    X = X32.astype(np.float64)
    ref = osvm.svm_solve(X, y, eps=1e-2, mode="certified", max_iters=60_000, poll_every=64)
    w, rep = api.svm_solve(_cuda(X32), _cuda(y), eps=1e-2, mode="certified", max_iters=60_000, poll_every=64)
    assert rep["status"] == 0 and ref["upper_bound"] <= (1 + 1e-2) * ref["lower_bound"]
    assert rep["upper_bound"] <= (1 + 1e-2) * rep["lower_bound"]
    assert rep["lower_bound"] <= ref["upper_bound"] * (1 + FP) and ref["lower_bound"] <= rep["upper_bound"] * (1 + FP)


def test_ses_certified_full_size():
    # the benchmarked workload: n = 1e6, d = 32, N(0, I), eps = 1e-3
    V32 = datagen.ses_gaussian(1_000_000, 32, seed=0)
    center, rep = api.ses_solve(_cuda(V32), eps=1e-3, mode="certified", max_iters=200_000, poll_every=256)
    assert rep["status"] == 0
    assert rep["value"] <= (1 + 1e-3) * rep["lower_bound"]
    # the centre's radius, recomputed in FP64 over all points, is the reported one
    c = center.cpu().numpy().astype(np.float64)
    r = float(np.sqrt(np.max(np.sum((V32.astype(np.float64) - c) ** 2, axis=1))))
    assert abs(r - rep["value"]) <= FP * r


@pytest.mark.parametrize("name", ["two points", "d = 1", "duplicates", "collinear"])
def test_ses_certified_degenerate_inputs(name):
    rng = np.random.default_rng(5)
    V = {"two points": np.array([[0.0, 0.0], [3.0, 4.0]]),
         "d = 1": rng.standard_normal((50, 1)),
         "duplicates": np.repeat(rng.standard_normal((5, 2)), 10, axis=0),
         "collinear": np.outer(np.linspace(-1, 2, 40), [1.0, 2.0, -1.0])}[name].astype(np.float32)
    V64 = V.astype(np.float64)
    if V.shape[1] == 2:
        opt = exact.mec_2d(V64)[1]
    elif V.shape[1] == 1:
        opt = 0.5 * float(V64.max() - V64.min())
    else:
        opt = 0.5 * float(np.max(np.linalg.norm(V64[:, None, :] - V64[None, :, :], axis=2)))  # collinear: half the diameter
    center, rep = api.ses_solve(_cuda(V), eps=1e-3, mode="certified", max_iters=100_000, poll_every=64)
    assert rep["status"] == 0
    assert rep["lower_bound"] <= opt * (1 + FP) <= rep["value"] * (1 + FP) + 1e-6
    assert rep["value"] <= (1 + 1e-3) * rep["lower_bound"] * (1 + FP)
    assert oses.ses_objective(V64, None, center.cpu().numpy().astype(np.float64)) <= rep["value"] * (1 + FP)


def test_svm_certified_not_separable():
    # both classes from one distribution: OPT = 0. No direction has a positive margin, so the search
    # spends its budget (status 5) with margin 0 and a Claim 8 bound that shrinks towards 0 (the oracle
    # reaches 0.017 on this set within the same budget)
    rng = np.random.default_rng(0)
    X = rng.standard_normal((200, 3)).astype(np.float32)
    y = np.where(np.arange(200) < 100, 1, -1).astype(np.int8)
    w, rep = api.svm_solve(_cuda(X), _cuda(y), eps=1e-2, mode="certified", max_iters=20_000, poll_every=64)
    assert rep["status"] == 5
    assert rep["value"] == 0.0 and rep["lower_bound"] == 0.0
    assert 0.0 <= rep["upper_bound"] < 0.1
    ref = osvm.svm_solve(X.astype(np.float64), y, eps=1e-2, mode="certified", max_iters=20_000, poll_every=64)
    assert ref["margin"] == 0.0 and ref["upper_bound"] < 0.1


def test_ses_certified_bf16_points():
    # BF16-stored points: a certified ball of the BF16-rounded point set (the oracle gets the same values)
    V32 = datagen.ses_gaussian(3000, 16, seed=4)
    pb = _cuda(V32).to(torch.bfloat16)
    V = pb.to(torch.float32).cpu().numpy().astype(np.float64)
    center, rep = api.ses_solve(pb, eps=1e-3, mode="certified", max_iters=100_000, poll_every=64)
    ref = oses.ses_solve(V, eps=1e-3, mode="certified", max_iters=100_000, poll_every=64)
    assert rep["status"] == 0 and rep["value"] <= (1 + 1e-3) * rep["lower_bound"]
    assert rep["lower_bound"] <= ref["radius"] * (1 + FP) and ref["lower_bound"] <= rep["value"] * (1 + FP)
    assert oses.ses_objective(V, None, center.cpu().numpy().astype(np.float64)) <= rep["value"] * (1 + FP)


def _margin64(X, y, w):
    return exact.svm_margin_of(X[y > 0], X[y < 0], w.cpu().numpy().astype(np.float64))


def test_svm_coreset_matches_oracle_d128():
    # core-set certificates (mode "coreset") at d = 128: both searches bracket the exact optimum
    # (MDM on all 10,000 points) and close to eps = 1e-3
    X32, y = datagen.svm_clusters(5000, 5000, 128, seed=2)
    X = X32.astype(np.float64)
    opt = exact.pd_mdm(X[y > 0], X[y < 0], tol=1e-10)[0]
    ref = osvm.svm_solve(X, y, eps=1e-3, mode="coreset", max_iters=20_000, poll_every=64)
    w, rep = api.svm_solve(_cuda(X32), _cuda(y), eps=1e-3, mode="coreset", max_iters=20_000, poll_every=64)
    assert ref["upper_bound"] <= (1 + 1e-3) * ref["lower_bound"]
    assert rep["status"] == 0 and rep["upper_bound"] <= (1 + 1e-3) * rep["lower_bound"]
    assert rep["lower_bound"] <= opt * (1 + FP) and rep["upper_bound"] >= opt * (1 - FP)
    assert ref["lower_bound"] <= opt * (1 + FP) and ref["upper_bound"] >= opt * (1 - FP)
    assert math.isclose(_margin64(X, y, w), rep["value"], rel_tol=1e-4)
    # the first check (256 iterations of the search) closes it in both
    assert rep["iters"] <= 2 * 256 and ref["iters"] <= 2 * 256


def test_svm_coreset_small_classes_take_every_point():
    # classes of at most 512 points: the first core set is the whole set, its distance is OPT
    X32, y = datagen.svm_clusters(300, 200, 16, seed=3)
    X = X32.astype(np.float64)
    opt = exact.pd_mdm(X[y > 0], X[y < 0], tol=1e-12)[0]
    w, rep = api.svm_solve(_cuda(X32), _cuda(y), eps=1e-3, mode="coreset", max_iters=20_000, poll_every=64)
    assert rep["status"] == 0
    assert opt * (1 - 1e-9) <= rep["upper_bound"] <= opt * (1 + 1e-4)  # core-set solve to a gap of eps/10
    assert rep["lower_bound"] <= opt * (1 + FP) and rep["lower_bound"] >= opt * (1 - 1e-3)
    assert math.isclose(_margin64(X, y, w), rep["value"], rel_tol=1e-4)


def test_svm_coreset_bf16_points():
    # BF16-stored points: certificates of the BF16-rounded set
    X32, y = datagen.svm_clusters(4000, 3000, 64, seed=4)
    xb = _cuda(X32).to(torch.bfloat16)
    X = xb.to(torch.float32).cpu().numpy().astype(np.float64)
    opt = exact.pd_mdm(X[y > 0], X[y < 0], tol=1e-10)[0]
    w, rep = api.svm_solve(xb, _cuda(y), eps=1e-3, mode="coreset", max_iters=20_000, poll_every=64)
    assert rep["status"] == 0 and rep["upper_bound"] <= (1 + 1e-3) * rep["lower_bound"]
    assert rep["lower_bound"] <= opt * (1 + FP) and rep["upper_bound"] >= opt * (1 - FP)
    assert math.isclose(_margin64(X, y, w), rep["value"], rel_tol=1e-4)


def test_svm_coreset_full_size():
    # the benchmarked SVM workload: n1 = n2 = 5e5, d = 128, eps = 1e-3
    X32, y = datagen.svm_clusters(500_000, 500_000, 128, seed=0)
    w, rep = api.svm_solve(_cuda(X32), _cuda(y), eps=1e-3, mode="coreset", max_iters=200_000, poll_every=256)
    assert rep["status"] == 0 and rep["upper_bound"] <= (1 + 1e-3) * rep["lower_bound"]
    assert math.isclose(_margin64(X32.astype(np.float64), y, w), rep["value"], rel_tol=1e-4)


# ---------------------------------------------------------------- SES core sets
@pytest.mark.parametrize("n,seed", [(3000, 0), (20_000, 1), (2, 2), (700, 3)])
def test_ses_coreset_brackets_welzl_in_the_plane(n, seed):
    """SES core-set mode on points in the plane against Welzl's exact radius:
    the certificates bracket it and close within eps (the returned centre's
    ball encloses every point)."""
    from oracle import exact
    V32 = datagen.ses_uniform(n, 2, seed=seed)
    V = V32.astype(np.float64)
    opt = exact.mec_2d(V)[1]
    eps = 1e-3
    c, rep = api.ses_solve(torch.from_numpy(V32).cuda(), eps=eps, mode="coreset", max_iters=100_000)
    assert rep["status"] == 0, rep
    assert rep["lower_bound"] <= opt * (1 + FP) and rep["upper_bound"] >= opt * (1 - FP), (rep, opt)
    assert rep["upper_bound"] <= (1 + eps) * rep["lower_bound"]
    far = float(np.linalg.norm(V - c.cpu().numpy().astype(np.float64), axis=1).max())
    assert far <= rep["upper_bound"] * (1 + FP), (far, rep["upper_bound"])


def test_ses_coreset_full_size_closes_early():
    """The benchmark workload (n = 1e6, d = 32, N(0, I)): the core-set mode
    closes eps = 1e-3 within the first checks, its centre's ball encloses
    every point, and its interval and the plain CERTIFIED mode's overlap."""
    V32 = datagen.ses_gaussian(1_000_000, 32, seed=0)
    pts = torch.from_numpy(V32).cuda()
    eps = 1e-3
    c, rep = api.ses_solve(pts, eps=eps, mode="coreset", max_iters=200_000)
    assert rep["status"] == 0, rep
    assert rep["iters"] <= 1024, rep
    assert rep["upper_bound"] <= (1 + eps) * rep["lower_bound"]
    V = V32.astype(np.float64)
    far = float(np.linalg.norm(V - c.cpu().numpy().astype(np.float64), axis=1).max())
    assert far <= rep["upper_bound"] * (1 + FP)
    _, rep2 = api.ses_solve(pts, eps=eps, mode="certified", max_iters=200_000)
    assert rep["lower_bound"] <= rep2["upper_bound"] * (1 + FP) and rep2["lower_bound"] <= rep["upper_bound"] * (1 + FP)


def test_ses_coreset_with_radii_is_certified():
    """With radii the core-set mode runs as CERTIFIED: same report."""
    V32 = datagen.ses_uniform(500, 3, seed=4)
    g = np.random.default_rng(4).random(500).astype(np.float32) * 0.05
    pts = torch.from_numpy(V32).cuda()
    rad = torch.from_numpy(g).cuda()
    _, a = api.ses_solve(pts, radii=rad, eps=1e-2, mode="coreset", max_iters=50_000)
    _, b = api.ses_solve(pts, radii=rad, eps=1e-2, mode="certified", max_iters=50_000)
    assert a["iters"] == b["iters"] and a["upper_bound"] == b["upper_bound"] and a["lower_bound"] == b["lower_bound"]
