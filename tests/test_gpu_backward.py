"""Reverse sweep (mwu_backward) against the FP64 autograd oracle, through the C ABI.

Tolerance. The forward runs in FP32 per point (relative error ~k D 2^-24 per
weight, k D <= 10 here) and the sweep differentiates the same FP32 values, so
the GPU gradient differs from the FP64 one by the sensitivity of the gradient
to those perturbations. Gradients are compared in the max norm relative to the
largest entry, at GRAD_RTOL = 2e-4, over trajectories short enough (T <= 15)
that the alpha-FTP dynamics do not amplify rounding (see test_gpu_parity.py).
At the full size the oracle is out of reach; there the sweep is checked
against identities that hold at any size: f is invariant under a common
translation of all points (so the rows of the gradient sum to zero) and
equivariant under rotations (so sum_i v_i grad_i^T is symmetric).
"""

import numpy as np
import pytest
import torch

from oracle import ses as oses
from oracle import ses_grad
from paper_2405_09157_gb300 import _ffi, api, datagen

pytestmark = pytest.mark.gpu
RTOL = 1e-5
GRAD_RTOL = 2e-4


def _case(n, d, seed, radii, rel_alpha=0.9):
    V32 = datagen.ses_gaussian(n, d, seed)
    g32 = (0.1 * np.random.default_rng(seed).random(n)).astype(np.float32) if radii else None
    V = V32.astype(np.float64)
    g = None if g32 is None else g32.astype(np.float64)
    D = oses.ses_D(V, g)
    return V32, g32, V, g, D, rel_alpha * D, oses.ses_width(D)


def _gpu(V32, g32, alpha, eor, T, seed=None):
    pts = torch.from_numpy(V32).cuda()
    radii = None if g32 is None else torch.from_numpy(g32).cuda()
    out = api.new_steps(1)
    grad, _ = api.mwu_backward(pts, alpha, eor, T, radii=radii, seed=seed, out=out)
    torch.cuda.synchronize()
    return grad.cpu().numpy().astype(np.float64), api.decode_steps(out)[0]


@pytest.mark.parametrize("n,d,T,radii", [(300, 3, 10, False), (2000, 8, 15, True), (5000, 32, 12, False),
                                         (20000, 64, 8, False), (1001, 5, 6, True), (4099, 16, 15, False),
                                         (2, 3, 5, False)])
def test_backward_matches_oracle(n, d, T, radii):
    V32, g32, V, g, D, alpha, rho = _case(n, d, 21, radii)
    eta = 0.5
    L, want, steps = ses_grad.ses_unrolled_radius_grad(V, g, alpha, eta / rho, T)
    got, rec = _gpu(V32, g32, alpha, eta / rho, T)
    assert rec["status"] == 0 and rec["t"] == steps == T
    assert abs(rec["objective"] - L) <= RTOL * D
    # entries of the gradient of a radius with respect to the points are O(1):
    # the bound is relative to the largest entry, with 1 as its floor (for the
    # two-point case, whose radius alpha (T-1)/T does not depend on the points)
    scale = max(np.max(np.abs(want)), 1.0)
    err = np.max(np.abs(got - want))
    assert err <= GRAD_RTOL * scale, (err / scale, np.unravel_index(np.argmax(np.abs(got - want)), want.shape))


def test_backward_after_separation_differentiates_the_steps_taken():
    # alpha below OPT: the forward separates at some t_f < T (the run of test_ses_separation_then_noop)
    V32, _, V, _, D, _, rho = _case(800, 4, 6, False)
    alpha, eta, T = 0.45 * D, 1.0, 40
    L, want, steps = ses_grad.ses_unrolled_radius_grad(V, None, alpha, eta / rho, T)
    assert steps < T
    got, rec = _gpu(V32, None, alpha, eta / rho, T)
    assert rec["t"] == steps and rec["failed"] == 1
    assert abs(rec["objective"] - L) <= RTOL * D
    assert np.max(np.abs(got - want)) <= GRAD_RTOL * np.max(np.abs(want))


def test_one_iteration_closed_form_and_seed():
    V32, _, V, _, D, alpha, rho = _case(500, 8, 9, False)
    seed = torch.tensor([2.5], dtype=torch.float64, device="cuda")
    got, rec = _gpu(V32, None, alpha, 0.5 / rho, 1, seed=seed)
    dist = np.linalg.norm(V - V[0], axis=1)
    k = int(np.argmax(dist))
    want = np.zeros_like(V)
    want[0] = 2.5 * (V[0] - V[k]) / dist[k]
    want[k] = -want[0]
    assert int(rec["k"]) == k and rec["t"] == 1
    assert np.max(np.abs(got - want)) <= 1e-6


def test_autograd_function_matches_the_sweep():
    V32, _, V, _, D, alpha, rho = _case(3000, 16, 4, False)
    eor, T = 0.5 / rho, 10
    pts = torch.from_numpy(V32).cuda().requires_grad_(True)
    f = api.ses_unrolled_radius(pts, alpha, eor, T)
    (3.0 * f).backward()
    direct, _ = api.mwu_backward(pts.detach(), alpha, eor, T)
    torch.cuda.synchronize()
    assert torch.allclose(pts.grad, 3.0 * direct, rtol=1e-6, atol=1e-7)
    L, _, _ = ses_grad.ses_unrolled_radius_grad(V, None, alpha, eor, T)
    assert abs(float(f.detach()) - L) <= RTOL * D


@pytest.mark.parametrize("n,d,T", [(100_000, 64, 2000), (200_000, 32, 300)])
def test_full_size_invariances(n, d, T):
    V32, _, V, _, D, alpha, rho = _case(n, d, 0, False, rel_alpha=1.0)
    eta = 0.5
    got, rec = _gpu(V32, None, alpha, eta / rho, T)
    assert rec["status"] == 0 and rec["t"] == T and np.all(np.isfinite(got))
    tot = np.abs(got).sum(axis=0)
    # translation invariance: sum_i dL/dv_i = 0
    assert np.all(np.abs(got.sum(axis=0)) <= 1e-4 * np.maximum(tot, 1e-30) + 1e-6)
    # rotation equivariance: sum_i v_i grad_i^T is symmetric
    Mv = V.T @ got
    assert np.max(np.abs(Mv - Mv.T)) <= 1e-4 * np.abs(V).max() * tot.sum() + 1e-6


# --- SVM: margin of the minimisation alpha-FTP -------------------------------

from oracle import svm as osvm  # noqa: E402
from oracle import svm_grad  # noqa: E402


def _svm_case(n1, n2, d, seed):
    X32, y = datagen.svm_clusters(n1, n2, d, mu_norm=3.0, band=0.5, seed=seed)
    X = X32.astype(np.float64)
    D = osvm.svm_D(X)
    return X32, y, X, D, osvm.svm_width(D)


def _svm_gpu(X32, y, alpha, eor, T, D, seed=None):
    pts = torch.from_numpy(X32).cuda()
    lab = torch.from_numpy(y).cuda()
    out = api.new_steps(1)
    grad, _ = api.mwu_backward(pts, alpha, eor, T, seed=seed, out=out, problem=_ffi.SVM, labels=lab, D=D)
    torch.cuda.synchronize()
    return grad.cpu().numpy().astype(np.float64), api.decode_steps(out)[0]


@pytest.mark.parametrize("n1,n2,d,T", [(60, 50, 3, 10), (700, 900, 8, 15), (2000, 1500, 32, 12),
                                       (3000, 3000, 64, 8), (500, 400, 5, 6), (1, 1, 4, 5)])
def test_svm_backward_matches_oracle(n1, n2, d, T):
    X32, y, X, D, rho = _svm_case(n1, n2, d, 31)
    alpha, eta = 0.2 * D, 0.5
    L, want, steps = svm_grad.svm_unrolled_margin_grad(X, y, alpha, eta / rho, D, T)
    got, rec = _svm_gpu(X32, y, alpha, eta / rho, T, D)
    assert rec["status"] == 0 and rec["t"] == steps == T
    assert abs(rec["objective"] - L) <= RTOL * D
    scale = max(np.max(np.abs(want)), 1.0)
    err = np.max(np.abs(got - want))
    assert err <= GRAD_RTOL * scale, (err / scale, np.unravel_index(np.argmax(np.abs(got - want)), want.shape))


def test_svm_one_iteration_closed_form_and_seed():
    X32, y, X, D, rho = _svm_case(300, 200, 6, 9)
    n = X.shape[0]
    seed = torch.tensor([2.0], dtype=torch.float64, device="cuda")
    got, rec = _svm_gpu(X32, y, 0.1 * D, 0.5 / rho, 1, D, seed=seed)
    z = (X[y > 0].sum(axis=0) - X[y < 0].sum(axis=0)) / n
    w = z / np.linalg.norm(z)
    s = X @ w
    iP = np.flatnonzero(y > 0)[np.argmin(s[y > 0])]
    iQ = np.flatnonzero(y < 0)[np.argmax(s[y < 0])]
    proj = (np.eye(6) - np.outer(w, w)) @ (X[iP] - X[iQ]) / np.linalg.norm(z)
    want = np.outer(y.astype(np.float64) / n, proj)
    want[iP] += w
    want[iQ] -= w
    assert int(rec["k"]) == iP and abs(rec["objective"] - (s[iP] - s[iQ])) <= RTOL * D
    assert np.max(np.abs(got - 2.0 * want)) <= 1e-5


def test_svm_autograd_function_matches_the_sweep():
    X32, y, X, D, rho = _svm_case(1500, 1200, 16, 12)
    eor, T = 0.5 / rho, 10
    pts = torch.from_numpy(X32).cuda().requires_grad_(True)
    lab = torch.from_numpy(y).cuda()
    f = api.svm_unrolled_margin(pts, lab, 0.2 * D, eor, T, D)
    (1.5 * f).backward()
    direct, _ = api.mwu_backward(pts.detach(), 0.2 * D, eor, T, problem=_ffi.SVM, labels=lab, D=D)
    torch.cuda.synchronize()
    assert torch.allclose(pts.grad, 1.5 * direct, rtol=1e-6, atol=1e-7)
    L, _, _ = svm_grad.svm_unrolled_margin_grad(X, y, 0.2 * D, eor, D, T)
    assert abs(float(f.detach()) - L) <= RTOL * D


def test_svm_full_size_rotation_identity():
    # the margin and the whole alpha-FTP are rotation equivariant, so sum_i x_i grad_i^T is symmetric
    # alpha = 0.05 D (about 0.55) stays below OPT >= 1 (the band 0.5 on both sides of the Bayes
    # hyperplane), so the ORACLE never separates and all 500 iterations are differentiated
    X32, y, X, D, rho = _svm_case(50_000, 50_000, 64, 0)
    got, rec = _svm_gpu(X32, y, 0.05 * D, 0.5 / rho, 500, D)
    assert rec["status"] == 0 and rec["t"] == 500 and rec["objective"] > 0 and np.all(np.isfinite(got))
    M = X.T @ got
    tot = np.abs(got).sum()
    assert np.max(np.abs(M - M.T)) <= 1e-4 * np.abs(X).max() * tot + 1e-6


# --- bfloat16 points --------------------------------------------------------
# The sweep reads BF16 rows and widens them to FP32 on load; the gradient is the
# one of the BF16-rounded point set, so the oracle runs on those values (exact
# in FP64) and the tolerance is the FP32 one above.


def _bf16(a32):
    """(bf16 CUDA tensor, its values as float64 numpy)."""
    pb = torch.from_numpy(a32).cuda().to(torch.bfloat16)
    return pb, pb.float().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("n,d,T,radii", [(3000, 32, 12, False), (2000, 8, 15, True), (1001, 5, 6, True),
                                         (4099, 16, 10, False), (20000, 64, 8, False), (300, 3, 10, False)])
def test_backward_bf16_points_match_oracle(n, d, T, radii):
    V32, g32, _, g, _, _, _ = _case(n, d, 23, radii)
    pb, V = _bf16(V32)
    D = oses.ses_D(V, g)
    alpha, rho, eta = 0.9 * D, oses.ses_width(D), 0.5
    L, want, steps = ses_grad.ses_unrolled_radius_grad(V, g, alpha, eta / rho, T)
    out = api.new_steps(1)
    radii_t = None if g32 is None else torch.from_numpy(g32).cuda()
    grad, _ = api.mwu_backward(pb, alpha, eta / rho, T, radii=radii_t, out=out)
    torch.cuda.synchronize()
    rec = api.decode_steps(out)[0]
    assert grad.dtype == torch.float32 and grad.shape == (n, d)
    assert rec["status"] == 0 and rec["t"] == steps == T
    assert abs(rec["objective"] - L) <= RTOL * D
    got = grad.cpu().numpy().astype(np.float64)
    scale = max(np.max(np.abs(want)), 1.0)
    assert np.max(np.abs(got - want)) <= GRAD_RTOL * scale


def test_backward_bf16_rows_not_8_byte_aligned():
    # a view starting 2 elements (4 bytes) into its buffer takes the per-element path
    n, d, T = 1500, 8, 10
    V32, _, _, _, _, _, _ = _case(n, d, 24, False)
    buf = torch.zeros(n * d + 2, dtype=torch.bfloat16, device="cuda")
    buf[2:] = torch.from_numpy(V32).cuda().reshape(-1).to(torch.bfloat16)
    pb = buf[2:].view(n, d)
    assert pb.data_ptr() % 8 == 4
    V = pb.float().cpu().numpy().astype(np.float64)
    D = oses.ses_D(V)
    alpha, rho, eta = 0.9 * D, oses.ses_width(D), 0.5
    L, want, _ = ses_grad.ses_unrolled_radius_grad(V, None, alpha, eta / rho, T)
    grad, _ = api.mwu_backward(pb, alpha, eta / rho, T)
    got = grad.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - want)) <= GRAD_RTOL * max(np.max(np.abs(want)), 1.0)


@pytest.mark.parametrize("n1,n2,d,T", [(700, 900, 8, 15), (2000, 1500, 32, 12), (500, 400, 5, 6)])
def test_svm_backward_bf16_points_match_oracle(n1, n2, d, T):
    X32, y = datagen.svm_clusters(n1, n2, d, mu_norm=3.0, band=0.5, seed=33)
    pb, X = _bf16(X32)
    D = osvm.svm_D(X)
    rho, alpha, eta = osvm.svm_width(D), 0.2 * D, 0.5
    L, want, steps = svm_grad.svm_unrolled_margin_grad(X, y, alpha, eta / rho, D, T)
    out = api.new_steps(1)
    grad, _ = api.mwu_backward(pb, alpha, eta / rho, T, out=out, problem=_ffi.SVM,
                               labels=torch.from_numpy(y).cuda(), D=D)
    torch.cuda.synchronize()
    rec = api.decode_steps(out)[0]
    assert rec["status"] == 0 and rec["t"] == steps == T
    assert abs(rec["objective"] - L) <= RTOL * D
    got = grad.cpu().numpy().astype(np.float64)
    scale = max(np.max(np.abs(want)), 1.0)
    assert np.max(np.abs(got - want)) <= GRAD_RTOL * scale
