"""Batched SVM (one launch per iteration for many instances) against the FP64
oracle, instance by instance: trajectories of the minimisation alpha-FTP
(Sec. 3, Eq. min_implement; Sec. 4.2) at the per-step tolerance of
test_gpu_parity.py, D = max ||x_i|| per instance, and the device-side search
of svm_solve (certified and practical modes) against exact polytope
distances and the single-instance solve."""

import math

import numpy as np
import pytest
import torch

from oracle import exact, svm as osvm
from paper_2405_09157_gb300 import api, datagen

pytestmark = pytest.mark.gpu
RTOL = 1e-5
FP = 1e-5

# (n1, n2, d): ragged sizes, every lane layout (d % 4 == 0 chunks for d = 4 .. 64, scalar otherwise)
SHAPES = [(1, 1, 2), (3, 2, 3), (50, 40, 8), (700, 500, 16), (3000, 2000, 32), (5000, 5001, 64), (600, 634, 5),
          (250, 250, 3), (2049, 2050, 2), (4100, 4100, 33), (1000, 1049, 4), (700, 800, 12), (32, 32, 64),
          (150, 150, 1)]


def _instances(shapes, seed0, dtype=torch.float32):
    X32s, ys = [], []
    for k, (n1, n2, d) in enumerate(shapes):
        X32, y = datagen.svm_clusters(n1, n2, d, seed=seed0 + k, band=0.1)
        X32s.append(X32 * np.float32(1.0 + 0.5 * k))  # instance scales differ
        ys.append(y)
    pts, offs, n, d = api.pack_instances(X32s, dtype=dtype)
    lab, loffs = api.pack_labels(ys)
    if dtype == torch.bfloat16:  # the oracle sees the rounded values
        Xs = [torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64) for x in X32s]
    else:
        Xs = [x.astype(np.float64) for x in X32s]
    return pts, offs, n, d, lab, loffs, Xs, ys


def _trajectories(dtype):
    pts, offs, n, d, lab, loffs, Xs, ys = _instances(SHAPES, 500, dtype)
    batch = api.SvmBatch(pts, offs, n, d, lab, loffs, tile_rows=512)
    D = np.array([osvm.svm_D(X) for X in Xs])
    rho = np.array([osvm.svm_width(x) for x in D])
    _, _, Dg = batch.read()
    assert np.allclose(Dg, D, rtol=1e-12, atol=0.0), (Dg, D)
    alpha = 0.5 * D
    eta, T = 0.5, 20
    a_dev = torch.tensor(alpha, dtype=torch.float64, device="cuda")
    e_dev = torch.tensor(eta / rho, dtype=torch.float64, device="cuda")
    outs = [api.new_steps(len(SHAPES)) for _ in range(T)]
    for t in range(T):
        batch.step(a_dev, e_dev, out=outs[t])
    torch.cuda.synchronize()
    recs = [api.decode_steps(o) for o in outs]
    means, _, _ = batch.read()
    for k, (n1, n2, dk) in enumerate(SHAPES):
        X, y = Xs[k], ys[k]
        wbar, s1, s2 = np.zeros(dk), 0.0, 0.0
        avg = osvm.svm_dual_state(dk)
        tol = RTOL * D[k]
        for t in range(T):
            o = osvm.svm_step(X, y, wbar, s1, s2, t, alpha[k], eta, rho[k], D[k], avg=avg)
            r = recs[t][k]
            assert r["status"] == 0, (k, t)
            for key in ("objective", "oracle_value", "upper_bound"):
                assert abs(r[key] - o[key]) <= tol, (k, SHAPES[k], t, key, r[key], o[key])
            if t > 0:
                assert abs(r["dual_bound"] - o["dual_bound"]) <= tol, (k, t, r["dual_bound"], o["dual_bound"])
            if abs(o["oracle_value"]) > tol:
                assert bool(r["failed"]) == o["failed"], (k, t)
            if o["failed"]:
                break
            wbar, s1, s2 = o["wbar_next"], o["s1bar_next"], o["s2bar_next"]
        assert np.linalg.norm(means[k].astype(np.float64) - wbar) <= RTOL, (k, SHAPES[k])


def test_svm_batch_trajectories_match_oracle_per_instance():
    _trajectories(torch.float32)


def test_svm_batch_bf16_trajectories_match_oracle_per_instance():
    _trajectories(torch.bfloat16)


def test_svm_batch_misaligned_rows_take_the_scalar_layouts():
    # instances whose rows start one element off a 4-element boundary (d % 4 == 0 would otherwise
    # take 16-byte chunk loads): same trajectory as the aligned packing
    shapes = [(400, 300, 8), (100, 120, 16), (64, 64, 4)]
    X32s, ys = [], []
    for k, (n1, n2, d) in enumerate(shapes):
        X32, y = datagen.svm_clusters(n1, n2, d, seed=40 + k)
        X32s.append(X32)
        ys.append(y)
    offs = np.zeros(len(shapes), dtype=np.int64)
    pos = 1
    for k, x in enumerate(X32s):
        offs[k] = pos
        pos += x.size + 4  # every start stays one element past a 4-element boundary
    host = np.zeros(pos, dtype=np.float32)
    for k, x in enumerate(X32s):
        host[offs[k]:offs[k] + x.size] = x.reshape(-1)
    pts_mis = torch.from_numpy(host).cuda()
    n = np.array([x.shape[0] for x in X32s], dtype=np.int64)
    d = np.array([x.shape[1] for x in X32s], dtype=np.int32)
    lab, loffs = api.pack_labels(ys)
    pts_al, offs_al, _, _ = api.pack_instances(X32s)
    a = torch.tensor([1.0, 1.5, 0.7], dtype=torch.float64, device="cuda")
    e = torch.tensor([0.02, 0.02, 0.05], dtype=torch.float64, device="cuda")
    res = []
    for p, o in ((pts_mis, offs), (pts_al, offs_al)):
        b = api.SvmBatch(p, o, n, d, lab, loffs, tile_rows=128)
        out = api.new_steps(len(shapes))
        for _ in range(15):
            b.step(a, e, out=out)
        torch.cuda.synchronize()
        res.append((api.decode_steps(out), b.read()[0]))
    for k in range(len(shapes)):
        tol = RTOL * float(np.max(np.linalg.norm(X32s[k], axis=1)))
        for key in ("objective", "oracle_value", "upper_bound"):
            assert abs(res[0][0][key][k] - res[1][0][key][k]) <= 2 * tol, (k, key)
        assert np.linalg.norm(res[0][1][k] - res[1][1][k]) <= 2 * RTOL


def test_svm_batch_repeated_launches_reset_their_counters():
    shapes = [(2500, 2500, 32), (350, 350, 8), (2, 1, 3)]
    pts, offs, n, d, lab, loffs, _, _ = _instances(shapes, 7)
    batch = api.SvmBatch(pts, offs, n, d, lab, loffs, tile_rows=256)
    _, _, D = batch.read()
    a = torch.tensor(0.5 * D, dtype=torch.float64, device="cuda")
    e = torch.tensor(0.5 / (2.0 * D), dtype=torch.float64, device="cuda")
    out = api.new_steps(3)
    for _ in range(50):
        batch.step(a, e, out=out)
    torch.cuda.synchronize()
    r = api.decode_steps(out)
    assert np.all(r["status"] == 0)
    assert np.all((r["t"] == 50) | (r["stopped"] == 1))


def _search_batch():
    shapes = [(5, 5, 2), (40, 30, 3), (300, 300, 16), (1000, 800, 8), (2000, 2000, 4), (150, 200, 12)]
    return shapes, _instances(shapes, 900)


@pytest.mark.parametrize("mode", ["certified", "practical"])
def test_svm_batch_search_brackets_exact_distance(mode):
    shapes, (pts, offs, n, d, lab, loffs, Xs, ys) = _search_batch()
    batch = api.SvmBatch(pts, offs, n, d, lab, loffs, tile_rows=512)
    eps = 1e-2
    reps, ws, launches = batch.solve(eps=eps, mode=mode, max_iters=60_000, poll_every=64, launches_per_poll=64)
    assert launches > 0
    for k, (X, y) in enumerate(zip(Xs, ys)):
        P, Q = X[y > 0], X[y < 0]
        opt = exact.pd_bruteforce(P, Q)[0] if len(P) + len(Q) <= 12 else exact.pd_mdm(P, Q, tol=1e-12)[0]
        r = reps[k]
        assert r["status"] in (0, 5), (k, r["status"])
        # certificates hold whatever the mode: an actual direction's margin and a Claim 8 value
        assert r["lower_bound"] <= opt * (1 + FP) and r["upper_bound"] >= opt * (1 - FP), (k, r, opt)
        assert math.isclose(r["D"], osvm.svm_D(X), rel_tol=1e-12)
        w = ws[k].astype(np.float64)
        if r["lower_bound"] > 0:
            assert math.isclose(exact.svm_margin_of(P, Q, w), r["value"], rel_tol=1e-4), k
        if mode == "certified":
            assert r["status"] == 0, (k, r)
            assert r["upper_bound"] <= (1 + eps) * r["lower_bound"], (k, r)


def test_svm_batch_certified_search_agrees_with_single_instance_solve():
    shapes, (pts, offs, n, d, lab, loffs, Xs, ys) = _search_batch()
    batch = api.SvmBatch(pts, offs, n, d, lab, loffs, tile_rows=512)
    eps = 1e-2
    reps, _, _ = batch.solve(eps=eps, mode="certified", max_iters=60_000, poll_every=64)
    for k, (X, y) in enumerate(zip(Xs, ys)):
        _, one = api.svm_solve(torch.from_numpy(X.astype(np.float32)).cuda(), torch.from_numpy(y).cuda(), eps=eps,
                               mode="certified", max_iters=60_000, poll_every=64)
        r = reps[k]
        assert one["status"] == r["status"] == 0, (k, one, r)
        # each certified interval contains the other's margin
        assert r["lower_bound"] <= one["upper_bound"] * (1 + FP) and one["lower_bound"] <= r["upper_bound"] * (1 + FP)
