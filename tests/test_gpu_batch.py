"""Batched SES (one launch per iteration for many instances) against the
FP64 oracle, instance by instance (tolerance as in test_gpu_parity.py)."""

import numpy as np
import pytest
import torch

from oracle import ses as oses
from paper_2405_09157_gb300 import _ffi, api, datagen

pytestmark = pytest.mark.gpu
RTOL = 1e-5

SHAPES = [(2, 3), (3, 2), (50, 8), (777, 16), (3000, 32), (10001, 64), (1234, 5), (500, 3), (4099, 2),
          (8200, 33), (2049, 4), (1500, 12), (64, 64), (300, 1)]


def test_batch_trajectories_match_oracle_per_instance():
    arrays = [datagen.ses_gaussian(n, d, seed=100 + k, scale=1.0 + k) for k, (n, d) in enumerate(SHAPES)]
    pts, offs, n, d = api.pack_instances(arrays)
    batch = api.SesBatch(pts, offs, n, d, tile_rows=512)
    V = [a.astype(np.float64) for a in arrays]
    D = np.array([oses.ses_D(v) for v in V])
    rho = np.array([oses.ses_width(x) for x in D])
    alpha = 0.8 * D
    eta, T = 0.5, 20
    a_dev = torch.tensor(alpha, dtype=torch.float64, device="cuda")
    e_dev = torch.tensor(eta / rho, dtype=torch.float64, device="cuda")
    outs = [api.new_steps(len(SHAPES)) for _ in range(T)]
    for t in range(T):
        batch.step(a_dev, e_dev, out=outs[t])
    torch.cuda.synchronize()
    recs = [api.decode_steps(o) for o in outs]
    means, _ = batch.read()
    for k in range(len(SHAPES)):
        ubar = V[k][0].copy()
        tol = RTOL * D[k]
        for t in range(T):
            o = oses.ses_step(V[k], None, ubar, t, alpha[k], eta, rho[k])
            r = recs[t][k]
            assert r["status"] == 0, (k, t)
            for key in ("objective", "oracle_value", "lower_bound"):
                assert abs(r[key] - o[key]) <= tol, (k, SHAPES[k], t, key, r[key], o[key])
            if abs(o["oracle_value"]) > tol:
                assert bool(r["failed"]) == o["failed"], (k, t)
            if o["failed"]:
                break
            ubar = o["ubar_next"]
        assert np.linalg.norm(means[k].astype(np.float64) - ubar) <= tol, (k, SHAPES[k])


def test_batch_repeated_launches_reset_their_counters():
    arrays = [datagen.ses_gaussian(n, d, seed=7 + n) for n, d in [(5000, 32), (700, 8), (3, 3)]]
    pts, offs, n, d = api.pack_instances(arrays)
    batch = api.SesBatch(pts, offs, n, d, tile_rows=256)
    a = torch.tensor([5.0, 3.0, 2.0], dtype=torch.float64, device="cuda")
    e = torch.tensor([0.01, 0.01, 0.01], dtype=torch.float64, device="cuda")
    out = api.new_steps(3)
    for _ in range(50):
        batch.step(a, e, out=out)
    torch.cuda.synchronize()
    r = api.decode_steps(out)
    assert np.all(r["status"] == 0)
    assert np.all((r["t"] == 50) | (r["stopped"] == 1))
