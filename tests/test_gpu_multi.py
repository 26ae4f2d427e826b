"""Multi-candidate SES iteration (ses_multi_step) against the FP64 oracle:
every candidate's trajectory is that of an independent alpha-FTP with its own
alpha (tolerance as in test_gpu_parity.py), including candidates whose ORACLE
separates (they stop and keep their state while the others continue)."""

import numpy as np
import pytest
import torch

from oracle import ses as oses
from paper_2405_09157_gb300 import api, datagen

pytestmark = pytest.mark.gpu
RTOL = 1e-5


@pytest.mark.parametrize("n,d,k,radii", [(3001, 32, 2, False), (2000, 5, 4, False), (1500, 64, 8, False),
                                         (999, 2, 8, True), (4000, 8, 4, True), (5003, 16, 1, False),
                                         (2, 3, 2, False)])
def test_candidates_follow_their_own_oracle_trajectories(n, d, k, radii):
    V32 = datagen.ses_gaussian(n, d, seed=n + k)
    g32 = (0.1 * np.random.default_rng(n).random(n)).astype(np.float32) if radii else None
    V = V32.astype(np.float64)
    g = None if g32 is None else g32.astype(np.float64)
    D = oses.ses_D(V, g)
    rho = oses.ses_width(D)
    eta, T = 1.0, 20
    alphas = np.array([(0.45 + 0.1 * j) * D for j in range(k)])
    pts = torch.from_numpy(V32).cuda()
    rad = None if g32 is None else torch.from_numpy(g32).cuda()
    m = api.MultiMWU(pts, k, radii=rad)
    a_dev = torch.tensor(alphas, dtype=torch.float64, device="cuda")
    e_dev = torch.full((k,), eta / rho, dtype=torch.float64, device="cuda")
    outs = [api.new_steps(k) for _ in range(T)]
    for t in range(T):
        m.step(a_dev, e_dev, out=outs[t])
    torch.cuda.synchronize()
    recs = [api.decode_steps(o) for o in outs]
    for j in range(k):
        # Every step carries FP32 rounding of about 6e-8 D, which the
        # trajectory itself may amplify (measured here on the oracle by moving
        # ubar^2 by 1e-7 D); the bound is the larger of the usual tolerance and
        # T * 6e-8 D * amplification (equal to the usual one for all but the
        # ill-conditioned candidates).
        amp = _amplification(V, g, alphas[j], eta, rho, T)
        tol = max(RTOL * D, T * 6e-8 * amp * D)
        ubar, stopped_at = V[0].copy(), None
        for t in range(T):
            o = oses.ses_step(V, g, ubar, t, alphas[j], eta, rho)
            r = recs[t][j]
            assert r["status"] == 0
            for key in ("objective", "oracle_value", "lower_bound"):
                assert abs(r[key] - o[key]) <= tol, (j, t, key, r[key], o[key], amp)
            if abs(o["oracle_value"]) > tol:
                assert bool(r["failed"]) == o["failed"], (j, t)
            if o["failed"]:
                stopped_at = t
                break
            ubar = o["ubar_next"]
        if stopped_at is not None:
            assert all(recs[t][j]["t"] == 0 for t in range(stopped_at + 1, T))  # no record after the stop
        mean, _ = m.read(j)
        err = np.linalg.norm(mean.cpu().numpy().astype(np.float64) - ubar)
        assert err <= tol, (j, err / D, amp)


def _amplification(V, g, alpha, eta, rho, T):
    def run(p):
        ub = V[0].copy()
        for t in range(T):
            o = oses.ses_step(V, g, ub, t, alpha, eta, rho)
            if o["failed"]:
                break
            ub = o["ubar_next"] + (p if t == 1 else 0.0)
        return ub
    D = oses.ses_D(V, g)
    p = np.random.default_rng(1).standard_normal(V.shape[1])
    p *= 1e-7 * D / np.linalg.norm(p)
    return max(1.0, np.linalg.norm(run(p) - run(0.0)) / (1e-7 * D))


def test_candidates_match_single_candidate_steps():
    V32 = datagen.ses_gaussian(100_000, 32, seed=3)
    V = V32.astype(np.float64)
    D = oses.ses_D(V)
    rho = oses.ses_width(D)
    pts = torch.from_numpy(V32).cuda()
    k, T = 4, 30
    alphas = [0.6 * D, 0.7 * D, 0.8 * D, 1.0 * D]
    m = api.MultiMWU(pts, k)
    out_m = api.new_steps(k)
    singles = [api.MWU(api.SES, pts) for _ in range(k)]
    out_s = api.new_steps(k)
    a_dev = torch.tensor(alphas, dtype=torch.float64, device="cuda")
    e_dev = torch.full((k,), 0.5 / rho, dtype=torch.float64, device="cuda")
    for _ in range(T):
        m.step(a_dev, e_dev, out=out_m)
        for j in range(k):
            singles[j].step(alphas[j], 0.5 / rho, out=out_s[j])
    torch.cuda.synchronize()
    rm, rs = api.decode_steps(out_m), api.decode_steps(out_s)
    for j in range(k):
        assert rm[j]["t"] == rs[j]["t"]
        for key in ("objective", "oracle_value", "lower_bound"):
            assert abs(rm[j][key] - rs[j][key]) <= 2 * RTOL * D, (j, key)


def test_full_size_k8_against_oracle():
    """The benchmarked multi-candidate configuration (n = 1e6, d = 32, k = 8):
    three iterations of every candidate against the FP64 oracle."""
    V32 = datagen.ses_gaussian(1_000_000, 32, seed=0)
    V = V32.astype(np.float64)
    D = oses.ses_D(V)
    rho = oses.ses_width(D)
    k, T, eta = 8, 3, 0.5
    alphas = np.array([(0.7 + 0.05 * j) * D for j in range(k)])
    m = api.MultiMWU(torch.from_numpy(V32).cuda(), k)
    a_dev = torch.tensor(alphas, dtype=torch.float64, device="cuda")
    e_dev = torch.full((k,), eta / rho, dtype=torch.float64, device="cuda")
    outs = [api.new_steps(k) for _ in range(T)]
    for t in range(T):
        m.step(a_dev, e_dev, out=outs[t])
    torch.cuda.synchronize()
    recs = [api.decode_steps(o) for o in outs]
    tol = RTOL * D
    for j in range(k):
        ubar = V[0].copy()
        for t in range(T):
            o = oses.ses_step(V, None, ubar, t, alphas[j], eta, rho)
            for key in ("objective", "oracle_value", "lower_bound"):
                assert abs(recs[t][j][key] - o[key]) <= tol, (j, t, key)
            ubar = o["ubar_next"]
