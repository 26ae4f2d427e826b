"""The reverse sweep at the differentiable workload's size (n = 100,000 points
in d = 64, N(0, I), alpha = D) against central finite differences of the FP64
oracle's forward: for a direction U (unit Frobenius norm over all points) the
directional derivative <dL/dV, U> from mwu_backward must equal
(L(V + hU) - L(V - hU)) / 2h with h = 1e-3, L = f(ubar^T) the radius after T
alpha-FTP iterations at fixed alpha and eta/rho (Sec. 3, Eq. implement;
Sec. 5), within 1e-3 relative.

T = 20 and T = 50: the oracle's forward (materialised weights of every cone,
FP64) costs about 0.4 s per iteration at this size, so T = 2000 is out of
reach for it; on this map finite differences at h = 1e-3 and h = 1e-4 agree
with reverse-mode differentiation to ~1e-8 up to T = 100 (n = 1e4, measured),
so the map is smooth at these steps. The directions: two seeded Gaussian
directions over all points, one on the row attaining the radius (where the
gradient is largest) and the normalised GPU gradient itself (which checks its
length). The forwards run in a pool of spawned processes."""

import multiprocessing as mp

import numpy as np
import pytest
import torch

from oracle import ses as oses
from paper_2405_09157_gb300 import api, datagen

pytestmark = pytest.mark.gpu
N, D_DIM, H, FD_RTOL = 100_000, 64, 1e-3, 1e-3


def _radius(V, alpha, eta, rho, T):
    res = oses.ses_ftp(V, None, alpha, eta, rho, T, mode=oses.MODE_FIXED)
    return oses.ses_objective(V, np.zeros(V.shape[0]), res["ubar"])


@pytest.mark.parametrize("T", [20, 50])
def test_backward_matches_central_differences_at_full_size(T):
    V32 = datagen.ses_gaussian(N, D_DIM, 0)
    V = V32.astype(np.float64)
    D = oses.ses_D(V)
    rho = oses.ses_width(D)
    alpha, eta = D, 0.5
    grad, _ = api.mwu_backward(torch.from_numpy(V32).cuda(), alpha, eta / rho, T)
    g = grad.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(g))
    rng = np.random.default_rng(T)
    dirs = [rng.standard_normal(V.shape) for _ in range(2)]
    row = np.zeros_like(V)
    imax = int(np.argmax(np.abs(g).sum(axis=1)))
    row[imax] = rng.standard_normal(D_DIM)
    dirs += [row, g.copy()]
    dirs = [u / np.linalg.norm(u) for u in dirs]
    jobs = []
    for u in dirs:
        jobs += [(V + H * u, alpha, eta, rho, T), (V - H * u, alpha, eta, rho, T)]
    with mp.get_context("spawn").Pool(min(len(jobs), 8)) as pool:
        vals = pool.starmap(_radius, jobs)
    for k, u in enumerate(dirs):
        fd = (vals[2 * k] - vals[2 * k + 1]) / (2 * H)
        ad = float(np.sum(g * u))
        assert abs(fd - ad) <= FD_RTOL * abs(fd), (T, k, fd, ad)
