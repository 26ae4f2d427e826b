"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method: it only draws point sets.
Both the CUDA path's tests/benchmarks and the FP64 oracle receive the arrays
it returns. Every generator draws in float64 from numpy's PCG64 with the given
seed and returns float32 arrays (what the device stores); callers hand the
same float32 values, promoted to float64, to the oracle, so both sides see
bit-identical inputs.

The paper's experiments use "randomly generated" point sets (Sec. 5) without
naming a distribution; these recipes fix one for each workload:
  ses_uniform      n points i.i.d. U[0,1]^d
  ses_gaussian     n points i.i.d. N(0, I_d)
  svm_clusters     two Gaussian clusters N(+-mu, I_d), ||mu|| = mu_norm along a
                   seeded random unit direction; points within `band` of the
                   Bayes hyperplane mu^T x = 0 (y mu_hat^T x < band) are
                   dropped so the classes are linearly separable; labels +1
                   for the first n1 rows, -1 for the next n2 (P then Q).
  batched_ses      many SES instances of uneven n and d (log-uniform n,
                   d from a list, per-instance scale U[0.1, 10]).
"""

import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def ses_uniform(n, d, seed=0):
    """n points i.i.d. uniform in [0,1]^d, float32 (n, d)."""
    return _rng(seed).random((n, d)).astype(np.float32)


def ses_gaussian(n, d, seed=0, scale=1.0):
    """n points i.i.d. N(0, scale^2 I_d), float32 (n, d)."""
    return (scale * _rng(seed).standard_normal((n, d))).astype(np.float32)


def svm_clusters(n1, n2, d, mu_norm=3.0, band=0.1, seed=0):
    """Two separable Gaussian clusters. Returns (X float32 (n1+n2, d), y int8)."""
    rng = _rng(seed)
    mu_hat = rng.standard_normal(d)
    mu_hat /= np.linalg.norm(mu_hat)
    mu = mu_norm * mu_hat
    out = []
    for sign, cnt in ((1.0, n1), (-1.0, n2)):
        kept = []
        have = 0
        while have < cnt:
            batch = max(1024, int(1.2 * (cnt - have)) + 16)
            Z = rng.standard_normal((batch, d)) + sign * mu
            keep = Z[sign * (Z @ mu_hat) >= band]
            kept.append(keep)
            have += keep.shape[0]
        out.append(np.concatenate(kept, axis=0)[:cnt])
    X = np.concatenate(out, axis=0).astype(np.float32)
    y = np.concatenate([np.ones(n1, dtype=np.int8), -np.ones(n2, dtype=np.int8)])
    return X, y


def batched_ses_sizes(num, n_min=100, n_max=100_000, dims=(2, 3, 8, 16, 32, 64), seed=0):
    """Sizes of the batched workload: (n, d, scale) arrays of `num` instances,
    n log-uniform in [n_min, n_max], d uniform over `dims`, scale U[0.1, 10]."""
    rng = _rng(seed)
    n = np.round(np.exp(rng.uniform(np.log(n_min), np.log(n_max), num))).astype(np.int64)
    d = np.asarray(dims, dtype=np.int32)[rng.integers(len(dims), size=num)]
    scale = rng.uniform(0.1, 10.0, num)
    return n, d, scale


def batched_ses(num, n_min=100, n_max=100_000, dims=(2, 3, 8, 16, 32, 64), seed=0):
    """List of `num` SES instances (float32 (n_i, d_i) arrays): n_i log-uniform
    in [n_min, n_max], d_i uniform over `dims`, points N(0, I) times a
    per-instance scale drawn U[0.1, 10]."""
    rng = _rng(seed)
    out = []
    for _ in range(num):
        n = int(round(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))))
        d = int(dims[rng.integers(len(dims))])
        s = rng.uniform(0.1, 10.0)
        out.append((s * rng.standard_normal((n, d))).astype(np.float32))
    return out
