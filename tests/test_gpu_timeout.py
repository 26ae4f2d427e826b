"""The staged pass kernels wait for the bulk copies (cp.async.bulk) that fill
their shared-memory rings on mbarriers, with a bounded number of tries. A
wait that gives up records the timeout; the kernel then waits for the copies
still in flight (so none lands after the CTA exits), completes the launch,
and the finishing CTA reports PDSCP_ERR_TIMEOUT in the step record and the
state, which stops the alpha-FTP. PDSCP_WAIT_LIMIT=0 makes every wait give
up at once; the copies themselves complete, so nothing faults or hangs, and
the same process then runs normal iterations."""

import numpy as np
import pytest
import torch

from oracle import ses as oses
from paper_2405_09157_gb300 import _ffi, api, datagen

pytestmark = pytest.mark.gpu
TIMEOUT = 3
RTOL = 1e-5


def _hdr_status(state):
    b = state.cpu().numpy().tobytes()
    t = int(np.frombuffer(b[:8], dtype="<i8")[0])
    stopped, outcome, status = (int(v) for v in np.frombuffer(b[8:20], dtype="<i4"))
    return t, stopped, status


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_wait_limit_reports_timeout_then_normal_steps(monkeypatch, dtype):
    V32 = datagen.ses_gaussian(200_000, 32, seed=51)  # rows of 16-byte chunks: the staged kernel
    V = torch.from_numpy(V32).to(dtype).to(torch.float32).numpy().astype(np.float64)
    D = oses.ses_D(V)
    rho = oses.ses_width(D)
    pts = torch.from_numpy(V32).cuda().to(dtype)
    out = api.new_steps(2)
    m = api.MWU(_ffi.SES, pts)
    monkeypatch.setenv("PDSCP_WAIT_LIMIT", "0")
    m.step(0.8 * D, 0.5 / rho, out=out[0])
    torch.cuda.synchronize()
    monkeypatch.delenv("PDSCP_WAIT_LIMIT")
    r = api.decode_steps(out[0])[0]
    assert r["status"] == TIMEOUT and r["stopped"] == 1 and r["t"] == 0
    assert _hdr_status(m.state) == (0, 1, TIMEOUT)
    # the context is healthy: a fresh alpha-FTP runs and matches the oracle
    m2 = api.MWU(_ffi.SES, pts)
    m2.step(0.8 * D, 0.5 / rho, out=out[1])
    torch.cuda.synchronize()
    r = api.decode_steps(out[1])[0]
    o = oses.ses_step(V, None, V[0].copy(), 0, 0.8 * D, 0.5, rho)
    assert r["status"] == 0 and r["t"] == 1
    for key in ("objective", "oracle_value", "lower_bound"):
        assert abs(r[key] - o[key]) <= RTOL * D, key


def test_svm_wait_limit_reports_timeout(monkeypatch):
    X32, y = datagen.svm_clusters(60_000, 60_000, 64, seed=52)
    D = float(np.max(np.linalg.norm(X32.astype(np.float64), axis=1)))
    X = torch.from_numpy(X32).cuda().to(torch.bfloat16)  # bfloat16 rows of 16-byte chunks: the staged kernel
    lab = torch.from_numpy(y).cuda()
    out = api.new_steps(2)
    m = api.MWU(_ffi.SVM, X, labels=lab)
    monkeypatch.setenv("PDSCP_WAIT_LIMIT", "0")
    m.step(0.3 * D, 0.5 / (2 * D), out=out[0], D=D)
    torch.cuda.synchronize()
    monkeypatch.delenv("PDSCP_WAIT_LIMIT")
    r = api.decode_steps(out[0])[0]
    assert r["status"] == TIMEOUT and r["stopped"] == 1
    assert _hdr_status(m.state)[1:] == (1, TIMEOUT)
    m2 = api.MWU(_ffi.SVM, X, labels=lab)
    m2.step(0.3 * D, 0.5 / (2 * D), out=out[1], D=D)
    torch.cuda.synchronize()
    assert api.decode_steps(out[1])[0]["status"] == 0
