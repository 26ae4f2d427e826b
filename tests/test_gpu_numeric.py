"""The device's numeric guard: a point with a NaN or infinite coordinate makes
the trace normaliser (the sum of the exponentials, Sec. 2.3) or the ORACLE
value non-finite; the finishing warp then records PDSCP_ERR_NUMERIC in the
step record and the state, stops the alpha-FTP without advancing its mean,
and the solves return that status to the host. The inputs are made on the
host; nothing here reads out of bounds or waits."""

import numpy as np
import pytest
import torch

from oracle import ses as oses, svm as osvm
from paper_2405_09157_gb300 import _ffi, api, datagen

pytestmark = pytest.mark.gpu
NUMERIC = 6


def _hdr(state):
    b = state.cpu().numpy().tobytes()
    t = np.frombuffer(b[:8], dtype="<i8")[0]
    stopped, outcome, status = np.frombuffer(b[8:20], dtype="<i4")
    return int(t), int(stopped), int(outcome), int(status)


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
@pytest.mark.parametrize("row", [1, 777])
def test_ses_step_flags_non_finite_points(bad, row):
    V32 = datagen.ses_gaussian(1000, 8, seed=31)
    D = oses.ses_D(V32.astype(np.float64))
    rho = oses.ses_width(D)
    pts = torch.from_numpy(V32).cuda()
    m = api.MWU(_ffi.SES, pts)
    out = api.new_steps(3)
    m.step(0.8 * D, 0.5 / rho, out=out[0])          # a clean step first
    mean0, _ = m.read()
    pts[row, 3] = float(bad)
    m.step(0.8 * D, 0.5 / rho, out=out[1])
    m.step(0.8 * D, 0.5 / rho, out=out[2])          # after the stop: a no-op
    torch.cuda.synchronize()
    r = api.decode_steps(out)
    assert r["status"][0] == 0 and r["t"][0] == 1
    assert r["status"][1] == NUMERIC and r["stopped"][1] == 1 and r["t"][1] == 1
    assert r["t"][2] == 0  # no record after the stop
    t, stopped, _, status = _hdr(m.state)
    assert (t, stopped, status) == (1, 1, NUMERIC)
    mean1, _ = m.read()
    assert torch.equal(mean0, mean1)  # the mean was not advanced


def test_svm_step_flags_non_finite_points():
    X32, y = datagen.svm_clusters(600, 500, 16, seed=32)
    D = osvm.svm_D(X32.astype(np.float64))
    X = torch.from_numpy(X32).cuda()
    m = api.MWU(_ffi.SVM, X, labels=torch.from_numpy(y).cuda())
    out = api.new_steps(2)
    m.step(0.3 * D, 0.5 / (2 * D), out=out[0], D=D)
    X[900, 5] = float("nan")
    m.step(0.3 * D, 0.5 / (2 * D), out=out[1], D=D)
    torch.cuda.synchronize()
    r = api.decode_steps(out)
    assert r["status"][0] == 0
    assert r["status"][1] == NUMERIC and r["stopped"][1] == 1
    assert _hdr(m.state)[3] == NUMERIC


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_solves_return_numeric_status(bad):
    V32 = datagen.ses_gaussian(2000, 4, seed=33)
    V32[1234, 2] = bad
    with pytest.raises(_ffi.PdscpError) as e:
        api.ses_solve(torch.from_numpy(V32).cuda(), eps=1e-2, mode="certified")
    assert e.value.status == NUMERIC
    X32, y = datagen.svm_clusters(600, 500, 8, seed=34)
    X32[17, 0] = bad
    with pytest.raises(_ffi.PdscpError) as e:
        api.svm_solve(torch.from_numpy(X32).cuda(), torch.from_numpy(y).cuda(), eps=1e-2, mode="certified")
    assert e.value.status == NUMERIC
