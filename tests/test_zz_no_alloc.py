"""mwu_step_noalloc: the step for callers that cannot allocate device memory
(the scratch is the library's built-in array) must give the same results as
mwu_step with a caller workspace, on consecutive calls. This file is named so
that pytest collects it last."""

import ctypes

import numpy as np
import pytest
import torch

from paper_2405_09157_gb300 import _ffi, api, datagen

pytestmark = pytest.mark.gpu
RTOL = 1e-5  # the tolerance of the other GPU parity tests, relative to the problem scale D


def _vp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _run_pair(problem, pts, alpha, eor, D=0.0, labels=None, steps=2):
    lib = _ffi.load()
    n, d = pts.shape
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ref = api.MWU(problem, pts, labels=labels)          # workspace path
    state = api.new_state(problem, d)                   # built-in scratch path
    ws_init = api.workspace(problem, n, d)              # only to initialise the state
    api.state_init(problem, pts, state, ws_init)
    out_ref, out_na = api.new_steps(steps), api.new_steps(steps)
    for k in range(steps):
        ref.step(alpha, eor, out=out_ref[k], D=D)
        st = lib.mwu_step_noalloc(problem, _vp(pts), api.dtype_code(pts), None, _vp(labels), n, d, alpha, eor,
                                  D, 0, _vp(state), stream, _vp(out_na[k]))
        assert st == 0, lib.pdscp_last_error()
    torch.cuda.synchronize()
    a, b = api.decode_steps(out_ref), api.decode_steps(out_na)
    mean_ref, _ = ref.read()
    mean_na, _ = api.state_read(problem, d, state)
    return a, b, mean_ref.cpu().numpy(), mean_na.cpu().numpy()


def test_noalloc_step_matches_workspace_step_ses_and_svm():
    V = torch.from_numpy(datagen.ses_gaussian(4099, 32, seed=21)).cuda()
    D = float(api.bounds(_ffi.SES, V).item())
    a, b, ma, mb = _run_pair(_ffi.SES, V, 0.8 * D, 0.5 / (3 * D / np.sqrt(2)))
    for key in ("oracle_value", "objective", "lower_bound", "upper_bound"):
        assert np.all(np.abs(a[key] - b[key]) <= RTOL * D), key
    assert np.array_equal(a["t"], b["t"]) and np.all(b["status"] == 0) and b["t"][-1] == 2
    assert np.linalg.norm(ma - mb) <= RTOL * D

    X, y = datagen.svm_clusters(1500, 1200, 64, seed=22)
    X, y = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    D = float(api.bounds(_ffi.SVM, X).item())
    a, b, ma, mb = _run_pair(_ffi.SVM, X, 0.3 * D, 0.5 / (2 * D), D=D, labels=y)
    for key in ("oracle_value", "objective", "upper_bound"):
        assert np.all(np.abs(a[key] - b[key]) <= RTOL * D), key
    assert np.all(b["status"] == 0) and b["t"][-1] == 2
    assert np.linalg.norm(ma - mb) <= RTOL * D


def test_noalloc_rejects_problems_beyond_its_scratch():
    lib = _ffi.load()
    pts = torch.zeros((16, 1024), dtype=torch.float32, device="cuda")
    state = api.new_state(_ffi.SVM, 1024)
    lab = torch.ones(16, dtype=torch.int8, device="cuda")
    st = lib.mwu_step_noalloc(_ffi.SVM, _vp(pts), _ffi.F32, None, _vp(lab), 16, 1024, 1.0, 0.1, 1.0, 0,
                              _vp(state), None, None)
    assert st == 8 and b"built-in scratch" in lib.pdscp_last_error()
