"""mwu_step_noalloc: the step for callers that cannot allocate device memory
(code inside a host program that owns all GPU memory through its own pool, or
that must avoid the implicit synchronisation an allocation can cause) takes
its scratch from an array built into the library. It runs the same kernel with
the same fixed-order reductions as mwu_step with a caller workspace, so on
consecutive calls its records, running means and whole states must equal
mwu_step's bit for bit (a tolerance would let a scratch-layout fault that
shifts the results slightly pass). This file is named so that pytest collects
it last."""

import ctypes

import numpy as np
import pytest
import torch

from paper_2405_09157_gb300 import _ffi, api, datagen

pytestmark = pytest.mark.gpu


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
    assert torch.equal(ref.state.cpu(), state.cpu())  # header, FP64 and FP32 means, best point, dual vector
    return a, b, mean_ref.cpu().numpy(), mean_na.cpu().numpy()


def _assert_identical(a, b, ma, mb):
    for key in a.dtype.names:  # every field of every record, NaN-free by the status check
        assert np.array_equal(a[key], b[key]), key
    assert np.array_equal(ma, mb)


def test_noalloc_step_matches_workspace_step_ses_and_svm():
    V = torch.from_numpy(datagen.ses_gaussian(4099, 32, seed=21)).cuda()
    D = float(api.bounds(_ffi.SES, V).item())
    a, b, ma, mb = _run_pair(_ffi.SES, V, 0.8 * D, 0.5 / (3 * D / np.sqrt(2)))
    assert np.all(b["status"] == 0) and b["t"][-1] == 2
    _assert_identical(a, b, ma, mb)

    X, y = datagen.svm_clusters(1500, 1200, 64, seed=22)
    X, y = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    D = float(api.bounds(_ffi.SVM, X).item())
    a, b, ma, mb = _run_pair(_ffi.SVM, X, 0.3 * D, 0.5 / (2 * D), D=D, labels=y)
    assert np.all(b["status"] == 0) and b["t"][-1] == 2
    _assert_identical(a, b, ma, mb)


def test_noalloc_rejects_problems_beyond_its_scratch():
    lib = _ffi.load()
    pts = torch.zeros((16, 1024), dtype=torch.float32, device="cuda")
    state = api.new_state(_ffi.SVM, 1024)
    lab = torch.ones(16, dtype=torch.int8, device="cuda")
    st = lib.mwu_step_noalloc(_ffi.SVM, _vp(pts), _ffi.F32, None, _vp(lab), 16, 1024, 1.0, 0.1, 1.0, 0,
                              _vp(state), None, None)
    assert st == 8 and b"built-in scratch" in lib.pdscp_last_error()
