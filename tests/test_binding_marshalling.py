"""Every entry point of the Python binding, run on the CPU against a stand-in
for libpdscp.so that checks each call's arity and argument kinds against the
ctypes signatures of the C ABI (no kernel runs): catches marshalling mistakes
(a missing or extra argument, a tensor where a size goes) and checks that the
binding's own argument validation rejects buffers that are too small or of
the wrong type before anything reaches the library."""

import ctypes

import numpy as np
import pytest
import torch

from paper_2405_09157_gb300 import _ffi, api

SIZE = 1 << 16  # every size query of the stand-in answers this many bytes


class _Arg:
    CArgObject = type(ctypes.byref(ctypes.c_int()))


def _kind_ok(argtype, v):
    if argtype is _ffi.c_vp:  # a plain int here is a host array's address (numpy .ctypes.data), never small
        return v is None or isinstance(v, (ctypes.c_void_p, _Arg.CArgObject)) or (
            isinstance(v, int) and v >= 1 << 16)
    if argtype in (_ffi.c_i32, _ffi.c_i64, _ffi.c_sz):
        return isinstance(v, (int, np.integer)) and not isinstance(v, bool)
    if argtype is _ffi.c_dbl:
        return isinstance(v, (int, float, np.floating)) and not isinstance(v, bool)
    return isinstance(v, _Arg.CArgObject)  # POINTER(...) outputs and structs by reference


class FakeLib:
    """Checks calls against _ffi.SIGNATURES and fills size outputs."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        if name not in _ffi.SIGNATURES:
            raise AttributeError(name)
        _, argtypes = _ffi.SIGNATURES[name]

        def call(*args):
            assert len(args) == len(argtypes), (name, len(args), len(argtypes))
            for i, (at, v) in enumerate(zip(argtypes, args)):
                assert _kind_ok(at, v), (name, i, at, type(v))
                if isinstance(v, _Arg.CArgObject) and isinstance(v._obj, (ctypes.c_size_t, ctypes.c_int64,
                                                                           ctypes.c_int32)):
                    v._obj.value = SIZE if "size" in name or "stride" in name else 1
                if isinstance(v, _Arg.CArgObject) and isinstance(v._obj, ctypes.c_float):
                    v._obj.value = 1.0
            self.calls.append(name)
            return b"" if name == "pdscp_last_error" else 0
        return call


@pytest.fixture
def fake(monkeypatch):
    lib = FakeLib()
    monkeypatch.setattr(_ffi, "_lib", lib)
    monkeypatch.setattr(api, "load", lambda: lib)
    monkeypatch.setattr(api, "_stream", lambda stream=None: None)
    monkeypatch.setattr(api, "_vp", lambda t: None if t is None else ctypes.c_void_p(t.data_ptr()))

    def points(pts):
        assert pts.dim() == 2 and pts.is_contiguous()
        return pts.shape[0], pts.shape[1], api.dtype_code(pts)
    monkeypatch.setattr(api, "_points", points)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    api.state_size.cache_clear()
    yield lib
    api.state_size.cache_clear()


def test_every_entry_point_marshals(fake):
    cpu = torch.device("cpu")
    n, d = 64, 8
    pts = torch.randn(n, d)
    radii = torch.zeros(n)
    labels = torch.where(torch.arange(n) < n // 2, 1, -1).to(torch.int8)
    api.bounds(_ffi.SES, pts, radii)
    for problem, kw in ((_ffi.SES, {"radii": radii}), (_ffi.SVM, {"labels": labels})):
        m = api.MWU(problem, pts, **kw)
        rec = api.new_steps(4, cpu)
        m.step(1.0, 0.1, out=rec[0], D=2.0)
        m.run(1.0, 0.1, 4, out=rec, D=2.0)
        m.set(3, torch.zeros(d + (2 if problem == _ffi.SVM else 0), dtype=torch.float64), D=2.0)
        m.read()
        api.mwu_step_noalloc(problem, pts, 1.0, 0.1, m.state, out=rec[1], D=2.0, **kw)
        api.mwu_backward(pts, 1.0, 0.1, 5, problem=problem, D=2.0, out=rec[2], **kw)
    api.decode_steps(api.new_steps(2, cpu))
    api.ses_solve(pts, radii, mode="certified")
    api.svm_solve(pts, labels, mode="certified")
    api.svm_solve(pts, labels, mode="coreset")
    api.polytope_distance(np.ones((3, d)), -np.ones((2, d)))
    f = api.ses_unrolled_radius(pts.clone().requires_grad_(True), 1.0, 0.1, 3)
    f.backward()
    g = api.svm_unrolled_margin(pts.clone().requires_grad_(True), labels, 1.0, 0.1, 3, 2.0)
    g.backward()
    mm = api.MultiMWU(pts, 4, radii=radii)
    mm.step(torch.ones(4, dtype=torch.float64), torch.ones(4, dtype=torch.float64), out=api.new_steps(4, cpu))
    mm.read(1)
    sh = api.ShardedMWU(_ffi.SES, pts, pts[0].contiguous(), 0, 1, radii=radii, first_radius=radii[0:1])
    sh.step(1.0, 0.1, out=api.new_steps(1, cpu))
    sh.read()
    arrays = [np.random.default_rng(0).standard_normal((nn, dd)).astype(np.float32) for nn, dd in [(30, 4), (9, 3)]]
    for dt in (torch.float32, torch.bfloat16):
        bp, offs, nn, dd = api.pack_instances(arrays, device=cpu, dtype=dt)
        b = api.SesBatch(bp, offs, nn, dd, tile_rows=512)
        b.step(torch.ones(2, dtype=torch.float64), torch.ones(2, dtype=torch.float64), out=api.new_steps(2, cpu))
        b.read()
        b.autotune()
        b.set_launch(2, 1)
        b.solve(mode="certified")
        lab, loffs = api.pack_labels([np.where(np.arange(nn_) % 2 == 0, 1, -1) for nn_ in nn], device=cpu)
        sb = api.SvmBatch(bp, offs, nn, dd, lab, loffs, tile_rows=512)
        sb.step(torch.ones(2, dtype=torch.float64), torch.ones(2, dtype=torch.float64), out=api.new_steps(2, cpu))
        sb.read()
        sb.solve(mode="certified")
    # every entry point the binding reaches was called with its declared arity
    assert {"mwu_step", "mwu_run", "mwu_backward", "ses_solve", "svm_solve", "ses_multi_step", "mwu_shard_partial",
            "mwu_shard_finish", "ses_batch_init", "ses_batch_step", "ses_batch_autotune", "ses_batch_solve_init",
            "ses_batch_solve_run", "ses_batch_solve_read", "mwu_step_noalloc", "mwu_state_set", "ses_batch_set_launch",
            "pdscp_polytope_distance", "svm_batch_init", "svm_batch_step", "svm_batch_read", "svm_batch_solve_init",
            "svm_batch_solve_run", "svm_batch_solve_read"} <= set(fake.calls)


def test_binding_rejects_bad_buffers(fake):
    n, d = 64, 8
    pts = torch.randn(n, d)
    m = api.MWU(_ffi.SES, pts)
    small_state = torch.zeros(16, dtype=torch.uint8)
    with pytest.raises(ValueError, match="state"):
        api.mwu_step(_ffi.SES, pts, 1.0, 0.1, small_state, m.ws)
    with pytest.raises(ValueError, match="radii"):
        api.mwu_step(_ffi.SES, pts, 1.0, 0.1, m.state, m.ws, radii=torch.zeros(n, dtype=torch.float64))
    with pytest.raises(ValueError, match="radii"):
        api.mwu_step(_ffi.SES, pts, 1.0, 0.1, m.state, m.ws, radii=torch.zeros(n - 1))
    with pytest.raises(ValueError, match="labels"):
        api.mwu_step(_ffi.SVM, pts, 1.0, 0.1, api.new_state(_ffi.SVM, d, "cpu"), m.ws,
                     labels=torch.ones(n, dtype=torch.int64))
    with pytest.raises(ValueError, match="step records"):
        api.mwu_run(_ffi.SES, pts, 1.0, 0.1, 3, m.state, m.ws, out=api.new_steps(2, "cpu"))
    with pytest.raises(ValueError, match="step records"):
        api.mwu_step(_ffi.SES, pts, 1.0, 0.1, m.state, m.ws, out=torch.zeros(71, dtype=torch.uint8))
    with pytest.raises(ValueError, match="labels"):
        api.svm_solve(pts, torch.ones(n, dtype=torch.float32))
    with pytest.raises(ValueError, match="mean"):
        api.state_set(_ffi.SVM, pts, 1, torch.zeros(d), api.new_state(_ffi.SVM, d, "cpu"), m.ws,
                      labels=torch.ones(n, dtype=torch.int8))
    mm = api.MultiMWU(pts, 2)
    with pytest.raises(ValueError, match="alpha"):
        mm.step(torch.ones(1, dtype=torch.float64), torch.ones(2, dtype=torch.float64))
