"""The C-ABI library loads and exports every entry point of include/pdscp.h,
and rejects bad arguments before touching a GPU (CPU-only tests)."""

import ctypes
import os
import re

import pytest

from paper_2405_09157_gb300 import _ffi, build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "pdscp.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(build.LIB):
        build.build()
    return _ffi.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:pdscp_status|int32_t|const char\*)\s+(\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported_and_bound(lib):
    names = declared_functions()
    assert len(names) >= 11
    for name in names:
        assert hasattr(lib, name), name
        assert name in _ffi.SIGNATURES, name
    assert set(_ffi.SIGNATURES) == set(names)


def test_version_and_sizes(lib):
    assert lib.pdscp_version() >= 100
    out = ctypes.c_size_t()
    assert lib.pdscp_state_size(_ffi.SES, 32, ctypes.byref(out)) == 0
    # header | FP64 mean | FP32 mean | FP32 best point | FP64 averaged dual vector
    assert out.value == 128 + 32 * 8 + 2 * 32 * 4 + 32 * 8
    assert lib.pdscp_workspace_size(_ffi.SVM, 1000, 128, ctypes.byref(out)) == 0 and out.value > 0
    assert lib.pdscp_workspace_size(_ffi.SES, 10, 0, ctypes.byref(out)) == 7


def test_argument_validation_without_gpu(lib):
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: every call below fails validation first
    st = lib.mwu_step(_ffi.SES, fake, _ffi.F32, None, None, 1, 4, 1.0, 0.1, 0.0, 0, fake, fake, 1 << 30, None, None)
    assert st == 1 and b"n >= 2" in lib.pdscp_last_error()
    st = lib.mwu_step(_ffi.SES, fake, _ffi.F32, None, None, 10, 0, 1.0, 0.1, 0.0, 0, fake, fake, 1 << 30, None, None)
    assert st == 7
    st = lib.mwu_step(_ffi.SES, fake, 9, None, None, 10, 4, 1.0, 0.1, 0.0, 0, fake, fake, 1 << 30, None, None)
    assert st == 1
    st = lib.mwu_step(_ffi.SES, fake, _ffi.F32, None, None, 10, 4, -1.0, 0.1, 0.0, 0, fake, fake, 1 << 30, None, None)
    assert st == 1 and b"alpha" in lib.pdscp_last_error()
    st = lib.mwu_step(_ffi.SVM, fake, _ffi.F32, None, None, 10, 4, 1.0, 0.1, 1.0, 0, fake, fake, 1 << 30, None, None)
    assert st == 1 and b"labels" in lib.pdscp_last_error()
    st = lib.mwu_step(_ffi.SVM, fake, _ffi.F32, None, fake, 10, 4, 1.0, 0.1, 0.0, 0, fake, fake, 1 << 30, None, None)
    assert st == 1 and b"D > 0" in lib.pdscp_last_error()
    st = lib.mwu_step(_ffi.SES, fake, _ffi.F32, None, None, 10, 4, 1.0, 0.1, 0.0, 0, None, fake, 1 << 30, None, None)
    assert st == 1
    st = lib.mwu_step(_ffi.SES, ctypes.c_void_p((1 << 20) + 2), _ffi.F32, None, None, 10, 4, 1.0, 0.1, 0.0, 0,
                      fake, fake, 1 << 30, None, None)
    assert st == 1 and b"aligned" in lib.pdscp_last_error()
    st = lib.mwu_step(_ffi.SES, fake, _ffi.F32, None, None, 10, 4, 1.0, 0.1, 0.0, 0, fake, fake, 16, None, None)
    assert st == 8
    # mwu_run: the same checks, plus k >= 0; k = 0 with valid arguments enqueues nothing
    st = lib.mwu_run(_ffi.SES, fake, _ffi.F32, None, None, 10, 4, 1.0, 0.1, 0.0, -1, fake, fake, 1 << 30, None, None)
    assert st == 1 and b"k =" in lib.pdscp_last_error()
    st = lib.mwu_run(_ffi.SVM, fake, _ffi.F32, None, None, 10, 4, 1.0, 0.1, 1.0, 5, fake, fake, 1 << 30, None, None)
    assert st == 1 and b"labels" in lib.pdscp_last_error()
    st = lib.mwu_run(_ffi.SES, fake, _ffi.F32, None, None, 10, 4, 1.0, 0.1, 0.0, 5, fake, fake, 16, None, None)
    assert st == 8
    assert lib.mwu_run(_ffi.SES, fake, _ffi.F32, None, None, 10, 4, 1.0, 0.1, 0.0, 0, fake, fake, 1 << 30, None,
                       None) == 0
    opts = _ffi.Options(0.0, 1e-4, 10, 0, 1000, 16, 10, 0.0)
    rep = _ffi.Report()
    st = lib.ses_solve(fake, _ffi.F32, None, 10, 4, ctypes.byref(opts), fake, 1 << 30, None, fake, ctypes.byref(rep))
    assert st == 1 and b"eps" in lib.pdscp_last_error()
    opts = _ffi.Options(1e-3, 1e-4, 10, 0, 1000, 0, 10, 0.0)
    st = lib.svm_solve(fake, _ffi.F32, fake, 10, 4, ctypes.byref(opts), fake, 1 << 30, None, fake, ctypes.byref(rep))
    assert st == 1 and b"poll_every" in lib.pdscp_last_error()
    # the certified mode is a known mode (the call then fails on the too-small workspace, before any launch);
    # an unknown one and an eta outside (0, 1] are rejected
    opts = _ffi.Options(1e-3, 0.0, 10, _ffi.MODE_CERTIFIED, 1000, 64, 10, 0.0)
    st = lib.ses_solve(fake, _ffi.F32, None, 10, 4, ctypes.byref(opts), fake, 16, None, fake, ctypes.byref(rep))
    assert st == 8
    opts = _ffi.Options(1e-3, 0.0, 10, 4, 1000, 64, 10, 0.0)
    st = lib.ses_solve(fake, _ffi.F32, None, 10, 4, ctypes.byref(opts), fake, 1 << 30, None, fake, ctypes.byref(rep))
    assert st == 1 and b"mode" in lib.pdscp_last_error()
    # the core-set mode needs the larger SVM workspace pdscp_workspace_size reports
    size = ctypes.c_size_t()
    assert lib.pdscp_workspace_size(_ffi.SVM, 10, 4, ctypes.byref(size)) == 0
    opts = _ffi.Options(1e-3, 0.0, 10, _ffi.MODE_CORESET, 1000, 64, 10, 0.0)
    st = lib.svm_solve(fake, _ffi.F32, fake, 10, 4, ctypes.byref(opts), fake, size.value - 256, None, fake,
                       ctypes.byref(rep))
    assert st == 8
    opts = _ffi.Options(1e-3, 0.0, 10, _ffi.MODE_CERTIFIED, 1000, 64, 10, 1.5)
    st = lib.svm_solve(fake, _ffi.F32, fake, 10, 4, ctypes.byref(opts), fake, 1 << 30, None, fake, ctypes.byref(rep))
    assert st == 1 and b"eta" in lib.pdscp_last_error()
    bwd = lambda problem, dtype, T, ws_bytes: lib.mwu_backward(problem, fake, dtype, None, None, 10, 4, 1.0, 0.1,
                                                               0.0, T, None, fake, ws_bytes, None, fake, None)
    assert bwd(_ffi.SVM, _ffi.F32, 5, 1 << 30) == 1 and b"labels" in lib.pdscp_last_error()
    assert bwd(_ffi.SES, 3, 5, 1 << 30) == 1 and b"dtype" in lib.pdscp_last_error()
    assert bwd(_ffi.SES, _ffi.BF16, 5, 1024) == 8  # bfloat16 points pass the checks up to the workspace size
    assert bwd(_ffi.SES, _ffi.F32, 0, 1 << 30) == 1
    assert bwd(_ffi.SES, _ffi.F32, 5, 1024) == 8
    size = ctypes.c_size_t()
    assert lib.mwu_backward_workspace_size(_ffi.SES, 10, 4, 5, ctypes.byref(size)) == 0
    small = size.value
    assert lib.mwu_backward_workspace_size(_ffi.SES, 10, 4, 500, ctypes.byref(size)) == 0
    assert size.value >= small + 495 * (4 + 2 * 4) * 4  # one tape entry per iteration


def test_batch_validation_without_gpu(lib):
    n = (ctypes.c_int64 * 2)(100, 1)
    d = (ctypes.c_int32 * 2)(8, 8)
    size = ctypes.c_size_t()
    assert lib.ses_batch_workspace_size(2, n, d, 4096, ctypes.byref(size)) == 1  # n < 2
    n[1] = 50
    d[1] = 65
    assert lib.ses_batch_workspace_size(2, n, d, 4096, ctypes.byref(size)) == 7  # d > 64
    d[1] = 8
    assert lib.ses_batch_workspace_size(2, n, d, 16, ctypes.byref(size)) == 1    # tile_rows < 32
    assert lib.ses_batch_workspace_size(2, n, d, 4096, ctypes.byref(size)) == 0 and size.value > 0
    offs = (ctypes.c_int64 * 2)(0, 800)
    fake = ctypes.c_void_p(1 << 20)
    st = lib.ses_batch_init(2, fake, _ffi.F32, 1000, offs, n, d, 4096, fake, 1 << 30, None)  # 800 + 400 > 1000
    assert st == 1 and b"extends past" in lib.pdscp_last_error()
    st = lib.ses_batch_init(2, fake, _ffi.BF16, 1000, offs, n, d, 4096, fake, 1 << 30, None)  # lengths in elements
    assert st == 1 and b"extends past" in lib.pdscp_last_error()
    st = lib.ses_batch_init(2, fake, 5, 2000, offs, n, d, 4096, fake, 1 << 30, None)
    assert st == 1 and b"dtype" in lib.pdscp_last_error()
    odd = ctypes.c_void_p((1 << 20) + 1)  # not aligned to a bfloat16 element
    st = lib.ses_batch_init(2, odd, _ffi.BF16, 2000, offs, n, d, 4096, fake, 1 << 30, None)
    assert st == 1 and b"aligned" in lib.pdscp_last_error()
    alpha = ctypes.c_void_p(1 << 21)
    assert lib.ses_batch_step(2, fake, 9, alpha, alpha, fake, 1 << 30, None, None) == 1


def test_svm_batch_validation_without_gpu(lib):
    n = (ctypes.c_int64 * 2)(100, 1)
    d = (ctypes.c_int32 * 2)(8, 8)
    size = ctypes.c_size_t()
    assert lib.svm_batch_workspace_size(2, n, d, 4096, ctypes.byref(size)) == 1  # n < 2
    n[1] = 50
    d[1] = 65
    assert lib.svm_batch_workspace_size(2, n, d, 4096, ctypes.byref(size)) == 7  # d > 64
    d[1] = 8
    assert lib.svm_batch_workspace_size(2, n, d, 4096, ctypes.byref(size)) == 0
    ses = ctypes.c_size_t()
    assert lib.ses_batch_workspace_size(2, n, d, 4096, ctypes.byref(ses)) == 0
    assert size.value > ses.value  # wider partial rows, label offsets and D per instance
    offs = (ctypes.c_int64 * 2)(0, 800)
    loffs = (ctypes.c_int64 * 2)(0, 100)
    fake = ctypes.c_void_p(1 << 20)
    lab = ctypes.c_void_p(1 << 22)
    st = lib.svm_batch_init(2, fake, _ffi.F32, 1000, offs, n, d, lab, 150, loffs, 4096, fake, 1 << 30, None)
    assert st == 1 and b"extends past" in lib.pdscp_last_error()  # points: 800 + 400 > 1000
    st = lib.svm_batch_init(2, fake, _ffi.F32, 2000, offs, n, d, lab, 149, loffs, 4096, fake, 1 << 30, None)
    assert st == 1 and b"labels" in lib.pdscp_last_error()  # labels: 100 + 50 > 149
    st = lib.svm_batch_init(2, fake, _ffi.F32, 2000, offs, n, d, None, 150, loffs, 4096, fake, 1 << 30, None)
    assert st == 1 and b"null" in lib.pdscp_last_error()
    st = lib.svm_batch_init(2, fake, 5, 2000, offs, n, d, lab, 150, loffs, 4096, fake, 1 << 30, None)
    assert st == 1 and b"dtype" in lib.pdscp_last_error()
    st = lib.svm_batch_init(2, fake, _ffi.F32, 2000, offs, n, d, lab, 150, loffs, 4096, fake, 64, None)
    assert st == 8  # workspace too small
    opts = _ffi.Options(1e-3, 0.0, 10, 7, 1000, 64, 10, 0.0)
    st = lib.svm_batch_solve_init(2, fake, _ffi.F32, 2000, offs, n, d, lab, 150, loffs, 4096, ctypes.byref(opts),
                                  fake, 1 << 30, None)
    assert st == 1 and b"options" in lib.pdscp_last_error()
    alpha = ctypes.c_void_p(1 << 21)
    assert lib.svm_batch_step(2, fake, 9, lab, alpha, alpha, fake, 1 << 30, None, None) == 1
    assert lib.svm_batch_step(2, fake, _ffi.F32, None, alpha, alpha, fake, 1 << 30, None, None) == 1
    assert lib.svm_batch_solve_run(2, fake, None, fake, 1 << 30, 8, 100, None, None, None) == 1


def test_shard_validation_without_gpu(lib):
    w = ctypes.c_int32()
    assert lib.mwu_shard_row_width(_ffi.SES, 32, ctypes.byref(w)) == 0 and w.value == 4 + 32
    assert lib.mwu_shard_row_width(_ffi.SVM, 5, ctypes.byref(w)) == 0 and w.value == 4 + 2 * 8
    assert lib.mwu_shard_row_width(_ffi.SES, 0, ctypes.byref(w)) == 7
    fake = ctypes.c_void_p(1 << 20)
    st = lib.mwu_shard_partial(_ffi.SES, fake, _ffi.F32, None, None, 0, 4, 1, 1.0, 0.1, 0.0, 0, fake, fake,
                               1 << 30, None, fake)
    assert st == 1 and b"n >= 1" in lib.pdscp_last_error()
    st = lib.mwu_shard_partial(_ffi.SES, fake, _ffi.F32, None, None, 5, 4, 2, 1.0, 0.1, 0.0, 0, fake, fake,
                               1 << 30, None, fake)
    assert st == 1 and b"holds_first" in lib.pdscp_last_error()
    st = lib.mwu_shard_partial(_ffi.SES, fake, _ffi.F32, None, None, 5, 4, 1, 1.0, 0.1, 0.0, 0, fake, fake,
                               1 << 30, None, None)
    assert st == 1
    st = lib.mwu_shard_finish(_ffi.SES, fake, 0, fake, _ffi.F32, None, 4, 1.0, 0.1, 0.0, 0, fake, None, None)
    assert st == 1 and b"ranks" in lib.pdscp_last_error()
    st = lib.mwu_shard_finish(_ffi.SES, fake, 2, None, _ffi.F32, None, 4, 1.0, 0.1, 0.0, 0, fake, None, None)
    assert st == 1 and b"v_1" in lib.pdscp_last_error()
    st = lib.mwu_shard_finish(_ffi.SVM, fake, 2, None, _ffi.F32, None, 4, 1.0, 0.1, 0.0, 0, fake, None, None)
    assert st == 1 and b"D > 0" in lib.pdscp_last_error()
    st = lib.mwu_shard_init(_ffi.SES, None, _ffi.F32, 4, 0, 1e-4, 10, fake, fake, 1 << 30, None)
    assert st == 1 and b"v_1" in lib.pdscp_last_error()


def test_batch_search_validation_without_gpu(lib):
    n = (ctypes.c_int64 * 2)(100, 50)
    d = (ctypes.c_int32 * 2)(8, 8)
    offs = (ctypes.c_int64 * 2)(0, 800)
    fake = ctypes.c_void_p(1 << 20)
    bad = _ffi.Options(0.0, 1e-4, 10, 0, 1000, 1, 10, 0.0)  # eps = 0
    st = lib.ses_batch_solve_init(2, fake, _ffi.F32, 1200, offs, n, d, 512, ctypes.byref(bad), fake, 1 << 30, None)
    assert st == 1 and b"options" in lib.pdscp_last_error()
    bad = _ffi.Options(1e-3, 1e-4, 10, 7, 1000, 1, 10, 0.0)  # unknown mode
    assert lib.ses_batch_solve_init(2, fake, _ffi.F32, 1200, offs, n, d, 512, ctypes.byref(bad), fake, 1 << 30, None) == 1
    bad = _ffi.Options(1e-3, 0.0, 10, _ffi.MODE_CERTIFIED, 1000, 0, 10, 0.0)  # certified needs a poll interval
    assert lib.ses_batch_solve_init(2, fake, _ffi.F32, 1200, offs, n, d, 512, ctypes.byref(bad), fake, 1 << 30, None) == 1
    launches, done = ctypes.c_int64(), ctypes.c_int32()
    assert lib.ses_batch_solve_run(2, fake, fake, 1 << 30, 0, 10, None, ctypes.byref(launches),
                                   ctypes.byref(done)) == 1
    tr = ctypes.c_int32()
    assert lib.ses_batch_autotune(2, fake, _ffi.F32, 1200, offs, n, d, None, fake, 1 << 30, None, None, None, None,
                                  None) == 1
    assert lib.ses_batch_set_launch(2, fake, fake, 4, 0, None) == 1  # CTAs per SM outside [0, 3]
    assert lib.ses_batch_set_launch(2, fake, fake, 1, 2, None) == 1  # unknown layout policy
    assert lib.ses_batch_set_launch(2, None, fake, 1, 0, None) == 1


def test_multi_validation_without_gpu(lib):
    size = ctypes.c_size_t()
    assert lib.ses_multi_workspace_size(32, 3, ctypes.byref(size)) == 7
    assert lib.ses_multi_workspace_size(65, 2, ctypes.byref(size)) == 7
    assert lib.ses_multi_workspace_size(64, 8, ctypes.byref(size)) == 0 and size.value > 0
    assert lib.ses_multi_state_stride(32, ctypes.byref(size)) == 0 and size.value % 256 == 0
    fake = ctypes.c_void_p(1 << 20)
    assert lib.ses_multi_step(fake, None, 1, 4, 2, fake, fake, fake, fake, 1 << 30, None, None) == 1
    st = lib.ses_multi_step(fake, None, 10, 4, 2, fake, fake, ctypes.c_void_p((1 << 20) + 16), fake, 1 << 30,
                            None, None)
    assert st == 1 and b"misaligned" in lib.pdscp_last_error()
    assert lib.ses_multi_step(fake, None, 10, 4, 2, fake, fake, fake, fake, 64, None, None) == 8


def test_pack_instances_layout_without_gpu():
    # host logic of the batch binding: every instance starts on a 4-element boundary (16 bytes for
    # float32, 8 for bfloat16, the chunk loads of the batched pass), rows are stored in order, and the
    # bfloat16 buffer holds the rounded values
    import numpy as np
    import torch

    from paper_2405_09157_gb300 import api
    rng = np.random.default_rng(0)
    arrays = [rng.standard_normal((n, d)).astype(np.float32) for n, d in [(3, 5), (7, 4), (2, 1), (5, 3)]]
    for dt in (torch.float32, torch.bfloat16):
        pts, offs, n, d = api.pack_instances(arrays, device="cpu", dtype=dt)
        assert pts.dtype == dt and pts.dim() == 1
        assert list(n) == [3, 7, 2, 5] and list(d) == [5, 4, 1, 3]
        assert np.all(offs % 4 == 0) and np.all(np.diff(offs) >= (n * d)[:-1])
        for k, a in enumerate(arrays):
            got = pts[offs[k]:offs[k] + a.size].float().view(a.shape)
            want = torch.from_numpy(a).to(dt).float()
            assert torch.equal(got, want)


def test_binding_rejects_host_tensors_without_gpu():
    # a host pointer never reaches a kernel: the binding refuses CPU tensors before the call
    import pytest
    import torch

    from paper_2405_09157_gb300 import api
    with pytest.raises(ValueError, match="CUDA tensor"):
        api._vp(torch.zeros(4))
    assert api._vp(None) is None
    with pytest.raises(ValueError, match="CUDA"):
        api.bounds(api.SES, torch.zeros(8, 2))


def test_header_is_plain_c_and_links(lib, tmp_path):
    # a C99 program (no C++) includes the header with every warning on, links the library and calls it
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    src = tmp_path / "use.c"
    src.write_text(
        '#include <stdio.h>\n#include "pdscp.h"\n'
        "int main(void) {\n"
        "  size_t b = 0;\n"
        "  pdscp_status st = pdscp_state_size(PDSCP_SES, 32, &b);\n"
        '  printf("%d %zu\\n", (int)st, b);\n'
        "  st = mwu_step(7, NULL, PDSCP_F32, NULL, NULL, 10, 4, 1.0, 0.1, 0.0, 0, NULL, NULL, 0, NULL, NULL);\n"
        '  printf("%d %s\\n", (int)st, pdscp_last_error());\n'
        "  return 0;\n}\n")
    libdir = os.path.dirname(build.LIB)
    exe = tmp_path / "use"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.dirname(HEADER),
                        str(src), "-L", libdir, "-lpdscp", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    first, second = out.stdout.splitlines()
    size = ctypes.c_size_t()
    assert lib.pdscp_state_size(_ffi.SES, 32, ctypes.byref(size)) == 0
    assert first == f"0 {size.value}"
    assert second.startswith("1 ") and "problem" in second
