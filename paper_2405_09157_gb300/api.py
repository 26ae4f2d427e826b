"""Thin PyTorch-facing binding of the C ABI (argument marshalling only).

Torch supplies device memory (tensors) and the stream; every step of the
method runs in the library's CUDA kernels. Names follow include/pdscp.h.
"""

import ctypes
import functools

import numpy as np
import torch

from . import _ffi
from ._ffi import BF16, F32, SES, SVM, check, load

STEP_DTYPE = np.dtype([("oracle_value", "<f8"), ("objective", "<f8"), ("lower_bound", "<f8"),
                       ("upper_bound", "<f8"), ("t", "<i8"), ("failed", "<i4"), ("stopped", "<i4"),
                       ("status", "<i4"), ("outcome", "<i4"), ("k", "<f8"), ("dual_bound", "<f8")])
STEP_BYTES = 72
REPORT_DTYPE = np.dtype([("value", "<f8"), ("lower_bound", "<f8"), ("upper_bound", "<f8"), ("D", "<f8"),
                         ("search_L", "<f8"), ("search_U", "<f8"), ("iters", "<i8"), ("search_steps", "<i4"),
                         ("status", "<i4")])


def _vp(t):
    """Device pointer of a CUDA tensor (None passes NULL). Every pointer this
    binding hands to the library is dereferenced by a kernel, so a host tensor
    is rejected here rather than read by the GPU."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"expected a CUDA tensor, got one on {t.device}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def dtype_code(t):
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.bfloat16:
        return BF16
    raise TypeError(f"points must be float32 or bfloat16, got {t.dtype}")


def _points(pts):
    if not pts.is_cuda or pts.dim() != 2 or not pts.is_contiguous():
        raise ValueError("points must be a contiguous 2-D CUDA tensor (n, d)")
    return pts.shape[0], pts.shape[1], dtype_code(pts)


def _rows(t, n, dtype, name):
    """Checks an optional per-row argument (radii, labels, per-instance or
    per-candidate values): contiguous, of `dtype`, at least n entries."""
    if t is not None and (t.dtype != dtype or not t.is_contiguous() or t.numel() < n):
        raise ValueError(f"{name} must be a contiguous {dtype} tensor of at least {n} entries")


def _bytes(t, nbytes, name):
    """Checks an optional caller-owned buffer: contiguous and at least nbytes long."""
    if t is not None and (not t.is_contiguous() or t.numel() * t.element_size() < nbytes):
        raise ValueError(f"{name} must be a contiguous buffer of at least {nbytes} bytes")


def _state(problem, d, state):
    _bytes(state, state_size(problem, d), "state")


def _records(out, k=1):
    _bytes(out, k * STEP_BYTES, "out (step records)")


def _per_row(problem, n, radii, labels):
    _rows(radii, n, torch.float32, "radii")
    _rows(labels, n, torch.int8, "labels")


def workspace_size(problem, n, d):
    out = ctypes.c_size_t()
    check(load().pdscp_workspace_size(problem, n, d, ctypes.byref(out)), "pdscp_workspace_size")
    return out.value


@functools.lru_cache(maxsize=None)
def state_size(problem, d):
    out = ctypes.c_size_t()
    check(load().pdscp_state_size(problem, d, ctypes.byref(out)), "pdscp_state_size")
    return out.value


def workspace(problem, n, d, device="cuda"):
    """Zeroed device workspace for this problem size (uint8 tensor)."""
    return torch.zeros(workspace_size(problem, n, d), dtype=torch.uint8, device=device)


def new_state(problem, d, device="cuda"):
    return torch.zeros(state_size(problem, d), dtype=torch.uint8, device=device)


def new_steps(k, device="cuda"):
    """Device buffer for k pdscp_step_out records."""
    return torch.zeros((k, STEP_BYTES), dtype=torch.uint8, device=device)


def decode_steps(buf):
    """pdscp_step_out records (uint8 tensor, any device) -> numpy structured array."""
    a = buf.detach().to("cpu").contiguous().numpy().reshape(-1)
    return a.view(STEP_DTYPE)


def bounds(problem, pts, radii=None, ws=None, stream=None):
    """D of Sec. 4.1 (SES) or Lemma 6 (SVM) as a (1,) float64 CUDA tensor."""
    n, d, dt = _points(pts)
    _rows(radii, n, torch.float32, "radii")
    ws = workspace(problem, n, d, pts.device) if ws is None else ws
    out = torch.empty(1, dtype=torch.float64, device=pts.device)
    check(load().pdscp_bounds(problem, _vp(pts), dt, _vp(radii), n, d, _vp(ws), ws.numel(),
                              _stream(stream), _vp(out)), "pdscp_bounds")
    return out


def state_init(problem, pts, state, ws, rules=_ffi.RULES_NONE, delta=1e-4, patience=10, stream=None):
    n, d, dt = _points(pts)
    _state(problem, d, state)
    check(load().mwu_state_init(problem, _vp(pts), dt, n, d, rules, delta, patience, _vp(state),
                                _vp(ws), ws.numel(), _stream(stream)), "mwu_state_init")


def mwu_step(problem, pts, alpha, eta_over_rho, state, ws, out=None, D=0.0, radii=None, labels=None,
             eval_only=False, stream=None):
    """One alpha-FTP iteration on the device (no host sync)."""
    n, d, dt = _points(pts)
    _state(problem, d, state)
    _per_row(problem, n, radii, labels)
    _records(out)
    check(load().mwu_step(problem, _vp(pts), dt, _vp(radii), _vp(labels), n, d, float(alpha),
                          float(eta_over_rho), float(D), int(bool(eval_only)), _vp(state), _vp(ws),
                          ws.numel(), _stream(stream), _vp(out)), "mwu_step")


def mwu_run(problem, pts, alpha, eta_over_rho, k, state, ws, out=None, D=0.0, radii=None, labels=None, stream=None):
    """k alpha-FTP iterations enqueued back to back, consecutive launches
    overlapping (no host sync); out: k records or None. Bit-identical to k
    mwu_step calls."""
    n, d, dt = _points(pts)
    _state(problem, d, state)
    _per_row(problem, n, radii, labels)
    _records(out, int(k))
    check(load().mwu_run(problem, _vp(pts), dt, _vp(radii), _vp(labels), n, d, float(alpha), float(eta_over_rho),
                         float(D), int(k), _vp(state), _vp(ws), ws.numel(), _stream(stream), _vp(out)), "mwu_run")


def mwu_step_noalloc(problem, pts, alpha, eta_over_rho, state, out=None, D=0.0, radii=None, labels=None,
                     eval_only=False, stream=None):
    """mwu_step for callers that cannot allocate device memory: the scratch is
    the library's built-in 2 MiB array (shared by all calls on a device, so
    calls must not overlap on the GPU)."""
    n, d, dt = _points(pts)
    _state(problem, d, state)
    _per_row(problem, n, radii, labels)
    _records(out)
    check(load().mwu_step_noalloc(problem, _vp(pts), dt, _vp(radii), _vp(labels), n, d, float(alpha),
                                  float(eta_over_rho), float(D), int(bool(eval_only)), _vp(state),
                                  _stream(stream), _vp(out)), "mwu_step_noalloc")


def state_read(problem, d, state, stream=None, device="cuda"):
    """(mean, best) float32 tensors of a state: SES (ubar, best centre); SVM
    ((wbar, s1bar, s2bar), best direction)."""
    _state(problem, d, state)
    m = torch.empty(d + (2 if problem == SVM else 0), dtype=torch.float32, device=device)
    b = torch.empty(d, dtype=torch.float32, device=device)
    check(load().mwu_state_read(problem, d, _vp(state), _vp(m), _vp(b), _stream(stream)), "mwu_state_read")
    return m, b


def state_set(problem, pts, t, mean, state, ws, radii=None, labels=None, D=0.0, stream=None):
    """Resume from a checkpoint: t and the running mean (float64 CUDA tensor;
    SVM: wbar then s1bar, s2bar)."""
    n, d, dt = _points(pts)
    _state(problem, d, state)
    _per_row(problem, n, radii, labels)
    mean = mean.to(device=pts.device, dtype=torch.float64).contiguous()
    _rows(mean, d + (2 if problem == SVM else 0), torch.float64, "mean")
    check(load().mwu_state_set(problem, _vp(pts), dt, _vp(radii), _vp(labels), n, d, int(t), _vp(mean),
                               float(D), _vp(state), _vp(ws), ws.numel(), _stream(stream)), "mwu_state_set")


# --- multi-candidate iteration (SES) -----------------------------------------

class MultiMWU:
    """k alpha-FTPs of one SES instance (float32 points, d <= 64) advanced by
    one pass over the points per iteration, each with its own alpha and
    eta/rho (k in {1, 2, 4, 8, 16}; k = 16 needs d = 32 and runs on the
    tensor cores)."""

    def __init__(self, pts, k, radii=None, rules=_ffi.RULES_NONE, delta=1e-4, patience=10, stream=None):
        n, d, dt = _points(pts)
        if dt != F32:
            raise TypeError("multi-candidate iterations take float32 points")
        _rows(radii, n, torch.float32, "radii")
        lib = load()
        stride, size = ctypes.c_size_t(), ctypes.c_size_t()
        check(lib.ses_multi_state_stride(d, ctypes.byref(stride)), "ses_multi_state_stride")
        check(lib.ses_multi_workspace_size(d, k, ctypes.byref(size)), "ses_multi_workspace_size")
        self.pts, self.k, self.d, self.radii = pts, k, d, radii
        self.stride = stride.value
        self.states = torch.zeros(k * self.stride, dtype=torch.uint8, device=pts.device)
        self.ws = torch.zeros(size.value, dtype=torch.uint8, device=pts.device)
        init_ws = workspace(SES, n, d, pts.device)
        for j in range(k):
            state_init(SES, pts, self.state(j), init_ws, rules, delta, patience, stream)

    def state(self, j):
        return self.states[j * self.stride:(j + 1) * self.stride]

    def step(self, alpha, eta_over_rho, out=None, stream=None):
        """alpha, eta_over_rho: k float64 CUDA tensors; out: k records or None."""
        n = self.pts.shape[0]
        _rows(alpha, self.k, torch.float64, "alpha")
        _rows(eta_over_rho, self.k, torch.float64, "eta_over_rho")
        _records(out, self.k)
        check(load().ses_multi_step(_vp(self.pts), _vp(self.radii), n, self.d, self.k, _vp(alpha),
                                    _vp(eta_over_rho), _vp(self.states), _vp(self.ws), self.ws.numel(),
                                    _stream(stream), _vp(out)), "ses_multi_step")

    def read(self, j, stream=None):
        return state_read(SES, self.d, self.state(j), stream, self.pts.device)


# --- reverse sweep (SES) ----------------------------------------------------

def backward_workspace_size(n, d, T, problem=SES):
    out = ctypes.c_size_t()
    check(load().mwu_backward_workspace_size(problem, n, d, T, ctypes.byref(out)), "mwu_backward_workspace_size")
    return out.value


def mwu_backward(pts, alpha, eta_over_rho, T, radii=None, seed=None, ws=None, out=None, stream=None,
                 problem=SES, labels=None, D=0.0):
    """Gradient of seed * f at the final mean after T alpha-FTP iterations
    from t = 0 at fixed alpha, eta/rho (SES: the radius; SVM: the margin, with
    labels and D) with respect to the points (float32, or bfloat16 widened on
    load; the gradient is float32 either way). seed: one-element
    float64 CUDA tensor or None (1). Returns (grad, ws)."""
    n, d, dt = _points(pts)
    _per_row(problem, n, radii, labels)
    _records(out)
    if ws is None:
        ws = torch.empty(backward_workspace_size(n, d, T, problem), dtype=torch.uint8, device=pts.device)
    grad = torch.empty((n, d), dtype=torch.float32, device=pts.device)
    if seed is not None:
        seed = seed.to(device=pts.device, dtype=torch.float64).contiguous()
    check(load().mwu_backward(problem, _vp(pts), dt, _vp(radii), _vp(labels), n, d, float(alpha),
                              float(eta_over_rho), float(D), int(T), _vp(seed), _vp(ws), ws.numel(),
                              _stream(stream), _vp(grad), _vp(out)), "mwu_backward")
    return grad, ws


class SesUnrolledRadius(torch.autograd.Function):
    """f(ubar^T) of the SES alpha-FTP as a differentiable function of the
    points: forward = T mwu_step iterations and one evaluation pass; backward =
    mwu_backward seeded with the incoming gradient."""

    @staticmethod
    def forward(ctx, pts, alpha, eta_over_rho, T, radii=None):
        m = MWU(SES, pts.detach(), radii=radii)
        for _ in range(T):
            m.step(alpha, eta_over_rho)
        rec = new_steps(1, pts.device)
        m.step(alpha, eta_over_rho, out=rec, eval_only=True)
        ctx.save_for_backward(pts)
        ctx.args = (alpha, eta_over_rho, T, radii)
        return rec.view(torch.float64)[0, 1].clone()  # the record's objective: f at the final mean

    @staticmethod
    def backward(ctx, grad_out):
        (pts,) = ctx.saved_tensors
        alpha, eta_over_rho, T, radii = ctx.args
        grad, _ = mwu_backward(pts.detach(), alpha, eta_over_rho, T, radii, seed=grad_out.reshape(1))
        return grad, None, None, None, None


def ses_unrolled_radius(pts, alpha, eta_over_rho, T, radii=None):
    """Differentiable SES radius after T alpha-FTP iterations (float64 0-dim tensor)."""
    return SesUnrolledRadius.apply(pts, alpha, eta_over_rho, T, radii)


class SvmUnrolledMargin(torch.autograd.Function):
    """f(wbar^T) of the SVM alpha-FTP (the margin of Sec. 5) as a differentiable
    function of the points: forward = T mwu_step iterations and one evaluation
    pass; backward = mwu_backward seeded with the incoming gradient."""

    @staticmethod
    def forward(ctx, pts, labels, alpha, eta_over_rho, T, D):
        m = MWU(SVM, pts.detach(), labels=labels)
        for _ in range(T):
            m.step(alpha, eta_over_rho, D=D)
        rec = new_steps(1, pts.device)
        m.step(alpha, eta_over_rho, out=rec, D=D, eval_only=True)
        ctx.save_for_backward(pts)
        ctx.args = (labels, alpha, eta_over_rho, T, D)
        return rec.view(torch.float64)[0, 1].clone()  # the record's objective: the margin at the final mean

    @staticmethod
    def backward(ctx, grad_out):
        (pts,) = ctx.saved_tensors
        labels, alpha, eta_over_rho, T, D = ctx.args
        grad, _ = mwu_backward(pts.detach(), alpha, eta_over_rho, T, seed=grad_out.reshape(1), problem=SVM,
                               labels=labels, D=D)
        return grad, None, None, None, None, None


def svm_unrolled_margin(pts, labels, alpha, eta_over_rho, T, D):
    """Differentiable SVM margin after T alpha-FTP iterations (float64 0-dim tensor)."""
    return SvmUnrolledMargin.apply(pts, labels, alpha, eta_over_rho, T, D)


# --- row-sharded iteration -------------------------------------------------

def shard_rows(n, world, rank):
    """[lo, hi) of `rank`'s contiguous block of rows: n split as evenly as
    possible, in rank order (rank 0 holds row 0, the SES easy cone v_1)."""
    if not (0 <= rank < world) or n < world:
        raise ValueError(f"cannot split {n} rows over {world} ranks (rank {rank})")
    base, rem = divmod(n, world)
    lo = rank * base + min(rank, rem)
    return lo, lo + base + (1 if rank < rem else 0)


def shard_row_width(problem, d):
    """Width, in (float, float) pairs, of a shard's row of column totals."""
    w = ctypes.c_int32()
    check(load().mwu_shard_row_width(problem, d, ctypes.byref(w)), "mwu_shard_row_width")
    return w.value


def exchange_rows(row, world, group=None):
    """All-gather of one row per rank into a (world, len) tensor in rank order
    (torch.distributed: NCCL for CUDA tensors, gloo for CPU ones)."""
    if world == 1:
        return row.view(1, -1)
    import torch.distributed as dist
    rows = torch.empty((world, row.numel()), dtype=row.dtype, device=row.device)
    dist.all_gather(list(rows.unbind(0)), row.contiguous(), group=group)
    return rows


def shard_init(problem, first, d, state, ws, dtype=F32, rules=_ffi.RULES_NONE, delta=1e-4, patience=10,
               stream=None):
    _state(problem, d, state)
    _rows(first, d, torch.bfloat16 if dtype == BF16 else torch.float32, "first")
    check(load().mwu_shard_init(problem, _vp(first), dtype, d, rules, delta, patience, _vp(state), _vp(ws),
                                ws.numel(), _stream(stream)), "mwu_shard_init")


def shard_partial(problem, pts, holds_first, alpha, eta_over_rho, state, ws, row, D=0.0, radii=None,
                  labels=None, eval_only=False, stream=None):
    """One pass over this shard; writes its column totals to `row` (float32
    CUDA tensor of 2 * shard_row_width floats)."""
    n, d, dt = _points(pts)
    _state(problem, d, state)
    _per_row(problem, n, radii, labels)
    _rows(row, 2 * shard_row_width(problem, d), torch.float32, "row")
    check(load().mwu_shard_partial(problem, _vp(pts), dt, _vp(radii), _vp(labels), n, d, int(bool(holds_first)),
                                   float(alpha), float(eta_over_rho), float(D), int(bool(eval_only)), _vp(state),
                                   _vp(ws), ws.numel(), _stream(stream), _vp(row)), "mwu_shard_partial")


def shard_finish(problem, rows, d, alpha, eta_over_rho, state, first=None, first_radius=None, dtype=F32, D=0.0,
                 eval_only=False, out=None, stream=None):
    """Reduces the shards' rows ((ranks, 2 * width) float32, rank order) and
    finishes the iteration on this replica of the state."""
    _state(problem, d, state)
    _rows(rows, rows.shape[0] * 2 * shard_row_width(problem, d), torch.float32, "rows")
    _rows(first, d, torch.bfloat16 if dtype == BF16 else torch.float32, "first")
    _rows(first_radius, 1, torch.float32, "first_radius")
    _records(out)
    check(load().mwu_shard_finish(problem, _vp(rows), rows.shape[0], _vp(first), dtype, _vp(first_radius), d,
                                  float(alpha), float(eta_over_rho), float(D), int(bool(eval_only)), _vp(state),
                                  _stream(stream), _vp(out)), "mwu_shard_finish")


class ShardedMWU:
    """One alpha-FTP whose rows are split over the ranks of a process group
    (one GPU per rank, `shard` = this rank's rows from shard_rows). Every rank
    keeps a replica of the O(d) state; an iteration is a pass over the shard,
    an all-gather of one row of column totals per rank, and the same finish on
    every rank. first: v_1 (SES; the first row of rank 0's shard), on every
    rank."""

    def __init__(self, problem, shard, first, rank, world, labels=None, radii=None, first_radius=None,
                 group=None, rules=_ffi.RULES_NONE, delta=1e-4, patience=10, stream=None):
        n, d, dt = _points(shard)
        self.problem, self.shard, self.first, self.rank, self.world = problem, shard, first, rank, world
        self.labels, self.radii, self.first_radius, self.group = labels, radii, first_radius, group
        self.d, self.dtype = d, dt
        self.width = shard_row_width(problem, d)
        self.row = torch.zeros(2 * self.width, dtype=torch.float32, device=shard.device)
        self.ws = workspace(problem, n, d, shard.device)
        self.state = new_state(problem, d, shard.device)
        shard_init(problem, first, d, self.state, self.ws, dt, rules, delta, patience, stream)

    def step(self, alpha, eta_over_rho, D=0.0, out=None, eval_only=False, stream=None):
        shard_partial(self.problem, self.shard, self.rank == 0, alpha, eta_over_rho, self.state, self.ws, self.row,
                      D, self.radii, self.labels, eval_only, stream)
        rows = exchange_rows(self.row, self.world, self.group)
        shard_finish(self.problem, rows, self.d, alpha, eta_over_rho, self.state, self.first, self.first_radius,
                     self.dtype, D, eval_only, out, stream)

    def read(self, stream=None):
        return state_read(self.problem, self.d, self.state, stream, self.shard.device)


class MWU:
    """One alpha-FTP over resident points: state, workspace and step records."""

    def __init__(self, problem, pts, labels=None, radii=None, rules=_ffi.RULES_NONE, delta=1e-4,
                 patience=10):
        self.problem, self.pts, self.labels, self.radii = problem, pts, labels, radii
        self.n, self.d, _ = _points(pts)
        self.ws = workspace(problem, self.n, self.d, pts.device)
        self.state = new_state(problem, self.d, pts.device)
        self.rules, self.delta, self.patience = rules, delta, patience
        self.init()

    def init(self, stream=None):
        state_init(self.problem, self.pts, self.state, self.ws, self.rules, self.delta, self.patience, stream)

    def step(self, alpha, eta_over_rho, out=None, D=0.0, eval_only=False, stream=None):
        mwu_step(self.problem, self.pts, alpha, eta_over_rho, self.state, self.ws, out, D, self.radii,
                 self.labels, eval_only, stream)

    def run(self, alpha, eta_over_rho, k, out=None, D=0.0, stream=None):
        mwu_run(self.problem, self.pts, alpha, eta_over_rho, k, self.state, self.ws, out, D, self.radii, self.labels,
                stream)

    def set(self, t, mean, D=0.0, stream=None):
        state_set(self.problem, self.pts, t, mean, self.state, self.ws, self.radii, self.labels, D, stream)

    def read(self, stream=None):
        return state_read(self.problem, self.d, self.state, stream, self.pts.device)


def _options(eps, mode, max_iters, poll_every, max_steps, eta, delta, patience):
    m = {"practical": _ffi.MODE_PRACTICAL, "theory": _ffi.MODE_THEORY, "certified": _ffi.MODE_CERTIFIED,
         "coreset": _ffi.MODE_CORESET}[mode]
    return _ffi.Options(eps, delta, patience, m, max_iters, poll_every, max_steps, eta or 0.0)


def _report(r):
    return {k: getattr(r, k) for k, _ in _ffi.Report._fields_}


def ses_solve(pts, radii=None, eps=1e-3, mode="practical", max_iters=1_000_000, poll_every=256,
              max_steps=200, eta=None, delta=1e-4, patience=10, ws=None, stream=None, raise_on_budget=False):
    """(1+eps)-approximate smallest enclosing sphere; returns (centre tensor, report dict).

    mode: "practical" (the Sec. 5 rules; a stalled alpha-FTP is read as the
    affirmative answer, so the search range can close while the certificates
    stay wide), "theory" (T_i iterations of Theorem 2 per FTP) or "certified"
    (only proven conclusions; ends when the ball's radius is within 1 + eps of
    a certified lower bound; eta defaults to 1 and is halved when an FTP's own
    certificate gap stops shrinking); "coreset" (points only) is "certified"
    plus core-set certificates: the dual value of Frank-Wolfe weights on the
    points farthest from the running mean bounds the radius from below, the
    ball at their barycentre from above. The report holds the radius of an
    actual enclosing ball ("value" = "upper_bound"), the best lower bound, the
    search range, iterations and status (5 = budget spent, with valid bounds)."""
    n, d, dt = _points(pts)
    _rows(radii, n, torch.float32, "radii")
    ws = workspace(SES, n, d, pts.device) if ws is None else ws
    center = torch.empty(d, dtype=torch.float32, device=pts.device)
    opts = _options(eps, mode, max_iters, poll_every, max_steps, eta, delta, patience)
    rep = _ffi.Report()
    st = load().ses_solve(_vp(pts), dt, _vp(radii), n, d, ctypes.byref(opts), _vp(ws), ws.numel(),
                          _stream(stream), _vp(center), ctypes.byref(rep))
    if st != _ffi.PDSCP_OK and (raise_on_budget or st != 5):
        check(st, "ses_solve")
    return center, _report(rep)


def svm_solve(X, labels, eps=1e-3, mode="practical", max_iters=1_000_000, poll_every=256, max_steps=200,
              eta=None, delta=1e-4, patience=10, ws=None, stream=None, raise_on_budget=False):
    """(1-eps)-approximate hard-margin SVM; returns (best mean direction wbar, report dict).

    mode as in ses_solve, roles mirrored: "value" = "lower_bound" is the margin
    of the returned direction, "upper_bound" the best Claim 8 value (per
    iteration or averaged); "certified" ends when upper_bound <= (1 + eps)
    lower_bound; "coreset" is "certified" plus the core-set certificates
    (exact polytope distance of the 512 points per class nearest the best
    hyperplane, checked at 256, 512, 1024, ... iterations of the search)."""
    n, d, dt = _points(X)
    if labels is None or labels.numel() != n:
        raise ValueError("labels must be an int8 CUDA tensor of n entries in {+1, -1}")
    _rows(labels, n, torch.int8, "labels")
    ws = workspace(SVM, n, d, X.device) if ws is None else ws
    w = torch.empty(d, dtype=torch.float32, device=X.device)
    opts = _options(eps, mode, max_iters, poll_every, max_steps, eta, delta, patience)
    rep = _ffi.Report()
    st = load().svm_solve(_vp(X), dt, _vp(labels), n, d, ctypes.byref(opts), _vp(ws), ws.numel(),
                          _stream(stream), _vp(w), ctypes.byref(rep))
    if st != _ffi.PDSCP_OK and (raise_on_budget or st != 5):
        check(st, "svm_solve")
    return w, _report(rep)


def polytope_distance(P, Q, tol=1e-9, max_iter=None):
    """Exact polytope distance of two small point sets (Eq. PD), the host
    solver of the core-set certificates: P (nP x d), Q (nQ x d) array-likes,
    taken as float64. Returns (dist, mu, gamma) with mu, gamma the weights on
    the two simplices."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    if P.ndim != 2 or Q.ndim != 2 or P.shape[1] != Q.shape[1]:
        raise ValueError("P and Q must be 2-D with the same number of columns")
    nP, d = P.shape
    nQ = Q.shape[0]
    mu = np.zeros(max(nP, 1))
    ga = np.zeros(max(nQ, 1))
    dist = ctypes.c_double(0.0)
    it = 4 * (nP + nQ) + 64 if max_iter is None else int(max_iter)
    st = load().pdscp_polytope_distance(P.ctypes.data, nP, Q.ctypes.data, nQ, d, float(tol), it,
                                        mu.ctypes.data, ga.ctypes.data, ctypes.byref(dist))
    check(st, "pdscp_polytope_distance")
    return dist.value, mu[:nP], ga[:nQ]


def meb_dual(P, tol=1e-9, max_iter=200_000):
    """Dual bound of the minimum enclosing ball of a small point set (the host
    solver of the SES core-set certificates): P (m x d) array-like, taken as
    float64. Returns (lb, far, mu, centre): lb = sqrt(phi(mu)) <= OPT <= far,
    the radius of the ball at the centre (the weights' barycentre)."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    if P.ndim != 2:
        raise ValueError("P must be 2-D")
    m, d = P.shape
    mu = np.zeros(max(m, 1))
    c = np.zeros(max(d, 1))
    lb = ctypes.c_double(0.0)
    far = ctypes.c_double(0.0)
    st = load().pdscp_meb_dual(P.ctypes.data, m, d, float(tol), int(max_iter), mu.ctypes.data, c.ctypes.data,
                               ctypes.byref(lb), ctypes.byref(far))
    check(st, "pdscp_meb_dual")
    return lb.value, far.value, mu[:m], c[:d]


# ------------------------------------------------------------------ batched SES
def pack_instances(arrays, device="cuda", dtype=torch.float32):
    """Pack (n_i, d_i) arrays into one device buffer of dtype (torch.float32 or
    torch.bfloat16, rounded on the device), each instance starting on a
    4-element boundary. Returns (pts, offsets, n, d) where offsets, n (int64)
    and d (int32) are numpy arrays."""
    n = np.array([a.shape[0] for a in arrays], dtype=np.int64)
    d = np.array([a.shape[1] for a in arrays], dtype=np.int32)
    offs = np.zeros(len(arrays), dtype=np.int64)
    pos = 0
    for i, a in enumerate(arrays):
        pos = (pos + 3) & ~3
        offs[i] = pos
        pos += a.size
    host = np.zeros(max(pos, 4), dtype=np.float32)
    for i, a in enumerate(arrays):
        host[offs[i]:offs[i] + a.size] = np.ascontiguousarray(a, dtype=np.float32).reshape(-1)
    return torch.from_numpy(host).to(device).to(dtype), offs, n, d


class SesBatch:
    """Many independent SES alpha-FTPs advanced together, one launch per iteration."""

    def __init__(self, pts, offsets, n, d, tile_rows=4096, stream=None):
        """pts: the packed 1-D float32 or bfloat16 CUDA buffer of pack_instances."""
        self.pts, self.num = pts, len(n)
        self.dt = dtype_code(pts)
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self.n = np.ascontiguousarray(n, dtype=np.int64)
        self.d = np.ascontiguousarray(d, dtype=np.int32)
        self.tile_rows = int(tile_rows)
        self.ctas_per_sm, self.layout = 0, 0  # launch settings (ses_batch_set_launch; set by autotune)
        lib = load()
        size = ctypes.c_size_t()
        check(lib.ses_batch_workspace_size(self.num, self.n.ctypes.data, self.d.ctypes.data, self.tile_rows,
                                           ctypes.byref(size)), "ses_batch_workspace_size")
        self.ws = torch.zeros(size.value, dtype=torch.uint8, device=pts.device)
        self.init(stream)

    def init(self, stream=None):
        check(load().ses_batch_init(self.num, _vp(self.pts), self.dt, self.pts.numel(), self.offsets.ctypes.data,
                                    self.n.ctypes.data, self.d.ctypes.data, self.tile_rows, _vp(self.ws),
                                    self.ws.numel(), _stream(stream)), "ses_batch_init")
        self._apply_launch(stream)

    def _apply_launch(self, stream=None):
        if self.ctas_per_sm or self.layout:
            check(load().ses_batch_set_launch(self.num, _vp(self.pts), _vp(self.ws), self.ctas_per_sm, self.layout,
                                              _stream(stream)), "ses_batch_set_launch")

    def set_launch(self, ctas_per_sm=0, layout=0, stream=None):
        """CTAs per SM of the search's persistent grid (0: as many as fit) and
        the lane-layout policy (0: chunk loads where rows allow, 1: scalar)."""
        self.ctas_per_sm, self.layout = int(ctas_per_sm), int(layout)
        check(load().ses_batch_set_launch(self.num, _vp(self.pts), _vp(self.ws), self.ctas_per_sm, self.layout,
                                          _stream(stream)), "ses_batch_set_launch")

    def step(self, alpha, eta_over_rho, out=None, stream=None):
        """alpha, eta_over_rho: float64 CUDA tensors of one value per instance."""
        _rows(alpha, self.num, torch.float64, "alpha")
        _rows(eta_over_rho, self.num, torch.float64, "eta_over_rho")
        _records(out, self.num)
        check(load().ses_batch_step(self.num, _vp(self.pts), self.dt, _vp(alpha), _vp(eta_over_rho), _vp(self.ws),
                                    self.ws.numel(), _stream(stream), _vp(out)), "ses_batch_step")

    def _host_tables(self):
        return self.offsets.ctypes.data, self.n.ctypes.data, self.d.ctypes.data

    def autotune(self, eps=1e-3, mode="practical", stream=None, **kw):
        """Times the batched launch for each tile size that fits the workspace,
        1 to 3 CTAs per SM and both lane-layout policies (native autotuner)
        and re-initialises the batch with the fastest. Returns (tile_rows, ms
        per launch); the CTAs per SM and the layout are kept for solve()."""
        o = _options(eps, mode, kw.get("max_iters", 1_000_000), 1, kw.get("max_steps", 200), kw.get("eta"),
                     kw.get("delta", 1e-4), kw.get("patience", 10))
        lib = load()
        need = ctypes.c_size_t()
        check(lib.ses_batch_workspace_size(self.num, self.n.ctypes.data, self.d.ctypes.data, 512,
                                           ctypes.byref(need)), "ses_batch_workspace_size")
        if need.value > self.ws.numel():
            self.ws = torch.zeros(need.value, dtype=torch.uint8, device=self.pts.device)
        tr, ms, ctas, lay = ctypes.c_int32(), ctypes.c_float(), ctypes.c_int32(), ctypes.c_int32()
        offs, n, d = self._host_tables()
        check(lib.ses_batch_autotune(self.num, _vp(self.pts), self.dt, self.pts.numel(), offs, n, d, ctypes.byref(o),
                                     _vp(self.ws), self.ws.numel(), _stream(stream), ctypes.byref(tr),
                                     ctypes.byref(ms), ctypes.byref(ctas), ctypes.byref(lay)), "ses_batch_autotune")
        self.tile_rows = tr.value
        self.ctas_per_sm, self.layout = ctas.value, lay.value
        self.init(stream)
        return tr.value, ms.value

    def solve(self, eps=1e-3, mode="practical", max_iters=1_000_000, max_steps=200, eta=None, delta=1e-4,
              patience=10, launches_per_poll=32, max_launches=10_000_000, poll_every=256, stream=None):
        """The search of Sec. 3 for every instance, on the device. Returns
        (reports: structured numpy array of pdscp_report, centres: list of
        float32 arrays, launches run). poll_every: iterations between the
        certificate tests of mode "certified"."""
        o = _options(eps, mode, max_iters, poll_every, max_steps, eta, delta, patience)
        lib = load()
        offs, n, d = self._host_tables()
        check(lib.ses_batch_solve_init(self.num, _vp(self.pts), self.dt, self.pts.numel(), offs, n, d, self.tile_rows,
                                       ctypes.byref(o), _vp(self.ws), self.ws.numel(), _stream(stream)),
              "ses_batch_solve_init")
        self._apply_launch(stream)
        launches, done = ctypes.c_int64(), ctypes.c_int32()
        check(lib.ses_batch_solve_run(self.num, _vp(self.pts), _vp(self.ws), self.ws.numel(), launches_per_poll,
                                      max_launches, _stream(stream), ctypes.byref(launches), ctypes.byref(done)),
              "ses_batch_solve_run")
        return self.solve_read(eps, stream) + (launches.value,)

    def solve_read(self, eps, stream=None):
        reps = torch.zeros((self.num, ctypes.sizeof(_ffi.Report)), dtype=torch.uint8, device=self.pts.device)
        cen = torch.empty(int(self.d.sum()), dtype=torch.float32, device=self.pts.device)
        check(load().ses_batch_solve_read(self.num, _vp(self.ws), float(eps), _vp(reps), _vp(cen), _stream(stream)),
              "ses_batch_solve_read")
        torch.cuda.synchronize()
        rec = np.frombuffer(reps.cpu().numpy().tobytes(), dtype=REPORT_DTYPE)
        cut = np.concatenate([[0], np.cumsum(self.d)])
        ch = cen.cpu().numpy()
        return rec, [ch[cut[i]:cut[i + 1]] for i in range(self.num)]

    def read(self, stream=None):
        """(means, bests): lists of float32 numpy arrays, one per instance."""
        tot = int(self.d.sum())
        m = torch.empty(tot, dtype=torch.float32, device=self.pts.device)
        b = torch.empty(tot, dtype=torch.float32, device=self.pts.device)
        check(load().ses_batch_read(self.num, _vp(self.ws), _vp(m), _vp(b), _stream(stream)), "ses_batch_read")
        torch.cuda.synchronize()
        cut = np.concatenate([[0], np.cumsum(self.d)])
        mh, bh = m.cpu().numpy(), b.cpu().numpy()
        return [mh[cut[i]:cut[i + 1]] for i in range(self.num)], [bh[cut[i]:cut[i + 1]] for i in range(self.num)]


# ------------------------------------------------------------------ batched SVM
def pack_labels(labels, device="cuda"):
    """Pack per-instance label arrays (+1 / -1) into one int8 device buffer,
    one instance after another. Returns (labels tensor, label offsets int64)."""
    n = np.array([len(y) for y in labels], dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(n)[:-1]]).astype(np.int64)
    host = np.concatenate([np.asarray(y, dtype=np.int8).reshape(-1) for y in labels]) if len(labels) else \
        np.zeros(0, dtype=np.int8)
    return torch.from_numpy(np.ascontiguousarray(host)).to(device), offs


class SvmBatch:
    """Many independent hard-margin SVM alpha-FTPs advanced together, one launch per iteration."""

    def __init__(self, pts, offsets, n, d, labels, label_offsets, tile_rows=4096, stream=None):
        """pts: the packed 1-D float32 or bfloat16 CUDA buffer of pack_instances;
        labels, label_offsets: from pack_labels."""
        self.pts, self.num = pts, len(n)
        self.dt = dtype_code(pts)
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self.n = np.ascontiguousarray(n, dtype=np.int64)
        self.d = np.ascontiguousarray(d, dtype=np.int32)
        self.lab_offsets = np.ascontiguousarray(label_offsets, dtype=np.int64)
        if labels is None or len(self.lab_offsets) != self.num:
            raise ValueError("labels and one label offset per instance are required")
        _rows(labels, int(np.max(self.lab_offsets + self.n)) if self.num else 0, torch.int8, "labels")
        self.labels = labels
        self.tile_rows = int(tile_rows)
        size = ctypes.c_size_t()
        check(load().svm_batch_workspace_size(self.num, self.n.ctypes.data, self.d.ctypes.data, self.tile_rows,
                                              ctypes.byref(size)), "svm_batch_workspace_size")
        self.ws = torch.zeros(size.value, dtype=torch.uint8, device=pts.device)
        self.init(stream)

    def _tables(self):
        return (self.pts.numel(), self.offsets.ctypes.data, self.n.ctypes.data, self.d.ctypes.data,
                _vp(self.labels), self.labels.numel(), self.lab_offsets.ctypes.data, self.tile_rows)

    def init(self, stream=None):
        check(load().svm_batch_init(self.num, _vp(self.pts), self.dt, *self._tables(), _vp(self.ws),
                                    self.ws.numel(), _stream(stream)), "svm_batch_init")

    def step(self, alpha, eta_over_rho, out=None, stream=None):
        """alpha, eta_over_rho: float64 CUDA tensors of one value per instance."""
        _rows(alpha, self.num, torch.float64, "alpha")
        _rows(eta_over_rho, self.num, torch.float64, "eta_over_rho")
        _records(out, self.num)
        check(load().svm_batch_step(self.num, _vp(self.pts), self.dt, _vp(self.labels), _vp(alpha),
                                    _vp(eta_over_rho), _vp(self.ws), self.ws.numel(), _stream(stream), _vp(out)),
              "svm_batch_step")

    def read(self, stream=None):
        """(means, best directions, D): lists of float32 arrays per instance and a float64 array of D."""
        tot = int(self.d.sum())
        m = torch.empty(tot, dtype=torch.float32, device=self.pts.device)
        b = torch.empty(tot, dtype=torch.float32, device=self.pts.device)
        D = torch.empty(self.num, dtype=torch.float64, device=self.pts.device)
        check(load().svm_batch_read(self.num, _vp(self.ws), _vp(m), _vp(b), _vp(D), _stream(stream)),
              "svm_batch_read")
        torch.cuda.synchronize()
        cut = np.concatenate([[0], np.cumsum(self.d)])
        mh, bh = m.cpu().numpy(), b.cpu().numpy()
        return ([mh[cut[i]:cut[i + 1]] for i in range(self.num)], [bh[cut[i]:cut[i + 1]] for i in range(self.num)],
                D.cpu().numpy())

    def solve(self, eps=1e-3, mode="practical", max_iters=1_000_000, max_steps=200, eta=None, delta=1e-4,
              patience=10, launches_per_poll=32, max_launches=10_000_000, poll_every=256, stream=None):
        """The search of svm_solve for every instance, on the device. Returns
        (reports: structured numpy array of pdscp_report, directions: list of
        float32 arrays, launches run)."""
        o = _options(eps, mode, max_iters, poll_every, max_steps, eta, delta, patience)
        lib = load()
        check(lib.svm_batch_solve_init(self.num, _vp(self.pts), self.dt, *self._tables(), ctypes.byref(o),
                                       _vp(self.ws), self.ws.numel(), _stream(stream)), "svm_batch_solve_init")
        launches, done = ctypes.c_int64(), ctypes.c_int32()
        check(lib.svm_batch_solve_run(self.num, _vp(self.pts), _vp(self.labels), _vp(self.ws), self.ws.numel(),
                                      launches_per_poll, max_launches, _stream(stream), ctypes.byref(launches),
                                      ctypes.byref(done)), "svm_batch_solve_run")
        reps = torch.zeros((self.num, ctypes.sizeof(_ffi.Report)), dtype=torch.uint8, device=self.pts.device)
        w = torch.empty(int(self.d.sum()), dtype=torch.float32, device=self.pts.device)
        check(lib.svm_batch_solve_read(self.num, _vp(self.ws), float(eps), _vp(reps), _vp(w), _stream(stream)),
              "svm_batch_solve_read")
        torch.cuda.synchronize()
        rec = np.frombuffer(reps.cpu().numpy().tobytes(), dtype=REPORT_DTYPE)
        cut = np.concatenate([[0], np.cumsum(self.d)])
        wh = w.cpu().numpy()
        return rec, [wh[cut[i]:cut[i + 1]] for i in range(self.num)], launches.value
