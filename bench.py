"""Benchmark of the MWU hot path on one GB300 (or N replicas under torchrun).

A step is one MWU iteration of the alpha-FTP (one launch of the iteration
kernel: the SOC exponential of every cone, the trace normaliser, the weighted
n x d reduction, the closed-form ORACLE and the running-mean update) over the
SES workload n = 1,000,000 points i.i.d. N(0, I_32), float32, seed 0, at
alpha = D (an upper bound on OPT, so the ORACLE never separates and every step
does the full work) with the step size Theorem 2 gives the first search step.

The steps run as a solve runs them: launched back to back (mwu_run, one
iteration per call, consecutive launches overlapping by programmatic dependent
launch), the K timed steps bracketed by one pair of CUDA events. The input
(128 MB) is smaller than L2, so the steps rotate over 4 copies of the point
set (512 MB): between two uses of a copy 384 MB of other points stream through
the 126 MB L2, and no step finds its points there. The same iteration launched
alone after an L2 flush, each launch between its own events, is reported
beside it (variants.ses_single_launch_l2_flushed).

Prints one JSON line. `--impl reference` times the FP64 oracle (the CPU
reference of this method) on the host cores instead.
"""

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import time

os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SES/SVM time-to-(1+ε) & MWU iters/s vs plain FP32 on GB300; % of HBM roofline"
UNIT = "MWU iters/s"
N_POINTS, DIM, SEED = 1_000_000, 32, 0
WORKLOAD = "SES n=1e6 d=32 N(0,I) fp32 seed 0, one MWU iteration per step at alpha=D"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


def theorem_eta_ses(D, n, alpha, eps_i):
    T = math.ceil(36.0 * D * D * math.log(2 * n - 2) / (eps_i * eps_i * alpha * alpha))
    return math.sqrt(math.log(2 * n - 2) / T), T


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        import tempfile
        self.path = os.path.join(os.environ.get("PDSCP_CLOCKS_DIR", tempfile.gettempdir()), f"clocks_gpu{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names[1:], parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


L2_FLUSH_NOTE = "flushed between timed steps (512 MB write, then 256 MB read) outside the events"
L2_NOTE = ("inputs larger than L2: 4 copies of the 128 MB point set (512 MB) used in rotation, so no step finds "
           "its points in L2; the K steps are launched back to back (dependent-launch overlap, as the solves run "
           "them) and timed together with CUDA events")


def rotation_note(R, nbytes):
    return (f"inputs larger than L2: {R} copies of the {nbytes / 1e6:.0f} MB point set ({R * nbytes / 1e6:.0f} MB) "
            "used in rotation, so no step finds its points in L2; the K steps are launched back to back "
            "(dependent-launch overlap, as the solves run them) and timed together with CUDA events")


def ses_params(V32):
    """The benchmark iteration's parameters, computed the same way in both
    arms from the float32 points: D = max_i ||v_1 - v_i|| (Sec. 4.1, points),
    rho = 3D/sqrt2, alpha = D (an upper bound on OPT: the ORACLE never
    separates) and the Theorem 2 step size of the first search step
    (alpha_1 = 2D/3, eps_1 = 1/4). Returns (D, rho, alpha, eta, T1)."""
    V = V32.astype(np.float64)
    D = float(np.max(np.linalg.norm(V[1:] - V[0], axis=1)))
    rho = 3.0 * D / math.sqrt(2.0)
    eta, T1 = theorem_eta_ses(D, V.shape[0], 2.0 * D / 3.0, 0.25)
    return D, rho, D, eta, T1


def arm_config(alpha, eta, eor, T1, world):
    """The benchmark configuration, identical in both arms: the SES workload at
    alpha = D with the first search step's Theorem 2 step size, one replica
    per rank."""
    return {"workload": WORKLOAD, "n": N_POINTS, "d": DIM, "alpha": alpha, "eta": eta, "eta_over_rho": eor,
            "theorem_T1": T1, "l2": L2_NOTE, "parallelism": "replicas" if world > 1 else "single"}


# ------------------------------------------------------------- oracle timing
def oracle_rate(V64, alpha, eta, rho, budget_s, max_steps=None):
    """Iterations per second of the FP64 oracle on the rows of V64, timed on
    the host. Runs steps until budget_s seconds (at least one)."""
    from oracle import ses as oses
    ubar = V64[0].copy()
    t, t0 = 0, time.perf_counter()
    while True:
        rec = oses.ses_step(V64, None, ubar, t, alpha, eta, rho)
        ubar = rec["ubar_next"]
        t += 1
        el = time.perf_counter() - t0
        if el >= budget_s or (max_steps is not None and t >= max_steps):
            return t / el, t, el


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2405_09157_gb300 import datagen
    from oracle import ses as oses
    V32 = datagen.ses_gaussian(N_POINTS, DIM, SEED)
    D, rho, alpha, eta, T1 = ses_params(V32)  # the GPU arm's iteration
    V = V32.astype(np.float64)
    # size each step's row sample so the whole K+W run stays within ~2 minutes
    probe_rows = 100_000
    r_probe, _, _ = oracle_rate(V[:probe_rows], alpha, eta, rho, 1.0, max_steps=3)
    per_row = 1.0 / (r_probe * probe_rows)
    total_steps = args.steps + args.warmup
    rows = int(min(N_POINTS, max(10_000, 120.0 / (total_steps * per_row))))
    Vs = V[:rows]
    ubar = Vs[0].copy()
    for t in range(args.warmup):
        ubar = oses.ses_step(Vs, None, ubar, t, alpha, eta, rho)["ubar_next"]
    t0 = time.perf_counter()
    for t in range(args.warmup, args.warmup + args.steps):
        ubar = oses.ses_step(Vs, None, ubar, t, alpha, eta, rho)["ubar_next"]
    el = time.perf_counter() - t0
    ms_per_step = 1e3 * el / args.steps
    value = (rows / N_POINTS) * args.steps / el  # full-workload iterations per second
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": arm_config(alpha, eta, eta / rho, T1, args.gpus),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": (f"each step: one FP64 oracle iteration over the first {rows} of the {N_POINTS} "
                                    f"rows (1 thread); iterations per second extrapolated to all rows by the "
                                    f"factor rows/n = {rows / N_POINTS:.4g} (the iteration is linear in n)"),
                         "host": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------------ our arm
def aggregate_timing(local_ms, steps, world, device):
    """Whole-job timing over ranks: the slowest rank's time for `steps` steps
    decides (MAX all-reduce); every rank processed `steps` iterations of its
    own replica, so the job's throughput is world * steps / max time.
    Returns (ms_per_step, iterations per second)."""
    tot_ms = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([tot_ms], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        tot_ms = float(tt.item())
    return tot_ms / steps, world * steps / (tot_ms / 1e3)


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2405_09157_gb300 import _ffi, api, datagen

    n, d = args.n, args.d
    tdt = torch.bfloat16 if args.dtype == "bf16" else torch.float32
    ebytes = 2 if args.dtype == "bf16" else 4
    shard = args.shard == "rows"
    if shard and args.problem != "ses":
        raise SystemExit("--shard rows is built for SES")
    if args.problem == "ses" and shard:
        # one instance, its rows split over the ranks (rank 0's shard starts with v_1)
        V32 = datagen.ses_gaussian(n, d, SEED)
        full = torch.from_numpy(V32).to(dev).to(tdt)
        D = float(api.bounds(_ffi.SES, full).item())
        lo, hi = api.shard_rows(n, world, rank)
        pts = full[lo:hi].contiguous()
        first = full[0].contiguous()
        del full
        m = api.ShardedMWU(_ffi.SES, pts, first, rank, world)
    elif args.problem == "ses":
        V32 = datagen.ses_gaussian(n, d, SEED + rank)
        pts = torch.from_numpy(V32).to(dev).to(tdt)
        m = api.MWU(_ffi.SES, pts)
    if args.problem == "ses":
        D, rho, alpha, eta, T1 = ses_params(V32)
        alg_bytes = n * d * ebytes
        label_D = 0.0
    else:
        V32, y = datagen.svm_clusters(n // 2, n - n // 2, d, seed=SEED + rank)
        pts = torch.from_numpy(V32).to(dev).to(tdt)
        m = api.MWU(_ffi.SVM, pts, labels=torch.from_numpy(y).to(dev))
        D = float(api.bounds(_ffi.SVM, pts).item())
        rho = 2.0 * D
        a1 = 4.0 * D / 3.0
        T1 = math.ceil(64.0 * D * D * math.log(n) / (0.25 * a1 * a1))
        eta = math.sqrt(math.log(n) / T1)
        alpha = 0.2  # <= the margin the 0.1 band guarantees: never separates
        alg_bytes = n * d * ebytes + n
        label_D = D
    eor = eta / rho
    default_workload = (args.problem == "ses" and n == N_POINTS and d == DIM and args.dtype == "f32" and not shard)
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    flush = L2Flush(dev, l2)
    stream = torch.cuda.current_stream()
    out = api.new_steps(1, dev)

    if shard:
        # one instance over the ranks: each step is a pass, an all-gather and a
        # finish, timed alone after an L2 flush
        def step(i):
            flush()
            starts[i].record(stream)
            m.step(alpha, eor, out=out[0])
            ends[i].record(stream)
        l2_note = L2_FLUSH_NOTE
    else:
        # R copies of the points, used in rotation: between two uses of a copy
        # at least 3 L2 sizes of other points stream through L2, so no step
        # finds its points there; the steps are launched back to back with the
        # dependent-launch overlap of the solves (mwu_run, one iteration each)
        R = max(2, math.ceil(4 * l2 / (n * d * ebytes)))
        copies = [m.pts] + [m.pts.clone() for _ in range(R - 1)]
        lab = m.labels

        def step(i):
            api.mwu_run(m.problem, copies[i % R], alpha, eor, 1, m.state, m.ws, out=out[0], D=label_D,
                        labels=lab)
        l2_note = rotation_note(R, n * d * ebytes)

    clocks = ClockSampler(local)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for i in range(args.warmup):
        if shard:
            step(i % args.steps)
        else:
            step(i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    if shard:
        for i in range(args.steps):
            step(i)
    else:
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(args.steps):
            step(args.warmup + i)
        t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    clk = clocks.stop()
    total_ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends)) if shard else t0.elapsed_time(t1)
    ms_per_step, value = aggregate_timing(total_ms, args.steps, world, dev)
    if shard:  # one instance over all ranks: its iterations per second, not the ranks' sum
        value = 1e3 / ms_per_step
    rec = api.decode_steps(out)[0]
    if int(rec["t"]) != args.warmup + args.steps or int(rec["status"]) != 0:
        raise RuntimeError(f"not every timed step ran the full iteration: t={int(rec['t'])}, "
                           f"status={int(rec['status'])}")

    # roofline of the dominant (only) kernel: algorithmic bytes = n d (element bytes)
    peak, peak_kind = peaks()
    achieved = alg_bytes / (ms_per_step * 1e-3) / 1e9
    traffic = None
    prof = os.path.join(ROOT, "profiles", "ses_iter_n1e6_d32_traffic.txt")
    if default_workload and os.path.exists(prof):
        try:
            kv = {}
            with open(prof) as f:
                for line in f:
                    if ":" in line and not line.startswith("#"):
                        k, v = line.split(":", 1)
                        kv[k.strip()] = v.strip()
            if kv.get("kernel_rev") == kernel_rev():
                traffic = int(kv["dram_bytes_per_launch"])
        except Exception:
            traffic = None

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "strong" if shard else "weak",
        "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": (arm_config(alpha, eta, eor, T1, world) if default_workload else
                   {"workload": f"{args.problem.upper()} n={n} d={d} {args.dtype} (non-default case)",
                    "n": n, "d": d, "alpha": alpha, "eta": eta, "eta_over_rho": eor, "theorem_T1": T1,
                    "l2": l2_note, "parallelism": ("rows" if shard else "replicas") if world > 1 else "single"}),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)",
                     "alg_bytes_per_launch": alg_bytes},
        "gpu_launches": args.steps * (2 if shard else 1),
        "clocks": clk,
        "wall_ms_per_step_incl_flush": 1e3 * wall / args.steps,
        "last_step": {"t": int(rec["t"]), "oracle_value": float(rec["oracle_value"]),
                      "objective": float(rec["objective"]), "status": int(rec["status"])},
    }
    if rank == 0 and not args.skip_extras and default_workload:
        result["e2e"] = e2e_host(args, V32, alpha, eor, dev)
        result["cpu_baseline"] = cpu_baseline(V32, alpha, eta, rho)
        result["variants"] = variants(dev, flush)
        result["variants"]["ses_single_launch_l2_flushed"] = single_launch_variant(m, alpha, eor, flush, alg_bytes)
        result["variants"]["batched_ses_4096"] = batched_variant(dev)
        result["variants"]["ses_backward_n1e5_d64_T2000"] = backward_variant(dev)
        result["variants"]["ses_multi_candidate_n1e6_d32"] = multi_variant(dev, flush)
        result["variants"]["batched_ses_4096_search"] = batched_solve_variant(dev)
        result["variants"]["batched_svm_512"] = batched_svm_variant(dev)
        result["time_to_eps"] = time_to_eps(pts)
        result["variants"]["svm_time_to_eps_n1e6_d128"] = svm_time_to_eps(dev)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result))


def single_launch_variant(m, alpha, eor, flush, alg_bytes, K=300):
    """The same iteration as one mwu_step launch timed alone (CUDA events
    around it) after an L2 flush: the launch and event overhead of a lone
    kernel (about 5 us on this GPU for an empty one) is inside this figure."""
    m.init()  # a fresh alpha-FTP: _time_steps checks t from 0
    ms = _time_steps(m, alpha, eor, 0.0, flush, K=K)
    peak, _ = peaks()
    return {"ms_per_step": ms, "iters_per_s": 1e3 / ms, "frac_hbm": alg_bytes / (ms * 1e-3) / 1e9 / peak,
            "timing": "one mwu_step per step, L2 flushed before it, CUDA events around the launch", "steps": K}


class L2Flush:
    """Evicts L2 between timed steps: writes a buffer of 4x L2 (at least
    512 MB), then reads half of it, so L2 ends up holding clean lines."""

    def __init__(self, dev, l2_bytes):
        import torch
        self.buf = torch.empty(max(4 * l2_bytes, 512 << 20) // 4, dtype=torch.float32, device=dev)
        self.half = self.buf[: self.buf.numel() // 2]
        self.device = dev

    def __call__(self):
        self.buf.zero_()
        self.sink = self.half.sum()


KERNEL_FILES = ("common.cuh", "dispatch.cuh", "ses_kernel.cuh", "kern_ses.cu")


def kernel_rev():
    """Hash of the sources of the SES iteration kernel: a stored ncu traffic
    figure is used only for the kernel revision it was measured on."""
    import hashlib
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2405_09157_gb300", "csrc")
    for name in KERNEL_FILES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def e2e_host(args, V32, alpha, eor, dev):
    """Same metric through the public API with host buffers: every step copies
    the points from pinned host memory to the device, runs the iteration and
    reads the step record back. Two device buffers let the copy of step k + 1
    (on a second stream) run while step k computes; a buffer is refilled only
    after the step that read it, and a step starts only after its copy. The
    timed region starts before the first copy and ends after the last record
    read."""
    import torch
    from paper_2405_09157_gb300 import _ffi, api
    host = torch.from_numpy(V32).pin_memory()
    bufs = [torch.empty_like(host, device=dev) for _ in range(2)]
    bufs[0].copy_(host)
    m = api.MWU(_ffi.SES, bufs[0])
    out = api.new_steps(1, dev)
    rec_host = torch.empty((1, api.STEP_BYTES), dtype=torch.uint8).pin_memory()
    comp = torch.cuda.current_stream()
    cs = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    used = [torch.cuda.Event(), torch.cuda.Event()]

    def run(K, start=None):
        if start is not None:
            cs.wait_event(start)
        with torch.cuda.stream(cs):
            bufs[0].copy_(host, non_blocking=True)
            copied[0].record(cs)
        for k in range(K):
            b = k % 2
            if k + 1 < K:  # the next step's inputs, into the other buffer once its last reader is done
                with torch.cuda.stream(cs):
                    if k >= 1:
                        cs.wait_event(used[1 - b])
                    bufs[1 - b].copy_(host, non_blocking=True)
                    copied[1 - b].record(cs)
            comp.wait_event(copied[b])
            api.mwu_step(_ffi.SES, bufs[b], alpha, eor, m.state, m.ws, out[0])
            used[b].record(comp)
            rec_host.copy_(out, non_blocking=True)

    K = max(10, min(args.steps, 200))
    run(3)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(comp)
    run(K, start=s)
    e.record(comp)
    torch.cuda.synchronize()
    ms = s.elapsed_time(e) / K
    return {"value": 1e3 / ms, "unit": UNIT, "h2d_bytes_per_step": int(V32.nbytes),
            "d2h_bytes_per_step": api.STEP_BYTES, "ms_per_step": ms, "steps": K,
            "copy": "two device buffers: step k+1's host-to-device copy overlaps step k"}


def host_cpu():
    """The host's processor model and logical CPU count (for the CPU baseline's context)."""
    model = platform.processor() or platform.machine()
    parts = {"0xd4f": "Arm Neoverse-V2 (NVIDIA Grace)", "0xd40": "Arm Neoverse-V1", "0xd0c": "Arm Neoverse-N1"}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
                if key == "cpu part":
                    part = line.split(":", 1)[1].strip().lower()
                    model = parts.get(part, f"Arm CPU part {part}")
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu": model, "arch": platform.machine()}


def cpu_baseline(V32, alpha, eta, rho):
    V64 = V32.astype(np.float64)
    rate, steps, el = oracle_rate(V64, alpha, eta, rho, budget_s=15.0)
    return {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} oracle iterations over all {V32.shape[0]} points ({el:.1f} s), FP64 numpy, 1 thread",
            "host": host_cpu(), "all_cores": oracle_all_cores()}


def oracle_all_cores(budget_s=10.0):
    """The same oracle iterations with numpy's thread pools opened to every
    host core (the thread counts must be set before numpy loads, so this runs
    in a child process). The oracle is numpy elementwise work and reductions,
    which run on one thread whatever the setting; only its BLAS products can
    use more. Returns the rate and the thread count offered."""
    cores = os.cpu_count() or 1
    env = dict(os.environ, OMP_NUM_THREADS=str(cores), OPENBLAS_NUM_THREADS=str(cores),
               MKL_NUM_THREADS=str(cores))
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-rate-child", str(budget_s)],
                           env=env, capture_output=True, text=True, timeout=120 + 3 * budget_s)
        v = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as e:  # reported, never fatal for the line
        return {"error": f"{type(e).__name__}: {e}"[:200], "cores": cores}
    return {"value": v["rate"], "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{v['steps']} oracle iterations over all {N_POINTS} points ({v['seconds']:.1f} s), "
                      f"numpy thread pools set to {cores} threads"}


def oracle_rate_child(budget_s):
    from paper_2405_09157_gb300 import datagen
    V32 = datagen.ses_gaussian(N_POINTS, DIM, SEED)
    D, rho, alpha, eta, _ = ses_params(V32)
    rate, steps, el = oracle_rate(V32.astype(np.float64), alpha, eta, rho, budget_s=budget_s)
    print(json.dumps({"rate": rate, "steps": steps, "seconds": el}))


def _time_steps(m, alpha, eor, D, flush, K=50):
    import torch
    from paper_2405_09157_gb300 import api
    s = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    e = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    out = api.new_steps(1, flush.device)
    for i in range(K + 5):
        flush()
        if i >= 5:
            s[i - 5].record()
        m.step(alpha, eor, out=out[0], D=D)
        if i >= 5:
            e[i - 5].record()
    torch.cuda.synchronize()
    if int(api.decode_steps(out)[0]["t"]) != K + 5:
        raise RuntimeError("a timed variant step did not run the full iteration")
    return sum(a.elapsed_time(b) for a, b in zip(s, e)) / K


def _back_to_back(problem, pts, alpha, eor, D=0.0, labels=None, K=300, W=20):
    """ms per iteration of K iterations launched back to back as the main
    line times them (mwu_run, one iteration per call, dependent-launch
    overlap) over copies of the points used in rotation (together at least
    four L2 sizes, so no iteration finds its points in L2); one event pair."""
    import torch
    from paper_2405_09157_gb300 import api
    l2 = torch.cuda.get_device_properties(pts.device).L2_cache_size
    nbytes = pts.numel() * pts.element_size()
    R = max(2, math.ceil(4 * l2 / nbytes))
    copies = [pts] + [pts.clone() for _ in range(R - 1)]
    m = api.MWU(problem, pts, labels=labels)
    out = api.new_steps(1, pts.device)
    for i in range(W):
        api.mwu_run(problem, copies[i % R], alpha, eor, 1, m.state, m.ws, out=out, D=D, labels=labels)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for i in range(K):
        api.mwu_run(problem, copies[(W + i) % R], alpha, eor, 1, m.state, m.ws, out=out, D=D, labels=labels)
    e1.record()
    torch.cuda.synchronize()
    rec = api.decode_steps(out)[0]
    if int(rec["t"]) != W + K or int(rec["status"]) != 0:
        raise RuntimeError("a back-to-back variant step did not run the full iteration")
    return e0.elapsed_time(e1) / K, R


def variants(dev, flush):
    """Per-iteration time of the other hot-path forms (same timing rules)."""
    import torch
    from paper_2405_09157_gb300 import _ffi, api, datagen
    peak, _ = peaks()
    out = {}
    V32 = datagen.ses_gaussian(N_POINTS, DIM, SEED)
    pb = torch.from_numpy(V32).to(dev).to(torch.bfloat16)
    m = api.MWU(_ffi.SES, pb)
    D = float(api.bounds(_ffi.SES, pb).item())
    ms = _time_steps(m, D, 0.01 / (3 * D / math.sqrt(2)), 0.0, flush)
    b = N_POINTS * DIM * 2
    out["ses_n1e6_d32_bf16"] = {"ms_per_iter": ms, "iters_per_s": 1e3 / ms, "GBps": b / ms / 1e6,
                               "frac_hbm": b / ms / 1e6 / peak, "timing": "single launches, L2 flushed"}
    msb, R = _back_to_back(_ffi.SES, pb, D, 0.01 / (3 * D / math.sqrt(2)))
    out["ses_n1e6_d32_bf16"]["back_to_back"] = {"ms_per_iter": msb, "iters_per_s": 1e3 / msb, "frac_hbm":
                                                b / msb / 1e6 / peak, "copies_in_rotation": R}
    # the certified time to (1 + 1e-3) with the points stored in BF16 (their own, rounded, point set)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, rep = api.ses_solve(pb, eps=1e-3, mode="certified", max_iters=200_000, poll_every=256)
    out["ses_n1e6_d32_bf16"]["time_to_eps"] = {
        "seconds": time.perf_counter() - t0, "iters": rep["iters"], "radius": rep["value"],
        "lower_bound": rep["lower_bound"], "gap": rep["value"] / rep["lower_bound"] - 1, "status": rep["status"]}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, rep = api.ses_solve(pb, eps=1e-3, mode="coreset", max_iters=200_000, poll_every=256)
    out["ses_n1e6_d32_bf16"]["time_to_eps"]["coreset"] = {
        "seconds": time.perf_counter() - t0, "iters": rep["iters"], "radius": rep["value"],
        "lower_bound": rep["lower_bound"], "gap": rep["value"] / rep["lower_bound"] - 1, "status": rep["status"]}
    V4b = torch.from_numpy(datagen.ses_gaussian(4 * N_POINTS, DIM, SEED)).to(dev).to(torch.bfloat16)
    D4 = float(api.bounds(_ffi.SES, V4b).item())
    msb, R = _back_to_back(_ffi.SES, V4b, D4, 0.01 / (3 * D4 / math.sqrt(2)))
    b4 = 4 * N_POINTS * DIM * 2
    out["ses_n4e6_d32_bf16"] = {"back_to_back": {"ms_per_iter": msb, "iters_per_s": 1e3 / msb,
                                                 "frac_hbm": b4 / msb / 1e6 / peak, "copies_in_rotation": R}}
    del pb, m, V4b
    # pure HBM regime: 4e6 points (512 MB, four times L2), same iteration
    V4 = torch.from_numpy(datagen.ses_gaussian(4 * N_POINTS, DIM, SEED)).to(dev)
    m = api.MWU(_ffi.SES, V4)
    D = float(api.bounds(_ffi.SES, V4).item())
    ms = _time_steps(m, D, 0.01 / (3 * D / math.sqrt(2)), 0.0, flush)
    b = 4 * N_POINTS * DIM * 4
    out["ses_n4e6_d32_f32"] = {"ms_per_iter": ms, "iters_per_s": 1e3 / ms, "GBps": b / ms / 1e6,
                              "frac_hbm": b / ms / 1e6 / peak, "note": "512 MB of points, 4x L2: streamed from HBM"}
    # the same iterations back to back (mwu_run: dependent-launch overlap); the input exceeds L2, so no flush
    K = 50
    m.run(D, 0.01 / (3 * D / math.sqrt(2)), 3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    m.run(D, 0.01 / (3 * D / math.sqrt(2)), K)
    e1.record()
    torch.cuda.synchronize()
    msr = e0.elapsed_time(e1) / K
    out["ses_n4e6_d32_f32"]["run_back_to_back"] = {"ms_per_iter": msr, "iters_per_s": 1e3 / msr,
                                                   "GBps": b / msr / 1e6, "frac_hbm": b / msr / 1e6 / peak,
                                                   "iterations": K}
    del V4, m
    X32, y = datagen.svm_clusters(500_000, 500_000, 128, seed=0)
    X = torch.from_numpy(X32).to(dev)
    lab = torch.from_numpy(y).to(dev)
    D = float(api.bounds(_ffi.SVM, X).item())
    for name, pts, eb in (("svm_n1e6_d128_f32", X, 4), ("svm_n1e6_d128_bf16", X.to(torch.bfloat16), 2)):
        m = api.MWU(_ffi.SVM, pts, labels=lab)
        ms = _time_steps(m, 0.2, 0.01 / (2 * D), D, flush)
        b = 1_000_000 * 128 * eb + 1_000_000
        out[name] = {"ms_per_iter": ms, "iters_per_s": 1e3 / ms, "GBps": b / ms / 1e6, "frac_hbm": b / ms / 1e6 / peak,
                     "timing": "single launches, L2 flushed"}
        msb, R = _back_to_back(_ffi.SVM, pts, 0.2, 0.01 / (2 * D), D=D, labels=lab)
        out[name]["back_to_back"] = {"ms_per_iter": msb, "iters_per_s": 1e3 / msb, "frac_hbm": b / msb / 1e6 / peak,
                                     "copies_in_rotation": R}
    return out


def multi_variant(dev, flush, K=50):
    """Multi-candidate pass (ses_multi_step) on the default workload: k alpha-FTPs
    (alpha_j = (1 + 0.05 j) D, never separating) advanced by one pass over the
    1,000,000 x 32 FP32 points, k in {1, 2, 4, 8, 16} (k = 16: the tensor-core
    pass), timed as the main line (L2
    flushed between steps, CUDA events around each step). Bytes per pass are
    those of one iteration; per point the arithmetic grows k-fold."""
    import torch
    from paper_2405_09157_gb300 import _ffi, api, datagen
    peak, _ = peaks()
    V32 = datagen.ses_gaussian(N_POINTS, DIM, SEED)
    pts = torch.from_numpy(V32).to(dev)
    D = float(api.bounds(_ffi.SES, pts).item())
    eor = 0.01 / (3 * D / math.sqrt(2))
    res = {}
    for k in (1, 2, 4, 8, 16):  # k = 16: the tensor-core pass
        m = api.MultiMWU(pts, k)
        a = torch.tensor([(1.0 + 0.05 * j) * D for j in range(k)], dtype=torch.float64, device=dev)
        e = torch.full((k,), eor, dtype=torch.float64, device=dev)
        out = api.new_steps(k, dev)
        s0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        s1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        for i in range(K + 5):
            flush()
            if i >= 5:
                s0[i - 5].record()
            m.step(a, e, out=out)
            if i >= 5:
                s1[i - 5].record()
        torch.cuda.synchronize()
        rec = api.decode_steps(out)
        if not np.all(rec["t"] == K + 5):
            raise RuntimeError("a multi-candidate step did not advance every candidate")
        ms = sum(x.elapsed_time(y) for x, y in zip(s0, s1)) / K
        b = N_POINTS * DIM * 4
        res[f"k{k}"] = {"ms_per_pass": ms, "candidate_iters_per_s": k * 1e3 / ms, "GBps": b / ms / 1e6,
                        "frac_hbm": b / ms / 1e6 / peak, "tensor_cores": k == 16}
    return res


def batched_inputs(dev, num=4096):
    """The batched SES workload on the device: sizes from the seeded generator
    (n log-uniform in [100, 1e5], d in {2,3,8,16,32,64}, scale U[0.1, 10]),
    N(0, I) points from a seeded device RNG times the instance's scale, each
    instance starting on a 16-byte boundary."""
    import torch
    from paper_2405_09157_gb300 import datagen
    n, d, scale = datagen.batched_ses_sizes(num, seed=0)
    sizes = n * d
    offs = np.zeros(len(n), dtype=np.int64)
    pos = 0
    for i, sz in enumerate(sizes):
        pos = (pos + 3) & ~3
        offs[i] = pos
        pos += int(sz)
    g = torch.Generator(device=dev)
    g.manual_seed(0)
    pts = torch.randn(pos, generator=g, device=dev, dtype=torch.float32)
    elem_scale = torch.zeros(pos, dtype=torch.float32, device=dev)
    for i in range(len(n)):  # per-instance scale (padding stays scaled by 0)
        elem_scale[offs[i]:offs[i] + sizes[i]] = float(scale[i])
    pts.mul_(elem_scale)
    del elem_scale
    return pts, offs, n, d, scale


def batched_svm_inputs(dev, num=512):
    """The batched SVM workload on the device: sizes from the seeded generator
    (n log-uniform in [100, 1e5], d in {2,3,8,16,32,64}, scale U[0.1, 10],
    numpy PCG64 seed 1); per instance, class P the first floor(n/2) rows,
    points N(+-mu, I) with ||mu|| = 3 along a random unit direction, each
    point's component along it clamped to at least 0.1 on its class's side
    (separable), times the scale; a seeded device RNG draws the points."""
    import torch
    from paper_2405_09157_gb300 import api, datagen
    n, d, scale = datagen.batched_ses_sizes(num, seed=1)
    offs = np.zeros(len(n), dtype=np.int64)
    pos = 0
    for i in range(len(n)):
        pos = (pos + 3) & ~3
        offs[i] = pos
        pos += int(n[i] * d[i])
    g = torch.Generator(device=dev)
    g.manual_seed(1)
    pts = torch.zeros(pos, dtype=torch.float32, device=dev)
    ys = []
    for i in range(len(n)):
        ni, di = int(n[i]), int(d[i])
        u = torch.randn(di, generator=g, device=dev)
        u /= u.norm()
        y = torch.ones(ni, device=dev)
        y[ni // 2:] = -1.0
        x = torch.randn(ni, di, generator=g, device=dev) + 3.0 * y[:, None] * u[None, :]
        s = x @ u
        x += ((torch.clamp(y * s, min=0.1) - y * s) * y)[:, None] * u[None, :]
        pts[offs[i]:offs[i] + ni * di] = (x * float(scale[i])).reshape(-1)
        ys.append(y.to(torch.int8).cpu().numpy())
    lab, loffs = api.pack_labels(ys, device=dev)
    return pts, offs, n, d, lab, loffs


def batched_svm_variant(dev, eps=1e-2, max_iters=30_000, K=10, W=3):
    """Batched SVM: one launch advances all 512 instances by one iteration
    (per-iteration time; inputs 0.6 GB, no flush needed), and the certified
    search of svm_solve on the device for every instance beside the plain
    single-instance svm_solve on a seeded sample of 32 instances."""
    import torch
    from paper_2405_09157_gb300 import api
    pts, offs, n, d, lab, loffs = batched_svm_inputs(dev)
    batch = api.SvmBatch(pts, offs, n, d, lab, loffs, tile_rows=4096)
    _, _, D = batch.read()
    # alpha below every instance's OPT (>= 0.2 scale against D <= ~12 scale): Claim 8 keeps the
    # ORACLE from failing, so every launch runs every instance's full iteration
    a = torch.tensor(1e-3 * D, dtype=torch.float64, device=dev)
    e = torch.tensor(0.01 / (2.0 * D), dtype=torch.float64, device=dev)
    out = api.new_steps(len(n), dev)
    for _ in range(W):
        batch.step(a, e, out=out)
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record()
    for _ in range(K):
        batch.step(a, e, out=out)
    s1.record()
    torch.cuda.synchronize()
    ms = s0.elapsed_time(s1) / K
    rec = api.decode_steps(out)
    if not (np.all(rec["t"] == W + K) and np.all(rec["status"] == 0)):
        raise RuntimeError("a batched SVM instance did not run every iteration")
    alg = int(np.sum(n * d)) * 4 + int(np.sum(n))
    peak, _ = peaks()
    res = {"workload": f"{len(n)} SVM instances, n in [100, 1e5] log-uniform, d in {{2,3,8,16,32,64}}, fp32",
           "ms_per_iteration": ms, "instance_iters_per_s": len(n) * 1e3 / ms, "alg_bytes": alg,
           "frac_hbm": alg / (ms * 1e-3) / 1e9 / peak}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps, _, launches = batch.solve(eps=eps, mode="certified", max_iters=max_iters, poll_every=256,
                                    launches_per_poll=64)
    sec = time.perf_counter() - t0
    gap = reps["upper_bound"] / np.maximum(reps["lower_bound"], 1e-300) - 1.0
    res["search"] = {"eps": eps, "max_iters": max_iters, "seconds": sec, "launches": int(launches),
                     "instances_converged": int(np.sum(reps["status"] == 0)),
                     "iters_total": int(reps["iters"].sum()), "certificate_gap_median": float(np.median(gap)),
                     "certificate_gap_max": float(np.max(gap))}
    S = 32
    pick = np.sort(np.random.default_rng(0).choice(len(n), size=S, replace=False))
    secs, conv = [], 0
    for i in pick:
        v = pts[int(offs[i]):int(offs[i]) + int(n[i]) * int(d[i])].view(int(n[i]), int(d[i]))
        li = lab[int(loffs[i]):int(loffs[i]) + int(n[i])]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, rep = api.svm_solve(v, li, eps=eps, mode="certified", max_iters=max_iters, poll_every=256)
        secs.append(time.perf_counter() - t0)
        conv += int(rep["status"] == 0)
    secs = np.array(secs)
    res["plain_per_instance"] = {"sample": f"{S} instances drawn uniformly (numpy PCG64 seed 0)",
                                 "seconds_sample": float(secs.sum()),
                                 "seconds_all_estimated": float(secs.mean() * len(n)),
                                 "instances_converged": conv}
    return res


def batched_solve_variant(dev, eps=1e-3, max_iters=20_000):
    """Time to solve the batched SES workload: every instance runs the search
    of Sec. 3 on the device, at eps = 1e-3 and at most max_iters MWU
    iterations per instance, after the native autotuner picked the tile size:
    under the certified mode (only proven conclusions; an instance converges
    when its ball is within 1 + eps of its certified lower bound) and under
    the paper's practical rules of Sec. 5. Wall time of each whole search,
    launches, converged instances and the certificate gaps."""
    import torch
    from paper_2405_09157_gb300 import api
    pts, offs, n, d, _ = batched_inputs(dev)
    batch = api.SesBatch(pts, offs, n, d, tile_rows=4096)
    tr, ms_launch = batch.autotune(eps=eps)
    out = {}
    for mode in ("certified", "practical"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps, _, launches = batch.solve(eps=eps, mode=mode, max_iters=max_iters, launches_per_poll=64,
                                        poll_every=256)
        sec = time.perf_counter() - t0
        gap = reps["upper_bound"] / np.maximum(reps["lower_bound"], 1e-300) - 1.0
        out[mode] = {"seconds": sec, "launches": int(launches), "instances_converged": int(np.sum(reps["status"] == 0)),
                     "iters_total": int(reps["iters"].sum()), "certificate_gap_median": float(np.median(gap)),
                     "certificate_gap_p90": float(np.quantile(gap, 0.9)), "certificate_gap_max": float(np.max(gap))}
        if mode == "certified":
            cert_reps = reps
    res = {"workload": f"{len(n)} SES instances, eps={eps}, <= {max_iters} iterations each",
           "tile_rows": int(tr), "ms_per_launch_autotune": ms_launch, "instances": int(len(n))}
    res.update(out["certified"])
    res["mode"] = "certified"
    res["practical_rules"] = out["practical"]
    res["plain_per_instance"] = plain_sample(pts, offs, n, d, cert_reps, eps, max_iters, dev)
    return res


def plain_sample(pts, offs, n, d, batch_reps, eps, max_iters, dev, S=128):
    """The same certified search run instance by instance through the plain
    single-instance path (ses_solve, mode "certified", float32) on a seeded
    uniform sample of S instances; its wall time scaled by count / S estimates
    solving all of them one after another (the instances are independent, so
    the sum of per-instance times is the plain path's total)."""
    import torch
    from paper_2405_09157_gb300 import api
    pick = np.sort(np.random.default_rng(0).choice(len(n), size=S, replace=False))
    secs, iters, conv, agree = [], [], 0, 0
    for i in pick:
        v = pts[int(offs[i]):int(offs[i]) + int(n[i]) * int(d[i])].view(int(n[i]), int(d[i]))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, rep = api.ses_solve(v, eps=eps, mode="certified", max_iters=max_iters, poll_every=256)
        secs.append(time.perf_counter() - t0)
        iters.append(rep["iters"])
        conv += int(rep["status"] == 0)
        # both certified balls lie within each other's certified interval
        agree += int(rep["lower_bound"] <= batch_reps["value"][i] * (1 + 1e-5)
                     and batch_reps["lower_bound"][i] <= rep["value"] * (1 + 1e-5))
    secs = np.array(secs)
    return {"sample": f"{S} instances drawn uniformly (numpy PCG64 seed 0) from the {len(n)}",
            "seconds_sample": float(secs.sum()), "seconds_per_instance_mean": float(secs.mean()),
            "seconds_all_estimated": float(secs.mean() * len(n)),
            "seconds_all_estimated_stderr": float(secs.std(ddof=1) / np.sqrt(S) * len(n)),
            "iters_sample": int(np.sum(iters)), "instances_converged": conv,
            "brackets_agree_with_batched": agree}


def batched_variant(dev, K=10, W=3):
    """Per-iteration time of the batched SES workload: 4096 instances, n log-uniform
    in [100, 1e5], d in {2,3,8,16,32,64}, N(0, I) points times a per-instance
    U[0.1, 10] scale (sizes from the seeded generator, points from a seeded
    device RNG); one launch advances every instance by one iteration. The input
    (about 5 GB) is far larger than L2, so no flush is needed between steps."""
    import torch
    from paper_2405_09157_gb300 import api
    pts, offs, n, d, scale = batched_inputs(dev)
    sizes = n * d
    batch = api.SesBatch(pts, offs, n, d, tile_rows=4096)
    tr, _ = batch.autotune()  # the native autotuner re-initialises the batch with the fastest tile size
    bound = 2.0 * scale * (np.sqrt(d) + 6.0)  # >= OPT with room: the ORACLE never separates
    a = torch.tensor(bound, dtype=torch.float64, device=dev)
    e = torch.tensor(0.01 / (3.0 * bound / np.sqrt(2.0)), dtype=torch.float64, device=dev)
    out = api.new_steps(len(n), dev)
    for _ in range(W):
        batch.step(a, e, out=out)
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record()
    for _ in range(K):
        batch.step(a, e, out=out)
    s1.record()
    torch.cuda.synchronize()
    ms = s0.elapsed_time(s1) / K
    rec = api.decode_steps(out)
    if not (np.all(rec["t"] == W + K) and np.all(rec["status"] == 0)):
        raise RuntimeError("a batched instance did not run every iteration")
    peak, _ = peaks()
    b = int(sizes.sum()) * 4
    return {"instances": int(len(n)), "points": int(n.sum()), "tile_rows": int(tr), "bytes_per_iter": b,
            "ms_per_iter": ms,
            "instance_iters_per_s": len(n) * 1e3 / ms, "GBps": b / ms / 1e6, "frac_hbm": b / ms / 1e6 / peak,
            "l2": "input larger than L2, no flush"}


def backward_variant(dev, n=100_000, d=64, T=2000):
    """Reverse sweep through T unrolled SES iterations (gradient of the final
    radius with respect to the points), n x d N(0, I) FP32 points at alpha = D.
    Times the whole mwu_backward call (T forward iterations recording the tape,
    then T reverse passes; consecutive passes overlap by dependent launch) with
    CUDA events, and reports it per unrolled iteration (one forward pass,
    4 n d bytes, and one reverse pass, which reads the points and reads and
    writes the n x d gradient, 12 n d bytes); at this size both (51 MB) stay
    in L2 across passes. The T single mwu_step calls of the forward alone
    (launched one by one, without the overlap) are timed for context."""
    import torch
    from paper_2405_09157_gb300 import _ffi, api, datagen
    V32 = datagen.ses_gaussian(n, d, seed=0)
    pts = torch.from_numpy(V32).to(dev)
    D = float(api.bounds(_ffi.SES, pts).item())
    rho = 3.0 * D / np.sqrt(2.0)
    eor = 0.5 / rho
    ws = torch.empty(api.backward_workspace_size(n, d, T), dtype=torch.uint8, device=dev)
    out = api.new_steps(1, dev)
    api.mwu_backward(pts, D, eor, T, ws=ws, out=out)  # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    grad, _ = api.mwu_backward(pts, D, eor, T, ws=ws, out=out)
    e1.record()
    torch.cuda.synchronize()
    total = e0.elapsed_time(e1)
    rec = api.decode_steps(out)[0]
    if not (rec["t"] == T and rec["status"] == 0):
        raise RuntimeError("the reverse sweep did not run every iteration")
    m = api.MWU(_ffi.SES, pts)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(T):
        m.step(D, eor)
    e1.record()
    torch.cuda.synchronize()
    fwd = e0.elapsed_time(e1)
    per = total / T
    b = 16 * n * d
    res = {"workload": f"SES n={n} d={d} T={T} fp32, alpha = D", "ms_total": total,
           "us_per_unrolled_iteration": 1e3 * per, "GBps_per_unrolled_iteration": b / per / 1e6,
           "ms_forward_single_steps": fwd,
           "note": "points and gradient (51 MB) are L2-resident across passes: GB/s is not an HBM figure"}
    # SVM: the margin of the minimisation alpha-FTP, two clusters as the SVM workload (n/2 per class)
    X32, y = datagen.svm_clusters(n // 2, n // 2, d, seed=0)
    X = torch.from_numpy(X32).to(dev)
    lab = torch.from_numpy(y).to(dev)
    Dv = float(api.bounds(_ffi.SVM, X).item())
    eor = 0.5 / (2.0 * Dv)
    alpha = 0.01 * Dv  # about 0.11, below OPT >= 0.2 (band 0.1 on both sides): the ORACLE never separates
    ws = torch.empty(api.backward_workspace_size(n, d, T, _ffi.SVM), dtype=torch.uint8, device=dev)
    api.mwu_backward(X, alpha, eor, T, ws=ws, out=out, problem=_ffi.SVM, labels=lab, D=Dv)  # warm-up
    torch.cuda.synchronize()
    e0.record()
    api.mwu_backward(X, alpha, eor, T, ws=ws, out=out, problem=_ffi.SVM, labels=lab, D=Dv)
    e1.record()
    torch.cuda.synchronize()
    total = e0.elapsed_time(e1)
    rec = api.decode_steps(out)[0]
    if not (rec["t"] == T and rec["status"] == 0):
        raise RuntimeError("the SVM reverse sweep did not run every iteration")
    m = api.MWU(_ffi.SVM, X, labels=lab)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(T):
        m.step(alpha, eor, D=Dv)
    e1.record()
    torch.cuda.synchronize()
    fwd = e0.elapsed_time(e1)
    per = total / T
    res["svm"] = {"workload": f"SVM n={n} d={d} T={T} fp32, alpha = 0.01 D", "ms_total": total,
                  "us_per_unrolled_iteration": 1e3 * per, "GBps_per_unrolled_iteration": (16 * n * d + 2 * n) / per / 1e6,
                  "ms_forward_single_steps": fwd}
    return res


def time_to_eps(pts):
    """Time to a certified (1+eps) ball at eps = 1e-3: ses_solve in CERTIFIED
    mode (only proven conclusions; ends when the radius of an actual
    enclosing ball is within 1 + eps of a lower bound), then the same solve
    under the paper's practical rules of Sec. 5 (a stalled alpha-FTP read as
    affirmative), whose search range can close while its certificates stay
    wide, and the CORESET mode (CERTIFIED plus core-set certificates: the dual
    value of Frank-Wolfe weights on the points farthest from the running mean,
    and the ball at their barycentre). Wall time of the whole solve, bounds
    pass and polls included."""
    import torch
    from paper_2405_09157_gb300 import api
    out = {}
    for mode, budget in (("certified", 200_000), ("practical", 200_000), ("coreset", 200_000)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, rep = api.ses_solve(pts, eps=1e-3, mode=mode, max_iters=budget, poll_every=256)
        el = time.perf_counter() - t0
        out[mode] = {"seconds": el, "iters": rep["iters"], "search_steps": rep["search_steps"],
                     "radius": rep["value"], "lower_bound": rep["lower_bound"],
                     "gap": rep["value"] / rep["lower_bound"] - 1 if rep["lower_bound"] > 0 else None,
                     "search_range": [rep["search_L"], rep["search_U"]], "status": rep["status"],
                     "budget_iters": budget}
    res = dict(out["coreset"])
    res["eps"] = 1e-3
    res["mode"] = "coreset (certified search plus core-set certificates; eta starts at 1)"
    res["certified_mwu_only"] = out["certified"]
    res["practical_rules"] = out["practical"]
    res["note"] = ("gap = radius of the returned ball / certified lower bound - 1 (<= eps: done); "
                   "status 5 = budget spent; the top-level figures are the search with core-set "
                   "certificates (the fastest certified solve), 'certified_mwu_only' the same search "
                   "with the MWU's own certificates only")
    return res


def svm_time_to_eps(dev):
    """svm_solve on the n = 1e6, d = 128 SVM workload at eps = 1e-3: wall time
    to a certified (1 - eps) margin with the core-set certificates (mode
    "coreset"), FP32 and BF16 points, and the MWU-only certified search within
    30,000 iterations for comparison (the margin of an actual direction, the
    best upper bound reached)."""
    import torch
    from paper_2405_09157_gb300 import api, datagen
    X32, y = datagen.svm_clusters(500_000, 500_000, 128, seed=0)
    X = torch.from_numpy(X32).to(dev)
    lab = torch.from_numpy(y).to(dev)
    out = {"workload": "SVM n=1e6 (5e5 + 5e5) d=128, eps = 1e-3"}
    for name, pts, mode, budget in (("coreset_f32", X, "coreset", 200_000),
                                    ("coreset_bf16", X.to(torch.bfloat16), "coreset", 200_000),
                                    ("certified_mwu_only_f32", X, "certified", 30_000)):
        ws = api.workspace(api.SVM, pts.shape[0], pts.shape[1], dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, rep = api.svm_solve(pts, lab, eps=1e-3, mode=mode, max_iters=budget, poll_every=256, ws=ws)
        el = time.perf_counter() - t0
        out[name] = {"seconds": el, "iters": rep["iters"], "margin": rep["value"],
                     "upper_bound": rep["upper_bound"],
                     "gap": rep["upper_bound"] / rep["value"] - 1 if rep["value"] > 0 else None,
                     "status": rep["status"], "budget_iters": budget}
    out["note"] = ("gap = certified upper bound / margin of the returned direction - 1 (<= eps: done); "
                   "status 5 = budget spent; seconds include the core-set checks' host solves")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-extras", action="store_true", help="only the timed steps (for profiling)")
    ap.add_argument("--problem", default="ses", choices=["ses", "svm"], help="non-default cases: profiling only")
    ap.add_argument("--n", type=int, default=N_POINTS)
    ap.add_argument("--d", type=int, default=DIM)
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16"])
    ap.add_argument("--shard", default="replicas", choices=["replicas", "rows"],
                    help="N > 1: independent replicas (default) or one instance with its rows split over the GPUs")
    ap.add_argument("--oracle-rate-child", type=float, default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_rate_child is not None:
        oracle_rate_child(args.oracle_rate_child)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
