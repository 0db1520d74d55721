"""Benchmark: CSR SpMV by speculative segmented sum on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload stencil160|rmat22|batch512|...] [--precision f64|f32|bf16]
                    [--tile-w 0] [--tile-s 0] [--variant 0] [--e2e-steps 10]

--precision f32/bf16 times ssspmv_csr_f32 / ssspmv_csr_bf16f32 on the workload
and the plain FP64 call beside it; --workload batch<count> times the batched
FP32 call over a seeded mixed batch as one CUDA-graph replay, beside the same
matrices as separate FP32 calls and separate plain FP64 calls.

A step is one full y = A x through ssspmv_csr_f64 (kernels (a) partition,
(b) segmented sum, (c) calibration) on the synthetic 27-point stencil over a
160^3 grid in FP64 (m = 4,096,000, nnz = 109,215,352), inputs resident in
HBM.  L2 is flushed (a 512 MB write, then a read) between timed steps, outside the timed
events.  value = algorithmic bytes / time, bytes = nnz*(8+4) + (m+1)*4 +
m*8 + n*8 (x read once), in GB/s.  Under torchrun each rank runs an
independent replica (the path needs no exchange); value sums all ranks'
bytes over the slowest rank's time.

--impl reference times the CPU oracle (rows split over OpenMP threads, the
paper's CPU row-block method) on this machine's host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SpMV effective GB/s & % of HBM peak vs plain FP64 kernel, at stated error"
FALLBACK_HBM_GBS = 6800.0


def algorithmic_bytes(m: int, n: int, nnz: int, val_bytes: int = 8, idx_bytes: int = 4,
                      y_bytes: int = 8, x_bytes: int = 8) -> int:
    """nnz*(val+idx) + (m+1)*idx + m*y + n*x (x counted once)."""
    return nnz * (val_bytes + idx_bytes) + (m + 1) * idx_bytes + m * y_bytes + n * x_bytes


def paper_bytes(m: int, nnz: int, val_bytes: int = 8, idx_bytes: int = 4) -> int:
    """The paper's bandwidth numerator (Sec. 4.3): (m+1+nnz)*idx + (2nnz+m)*val."""
    return (m + 1 + nnz) * idx_bytes + (2 * nnz + m) * val_bytes


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


# the sources that define kernel (b) and its launch (device code, tile shape,
# workspace carve-up, block shape); host-only files do not change its traffic
KERNEL_B_SOURCES = ("layout.h", "launch.cuh", "ptx.cuh", "segsum.cuh", "spmv_f64.cu")


def source_digest() -> str:
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1504_06474_gb300", "csrc")
    for name in KERNEL_B_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` from profiles/traffic.json, only if it
    was captured from the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    for rec in d.get("records", []):
        if (rec.get("kernel") == kernel and rec.get("workload") == workload
                and rec.get("source_digest") == source_digest()):
            return rec.get("dram_bytes_per_launch")
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = open(os.devnull, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "samples": 0}
        self.proc.terminate()
        try:
            text, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            text, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in text.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(v: float, device=None) -> float:
    """The largest v over the ranks of the process group (every rank calls
    it, and every rank gets the maximum); v itself without a group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return v
    t = torch.tensor([v], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(bytes_per_step: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job GB/s of `world` replicas that each did `steps` products of
    `bytes_per_step` in at most `seconds` (the slowest rank's time)."""
    return bytes_per_step * steps * world / seconds / 1e9


def cpu_oracle_rate(A, x, budget_s: float, max_reps: int = 1000):
    """Times the oracle's OpenMP row loop over the whole matrix, repeated until
    budget_s of CPU time has been spent.  Returns (GB/s, threads, reps, s)."""
    import numpy as np

    import oracle
    y = np.empty(A.m)
    oracle.spmv_omp(A.row_ptr, A.col, A.val, x, y=y)  # warm caches and threads
    reps, used, t0 = 0, 1, time.perf_counter()
    while reps < max_reps:
        _, used = oracle.spmv_omp(A.row_ptr, A.col, A.val, x, y=y)
        reps += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    nbytes = algorithmic_bytes(A.m, A.n, A.nnz)
    return nbytes * reps / dt / 1e9, used, reps, dt


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import synth
    import oracle
    oracle.build()
    A, x = synth.workload(args.workload)
    rate_w, used, reps, _ = cpu_oracle_rate(A, x, budget_s=1.0, max_reps=max(1, args.warmup))
    import numpy as np
    y = np.empty(A.m)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, used = oracle.spmv_omp(A.row_ptr, A.col, A.val, x, y=y)
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    nbytes = algorithmic_bytes(A.m, A.n, A.nnz)
    value = nbytes / t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(t * 1e3, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "m": A.m, "n": A.n, "nnz": A.nnz,
                   "bytes_per_step": nbytes},
        "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": used,
                         "kind": "oracle",
                         "sample": "the whole %s SpMV per step (oracle row loop, rows split "
                                   "over %d OpenMP threads)" % (args.workload, used)},
        "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import synth
    from paper_1504_06474_gb300 import _build, api
    from paper_1504_06474_gb300 import ssspmv as C
    if rank == 0 or world == 1:
        _build.build()
    if world > 1:
        dist.barrier()

    A, x = synth.workload(args.workload)
    Ad = api.to_device(A.row_ptr, A.col, A.val, A.n, dev)
    xd = torch.as_tensor(x, device=dev)
    y = torch.empty(A.m, dtype=torch.float64, device=dev)
    selected = None
    if args.select:
        # the shipped network's class for this matrix, from its device features
        from paper_1504_06474_gb300 import selector as SEL
        params = SEL.load_default()
        if params is None:
            raise RuntimeError("no selector weights shipped with the package")
        f = SEL.device_features(Ad.row_ptr, A.m, A.n, A.nnz).cpu().numpy()[None, :]
        k = int(SEL.select(params, f, dev)[0])
        kw = SEL.CLASSES[k][1]
        args.tile_w, args.variant = kw.get("W", 0), kw.get("variant", 0)
        args.block_warps = kw.get("block_warps", 0)
        selected = {"class": SEL.CLASSES[k][0], "index": k}

    def mk(timer=None, W=None, variant=None, block_warps=None):
        return C.make_opts(W=args.tile_w if W is None else W, S=args.tile_s, timer=timer,
                           variant=args.variant if variant is None else variant,
                           block_warps=args.block_warps if block_warps is None else block_warps)
    rows_variant = args.variant == C.VARIANT_ROWS
    shape = C.ssspmv_plan_shape(A.m, A.nnz, 8, mk())
    ws = api.workspace_for(Ad, mk(), device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    sink = torch.empty(1, dtype=torch.int64, device=dev)

    def flush_l2():
        # write, then read: the read evicts the dirty lines the write left, so
        # no write-back of the flush buffer lands inside the next timed step
        if args.hot:
            return  # inputs left in L2 (only meaningful for workloads that fit)
        flush.fill_(1)
        torch.sum(flush.view(torch.int64), 0, keepdim=True, out=sink)
    stream = torch.cuda.current_stream(dev)

    def step(opts):
        rc = C.ssspmv_csr_f64(A.m, A.n, A.nnz, Ad.row_ptr, Ad.col, Ad.val, xd, y, opts=opts,
                              workspace=ws, stream=stream)
        if rc != 0:
            raise C.SsspmvError(rc, "ssspmv_csr_f64")

    plain = mk()
    for _ in range(args.warmup):
        flush_l2()
        step(plain)
    torch.cuda.synchronize(dev)

    # each step timed by events on the launching stream around the whole call
    K = args.steps
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    time.sleep(0.25)
    t_wall = time.perf_counter()
    per_step = _event_loop(lambda: step(plain), flush_l2, K, stream)        # ms
    t_wall = time.perf_counter() - t_wall
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()

    # stage breakdown: the library's own events at the kernel boundaries, in a
    # run of its own (events between the kernels keep kernels (b) and (c)
    # from starting early, so these steps are a little longer)
    Ks = min(K, 200)
    timer = C.ssspmv_timer_create(Ks)
    opts_t = mk(timer=timer)
    for k in range(Ks):
        flush_l2()
        step(opts_t)
    torch.cuda.synchronize(dev)
    times = C.ssspmv_timer_read(timer, Ks)
    C.ssspmv_timer_destroy(timer)
    assert len(times) == Ks
    part = [t[0] for t in times]                                             # ms
    seg = [t[1] for t in times]
    cal = [t[2] for t in times]
    t_total = sum(per_step) / 1e3                                            # s
    if selected is not None:
        # the default configuration on the same matrix, timed the same way
        dflt = mk(W=0, variant=0, block_warps=0)
        ws_d = api.workspace_for(Ad, dflt, device=dev)

        def step_d():
            C.check(C.ssspmv_csr_f64(A.m, A.n, A.nnz, Ad.row_ptr, Ad.col, Ad.val, xd, y,
                                     opts=dflt, workspace=ws_d, stream=stream), "default")
        for _ in range(args.warmup):
            flush_l2()
            step_d()
        d_ms = sum(_event_loop(step_d, flush_l2, Ks, stream)) / Ks
        selected["default_ms_per_step"] = round(d_ms, 5)
        selected["speedup_vs_default"] = round(d_ms / (t_total / K * 1e3), 4)
        del ws_d
        step(plain)  # y from the selected configuration again
    # plan reuse (partition once; kernels (b) and (c) per product, the
    # iterative-solver form), timed the same way beside the one-shot call,
    # with y checked against it
    plan_ms = None
    if not rows_variant and not args.select:
        y_one = y.clone()
        plan = C.ssspmv_plan_create(A.m, A.n, A.nnz, Ad.row_ptr, 8, plain, stream=stream)
        try:
            def step_p():
                C.check(C.ssspmv_plan_execute(plan, Ad.col, Ad.val, xd, y, stream=stream),
                        "ssspmv_plan_execute")
            for _ in range(args.warmup):
                flush_l2()
                step_p()
            plan_ms = sum(_event_loop(step_p, flush_l2, Ks, stream)) / Ks
            torch.cuda.synchronize(dev)
            if not torch.equal(y, y_one):
                raise RuntimeError("plan execution differs from the one-shot call")
        finally:
            C.ssspmv_plan_destroy(plan)
        del y_one
    t_total = max_over_ranks(t_total, dev)  # the slowest replica
    nbytes = algorithmic_bytes(A.m, A.n, A.nnz)
    value = replica_throughput(nbytes, K, world, t_total)
    ms_step = t_total / K * 1e3

    # end to end through the host-buffer entry point: H2D of row_ptr, col,
    # val, x from pinned memory, the product, D2H of y, every step
    e2e = None
    if args.e2e_steps > 0:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        h_rp, h_col, h_val, h_x = pin(A.row_ptr), pin(A.col), pin(A.val), pin(x)
        h_y = torch.empty(A.m, dtype=torch.float64).pin_memory()
        nbuf = C.ssspmv_host_buffer_bytes(A.m, A.n, A.nnz, plain)
        del flush
        buf = torch.empty(nbuf, dtype=torch.uint8, device=dev)
        for _ in range(2):
            C.check(C.ssspmv_csr_f64_host(A.m, A.n, A.nnz, h_rp, h_col, h_val, h_x, h_y,
                                          opts=plain, dev_buffer=buf, stream=stream),
                    "ssspmv_csr_f64_host")
        tt0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            C.check(C.ssspmv_csr_f64_host(A.m, A.n, A.nnz, h_rp, h_col, h_val, h_x, h_y,
                                          opts=plain, dev_buffer=buf, stream=stream),
                    "ssspmv_csr_f64_host")
        te = (time.perf_counter() - tt0) / args.e2e_steps
        te = max_over_ranks(te, dev)
        assert np.array_equal(h_y.numpy(), y.cpu().numpy())
        h2d = (A.m + 1) * 4 + A.nnz * 4 + A.nnz * 8 + A.n * 8
        e2e = {"value": round(nbytes * world / te / 1e9, 3), "unit": "GB/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": A.m * 8,
               "ms_per_step": round(te * 1e3, 4)}

    status = C.ssspmv_device_status(ws, stream=stream)
    if status:
        raise RuntimeError("device status bits %#x" % status)

    hbm, peak_kind = peaks()
    seg_ms = sum(seg) / Ks
    achieved = nbytes / (seg_ms / 1e3) / 1e9
    # the ncu record holds for the default configuration it was captured with
    default_cfg = (not args.select and args.tile_w in (0, 15) and args.variant == 0
                   and args.block_warps == 0 and args.tile_s in (0, 4))
    traffic = ncu_traffic("segsum_kernel", args.workload) if default_cfg else None
    line = None
    if rank == 0:
        cpu = None
        if world == 1 and args.cpu_seconds > 0:
            rate, used, reps, dt = cpu_oracle_rate(A, x, budget_s=args.cpu_seconds)
            cpu = {"value": round(rate, 3), "unit": "GB/s", "cores": used, "kind": "oracle",
                   "sample": "%d whole %s SpMVs (oracle row loop over %d OpenMP threads), "
                             "%.1f s" % (reps, args.workload, used, dt)}
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": round(ms_step, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "m": A.m, "n": A.n, "nnz": A.nnz,
                       "W": shape["W"], "L": shape["L"], "S": shape["S"],
                       "variant": ["default", "speculative", "exact", "rows"][args.variant],
                       "block_warps": args.block_warps, "selector": selected,
                       "bunches": shape["nbunches"], "bytes_per_step": nbytes,
                       "ms_per_step_median": round(statistics.median(per_step), 5),
                       "paper_bytes_per_step": paper_bytes(A.m, A.nnz),
                       "hbm_frac": round(value / world / hbm, 4),
                       "gflops": round(2.0 * A.nnz * K * world / t_total / 1e9, 3),
                       "l2": ("not flushed (hot: inputs stay in L2 between steps)" if args.hot else
                              "flushed between steps (512 MB write then read, outside the timed events)"),
                       "stage_ms": {"partition": round(sum(part) / Ks, 5),
                                    "segsum": round(seg_ms, 5),
                                    "calibrate": round(sum(cal) / Ks, 5),
                                    "steps": Ks,
                                    "whole": round(sum(t[3] for t in times) / Ks, 5)},
                       "plan_reuse": None if plan_ms is None else {
                           "ms_per_step": round(plan_ms, 5),
                           "value": round(nbytes / (plan_ms / 1e3) / 1e9, 3), "unit": "GB/s",
                           "hbm_frac": round(nbytes / (plan_ms / 1e3) / 1e9 / hbm, 4),
                           "steps": Ks, "what": "ssspmv_plan_execute: kernels (b) and (c) on "
                                               "a partition computed once"},
                       "wall_s_timed_loop": round(t_wall, 3)},
            "roofline": {"bound": "hbm",
                         "kernel": "csr_rows_kernel" if rows_variant else "segsum_kernel",
                         "achieved": round(achieved, 2), "peak": hbm, "unit": "GB/s",
                         "frac": round(achieved / hbm, 4), "peak_kind": peak_kind,
                         "traffic": traffic},
            "clocks": clocks,
            "e2e": e2e,
            "gpu_launches": (1 if rows_variant else 3) * K,
            "cpu_baseline": cpu,
        }
        if world == 1 and args.configs and args.workload == "stencil160" and not args.select:
            # the other configurations, each with its own clock sample (their
            # kernels run after the headline's timed region)
            del Ad, xd, y, ws
            if "buf" in locals():
                del buf
            torch.cuda.empty_cache()
            line["configs"] = extra_configs(args, dev)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# reduced precision (FP32 val/x/y, or BF16 val with FP32 x/y) on one matrix

def _event_loop(step, flush_l2, K, stream):
    """K steps, each after an L2 flush outside the timed region, timed by
    events on the launching stream around the step (no host wait between
    steps); returns the per-step device times (ms)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    for e0, e1 in ev:
        flush_l2()
        e0.record(stream)
        step()
        e1.record(stream)
    torch.cuda.synchronize()
    return [e0.elapsed_time(e1) for e0, e1 in ev]


def _timed_loop(step, flush_l2, K, stream):
    """K steps, each after an L2 flush outside the timed region; returns the
    per-step device times (ms) from events on the launching stream."""
    import torch
    times = []
    for _ in range(K):
        flush_l2()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return times


def _flusher(dev):
    import torch
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    sink = torch.empty(1, dtype=torch.int64, device=dev)

    def flush_l2():
        flush.fill_(1)
        torch.sum(flush.view(torch.int64), 0, keepdim=True, out=sink)
    return flush_l2


def _cpu_baseline(mats, budget_s, bytes_of):
    """The oracle (FP64 row loop over OpenMP threads) on a bounded sample of
    the workload; GB/s in this workload's own byte count."""
    import numpy as np

    import oracle
    t0, done, nbytes, used, k = time.perf_counter(), 0, 0, 1, 0
    while time.perf_counter() - t0 < budget_s:
        A, x = mats[k % len(mats)]
        y = np.empty(A.m)
        _, used = oracle.spmv_omp(A.row_ptr, A.col, A.val, x, y=y)
        nbytes += bytes_of(A)
        done += 1
        k += 1
    dt = time.perf_counter() - t0
    return nbytes / dt / 1e9, used, done, dt


class _Single:
    """One matrix on the device in one precision: FP64 (val, x, y double),
    FP32 (val, x, y float) or BF16 values with FP32 x and y."""
    VB = {"f64": 8, "f32": 4, "bf16": 2}

    def __init__(self, A, x, dev, precision: str):
        import numpy as np
        import torch
        from paper_1504_06474_gb300 import ssspmv as C
        self.A, self.dev, self.precision = A, dev, precision
        self.vb = self.VB[precision]
        self.rp = torch.as_tensor(A.row_ptr, device=dev)
        self.col = torch.as_tensor(A.col, device=dev)
        if precision == "f64":
            self.val = torch.as_tensor(A.val, device=dev)
            self.x = torch.as_tensor(x, device=dev)
            self.fn = C.ssspmv_csr_f64
        elif precision == "f32":
            self.val = torch.as_tensor(A.val.astype(np.float32), device=dev)
            self.x = torch.as_tensor(x.astype(np.float32), device=dev)
            self.fn = C.ssspmv_csr_f32
        else:
            self.val = torch.as_tensor(A.val).to(torch.bfloat16).to(dev).view(torch.int16)
            self.x = torch.as_tensor(x.astype(np.float32), device=dev)
            self.fn = C.ssspmv_csr_bf16f32
        ydt = torch.float64 if precision == "f64" else torch.float32
        self.y = torch.empty(A.m, dtype=ydt, device=dev)
        self.yb = 8 if precision == "f64" else 4
        self.nbytes = algorithmic_bytes(A.m, A.n, A.nnz, val_bytes=self.vb, y_bytes=self.yb,
                                        x_bytes=self.yb)

    def workspace(self, opts):
        import torch
        from paper_1504_06474_gb300 import ssspmv as C
        return torch.empty(max(C.ssspmv_workspace_bytes(self.A.m, self.A.nnz, self.vb, opts), 256),
                           dtype=torch.uint8, device=self.dev)

    def call(self, opts, ws, stream):
        from paper_1504_06474_gb300 import ssspmv as C
        A = self.A
        C.check(self.fn(A.m, A.n, A.nnz, self.rp, self.col, self.val, self.x, self.y, opts=opts,
                        workspace=ws, stream=stream), "ssspmv_csr_" + self.precision)

    def rounded_inputs(self):
        """The values and x as the device stores them, in FP64 (host)."""
        import numpy as np
        import torch
        if self.precision == "f64":
            return self.A.val, self.x.cpu().numpy()
        if self.precision == "f32":
            v = self.val.cpu().numpy().astype(np.float64)
        else:
            v = self.val.view(torch.bfloat16).to(torch.float64).cpu().numpy()
        return v, self.x.cpu().numpy().astype(np.float64)


def _time_whole(step, K, flush_l2, stream, gpu, warmup=3):
    """Mean and median whole-call time (ms) over K flushed steps timed by
    events around each call, with a clock sample during the timed region."""
    import torch
    for _ in range(warmup):
        flush_l2()
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu)
    sampler.start()
    time.sleep(0.25)
    t = _event_loop(step, flush_l2, K, stream)
    clocks = sampler.stop()
    return sum(t) / K, statistics.median(t), clocks


def _stages(single, opts_kw, ws, K, flush_l2, stream):
    """Kernel (a), (b), (c) and whole times (ms) from the library's events
    at the kernel boundaries, in a run of their own."""
    from paper_1504_06474_gb300 import ssspmv as C
    timer = C.ssspmv_timer_create(K)
    ot = C.make_opts(timer=timer, **opts_kw)
    _timed_loop(lambda: single.call(ot, ws, stream), flush_l2, K, stream)
    t = C.ssspmv_timer_read(timer, K)
    C.ssspmv_timer_destroy(timer)
    return {"partition": round(sum(v[0] for v in t) / K, 5),
            "segsum": round(sum(v[1] for v in t) / K, 5),
            "calibrate": round(sum(v[2] for v in t) / K, 5), "steps": K,
            "whole": round(sum(v[3] for v in t) / K, 5)}


def _errors(single, x64):
    """Largest |y - yref| / s over rows with s > 0 (s = sum |a x|), against
    the FP64 oracle on the stored (rounded) inputs and on the FP64 inputs."""
    import numpy as np

    import oracle
    A = single.A
    y = single.y.cpu().numpy().astype(np.float64)
    out = {}
    v_r, x_r = single.rounded_inputs()
    yref, s = oracle.spmv_dot2(A.row_ptr, A.col, v_r, x_r)
    nz = s > 0
    out["max_err_over_s_rounded_inputs"] = float(np.max(np.abs(y - yref)[nz] / s[nz])) if nz.any() else 0.0
    out["empty_rows_exact_zero"] = bool(np.all(y[~nz] == 0.0))
    if single.precision != "f64":
        y64, s64 = oracle.spmv_dot2(A.row_ptr, A.col, A.val, x64)
        nz = s64 > 0
        out["max_err_over_s_fp64_inputs"] = float(np.max(np.abs(y - y64)[nz] / s64[nz])) if nz.any() else 0.0
    return out


def measure_single(A, x, dev, precision, opts_kw, K, workload, cpu_seconds=0.0, e2e_steps=0,
                   hot=False, compare_f64=True, errors=True):
    """One configuration of a single product: the JSON line of
    `--precision` (also used for the configurations of the default run)."""
    import numpy as np
    import torch
    from paper_1504_06474_gb300 import ssspmv as C
    gpu = dev.index or 0
    single = _Single(A, x, dev, precision)
    opts = C.make_opts(**opts_kw)
    ws = single.workspace(opts)
    stream = torch.cuda.current_stream(dev)
    flush = _flusher(dev)
    flush_l2 = (lambda: None) if hot else flush
    whole, med, clocks = _time_whole(lambda: single.call(opts, ws, stream), K, flush_l2, stream,
                                     gpu)
    st = _stages(single, opts_kw, ws, min(K, 200), flush_l2, stream)
    nbytes = single.nbytes
    value = nbytes / (whole / 1e3) / 1e9
    hbm, peak_kind = peaks()
    shape = C.ssspmv_plan_shape(A.m, A.nnz, single.vb, opts)
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": 1, "steps": K,
        "warmup": 3, "ms_per_step": round(whole, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"f64": "f64", "f32": "f32", "bf16": "bf16-val/f32"}[precision],
        "data": "synthetic",
        "config": {"workload": workload, "precision": precision, "m": A.m, "n": A.n,
                   "nnz": A.nnz, "W": shape["W"], "S": shape["S"], "bytes_per_step": nbytes,
                   "hbm_frac": round(value / hbm, 4), "us_per_call": round(whole * 1e3, 2),
                   "ms_per_step_median": round(med, 5), "stage_ms": st,
                   "l2": ("not flushed (hot: inputs stay in L2 between steps)" if hot else
                          "flushed between steps (512 MB write then read, outside the timed events)")},
        "roofline": {"bound": "hbm", "kernel": "segsum_kernel",
                     "achieved": round(nbytes / (st["segsum"] / 1e3) / 1e9, 2), "peak": hbm,
                     "unit": "GB/s", "frac": round(nbytes / (st["segsum"] / 1e3) / 1e9 / hbm, 4),
                     "peak_kind": peak_kind, "traffic": None},
        "clocks": clocks, "gpu_launches": 3 * K,
    }
    if precision != "f64":
        line["config"]["accumulation"] = "compensated FP32 pairs (TwoProduct + TwoSum)"
    if errors:
        line["config"]["error"] = _errors(single, x)
    if compare_f64 and precision != "f64":
        # the plain FP64 call on the same matrix, same GPU, same timing
        s64 = _Single(A, x, dev, "f64")
        ws64 = s64.workspace(None)
        ms64, _, _ = _time_whole(lambda: s64.call(None, ws64, stream), min(K, 200), flush_l2,
                                 stream, gpu)
        line["config"]["plain_f64_ms"] = round(ms64, 5)
        line["config"]["speedup_vs_plain_f64"] = round(ms64 / whole, 3)
        del s64, ws64
    e2e = None
    if e2e_steps > 0:
        # pinned host inputs in, y out, every step
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        h = [pin(A.row_ptr), pin(A.col), single.val.cpu().pin_memory(), single.x.cpu().pin_memory()]
        d = [single.rp, single.col, single.val, single.x]
        hy = torch.empty(A.m, dtype=single.y.dtype).pin_memory()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            for dst, src in zip(d, h):
                dst.copy_(src, non_blocking=True)
            single.call(opts, ws, stream)
            hy.copy_(single.y, non_blocking=True)
            torch.cuda.synchronize(dev)
        te = (time.perf_counter() - t0) / e2e_steps
        h2d = sum(v.numel() * v.element_size() for v in h)
        e2e = {"value": round(nbytes / te / 1e9, 3), "unit": "GB/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": A.m * single.yb, "ms_per_step": round(te * 1e3, 4)}
    line["e2e"] = e2e
    status = C.ssspmv_device_status(ws, stream=stream)
    if status:
        raise RuntimeError("device status bits %#x" % status)
    cpu = None
    if cpu_seconds > 0:
        rate, used, reps, dt = _cpu_baseline([(A, x)], cpu_seconds, lambda M: nbytes)
        cpu = {"value": round(rate, 3), "unit": "GB/s", "cores": used, "kind": "oracle",
               "sample": "%d whole %s SpMVs by the FP64 oracle row loop (%d OpenMP threads), "
                         "counted at this configuration's bytes per step, %.1f s"
                         % (reps, workload, used, dt)}
    line["cpu_baseline"] = cpu
    return line


def _select_compare(single, dev, K, flush_l2, gpu):
    """The shipped selector's class for this FP64 matrix (from its device
    features) timed beside the default configuration."""
    import torch
    from paper_1504_06474_gb300 import selector as SEL
    from paper_1504_06474_gb300 import ssspmv as C
    params = SEL.load_default()
    if params is None:
        return {"unavailable": "no selector weights shipped with the package"}
    A = single.A
    f = SEL.device_features(single.rp, A.m, A.n, A.nnz).cpu().numpy()[None, :]
    k = int(SEL.select(params, f, dev)[0])
    kw = SEL.CLASSES[k][1]
    stream = torch.cuda.current_stream(dev)
    o_sel = C.make_opts(W=kw.get("W", 0), variant=kw.get("variant", 0),
                        block_warps=kw.get("block_warps", 0))
    o_def = C.make_opts()
    ws_s, ws_d = single.workspace(o_sel), single.workspace(o_def)
    ms_s, _, clocks = _time_whole(lambda: single.call(o_sel, ws_s, stream), K, flush_l2, stream, gpu)
    ms_d, _, _ = _time_whole(lambda: single.call(o_def, ws_d, stream), K, flush_l2, stream, gpu)
    return {"class": SEL.CLASSES[k][0], "index": k, "selected_ms": round(ms_s, 5),
            "default_ms": round(ms_d, 5), "speedup_vs_default": round(ms_d / ms_s, 4),
            "clocks": clocks}


def _summary(line, keep_error=True):
    """The fields of a configuration's line that go into the default run's
    `configs` object."""
    c = line["config"]
    out = {"value": line["value"], "unit": line["unit"], "dtype": line["dtype"],
           "ms_per_step": line["ms_per_step"], "hbm_frac": c.get("hbm_frac"),
           "kernel_b_frac": line["roofline"]["frac"], "stage_ms": c.get("stage_ms"),
           "steps": line["steps"], "clocks": line["clocks"], "l2": c.get("l2")}
    for k in ("us_per_call", "speedup_vs_plain_f64", "plain_f64_ms", "W", "S", "m", "nnz"):
        if k in c:
            out[k] = c[k]
    if keep_error and "error" in c:
        out["error"] = c["error"]
    if line.get("cpu_baseline"):
        out["cpu_baseline"] = line["cpu_baseline"]
    return out


def extra_configs(args, dev):
    """The other configurations of the benchmark, measured in the same run
    beside the headline: the small uniform matrix (flushed and hot), the
    power-law graph in FP64, FP32 and BF16 values (each with its error
    against the FP64 oracle), the batch of 512 matrices under a CUDA graph,
    and the shipped selector on the stencil and the power-law graph."""
    import types
    import torch

    import synth
    gpu = dev.index or 0
    K = args.config_steps
    out = {}
    t0 = time.perf_counter()
    A, x = synth.workload("uniform4096")
    flushed = measure_single(A, x, dev, "f64", {}, 4 * K, "uniform4096",
                             cpu_seconds=args.config_cpu_seconds)
    hot = measure_single(A, x, dev, "f64", {}, 4 * K, "uniform4096", hot=True, errors=False)
    u = _summary(flushed)
    u["hot"] = {"us_per_call": hot["config"]["us_per_call"], "value": hot["value"],
                "stage_ms": hot["config"]["stage_ms"], "clocks": hot["clocks"]}
    out["uniform4096_f64"] = u
    A, x = synth.workload("rmat22")
    for prec in ("f64", "f32", "bf16"):
        line = measure_single(A, x, dev, prec, {}, K, "rmat22",
                              cpu_seconds=args.config_cpu_seconds if prec == "f64" else 0.0)
        out["rmat22_" + prec] = _summary(line)
        torch.cuda.empty_cache()
    flush = _flusher(dev)
    out["select_rmat22"] = _select_compare(_Single(A, x, dev, "f64"), dev, K, flush, gpu)
    del A, x
    S, xs = synth.workload("stencil160")
    out["select_stencil160"] = _select_compare(_Single(S, xs, dev, "f64"), dev, K, flush, gpu)
    del S, xs
    torch.cuda.empty_cache()
    ns = types.SimpleNamespace(workload="batch512", tile_w=0, tile_s=0, variant=0, warmup=3,
                               steps=max(10, K // 5), e2e_steps=2,
                               cpu_seconds=args.config_cpu_seconds)
    b = measure_batch(ns, dev)
    bs = {"value": b["value"], "unit": b["unit"], "dtype": b["dtype"],
          "ms_per_step": b["ms_per_step"], "hbm_frac": b["config"]["hbm_frac"],
          "kernel_b_frac": b["roofline"]["frac"], "steps": b["steps"], "clocks": b["clocks"]}
    for k in ("matrices", "families", "rows", "nnz", "W", "variant", "autotuned", "launch",
              "stage_ms", "speedup_vs_separate_f32_calls", "speedup_vs_plain_f64",
              "separate_f32_calls_ms", "separate_plain_f64_calls_ms", "l2"):
        bs[k] = b["config"][k]
    bs["e2e"] = b["e2e"]
    bs["cpu_baseline"] = b["cpu_baseline"]
    out["batch512_f32"] = bs
    torch.cuda.empty_cache()
    out["wall_s"] = round(time.perf_counter() - t0, 1)
    return out


def run_precision(args):
    import torch

    import synth
    from paper_1504_06474_gb300 import _build
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _build.build()
    A, x = synth.workload(args.workload)
    line = measure_single(A, x, dev, args.precision,
                          dict(W=args.tile_w, S=args.tile_s, variant=args.variant,
                               block_warps=args.block_warps), args.steps,
                          args.workload, cpu_seconds=args.cpu_seconds,
                          e2e_steps=args.e2e_steps, hot=args.hot)
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# a batch of many matrices (FP32) in one graph launch

def run_batch(args):
    import torch

    from paper_1504_06474_gb300 import _build
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _build.build()
    print(json.dumps(measure_batch(args, dev)), flush=True)
    return 0


def measure_batch(args, dev):
    """The batched FP32 call over a seeded mixed batch as one CUDA-graph
    replay, beside the same matrices as separate calls; returns the line."""
    import numpy as np
    import torch

    import synth
    from paper_1504_06474_gb300 import ssspmv as C
    local = dev.index or 0
    count = int(args.workload[len("batch"):])
    specs = synth.batch_specs(count, seed=3)
    t_gen = time.perf_counter()
    mats = [synth.batch_matrix(sp) for sp in specs]
    t_gen = time.perf_counter() - t_gen
    dd = []  # device arrays per matrix
    descs = []
    for A, x in mats:
        d = dict(rp=torch.as_tensor(A.row_ptr, device=dev), col=torch.as_tensor(A.col, device=dev),
                 val=torch.as_tensor(A.val.astype(np.float32), device=dev),
                 x=torch.as_tensor(x.astype(np.float32), device=dev),
                 y=torch.empty(A.m, dtype=torch.float32, device=dev))
        dd.append(d)
        descs.append((A.m, A.n, A.nnz, d["rp"], d["col"], d["val"], d["x"], d["y"]))
    desc = torch.as_tensor(np.frombuffer(C.batch_descriptors(descs), np.uint8).copy(), device=dev)
    total_nnz = sum(A.nnz for A, _ in mats)
    f32_bytes = lambda A: algorithmic_bytes(A.m, A.n, A.nnz, val_bytes=4, y_bytes=4, x_bytes=4)
    nbytes = sum(f32_bytes(A) for A, _ in mats)
    # tile shape and store variant chosen by the library's autotuner on this
    # batch (unless given on the command line)
    tuned = None
    if args.tile_w == 0 and args.variant == 0:
        from paper_1504_06474_gb300 import selector as S
        torch.cuda.synchronize(dev)
        kw, cand_ms = S.tune_batched(count, desc, total_nnz, dev)
        tuned = {"chosen": kw, "candidates_ms": {k: round(v, 4) for k, v in cand_ms.items()}}
        args.tile_w, args.variant = kw["W"], kw["variant"]
    bwarps = getattr(args, "block_warps", 0)
    opts = C.make_opts(W=args.tile_w, S=args.tile_s, variant=args.variant, block_warps=bwarps)
    ws = torch.empty(C.ssspmv_batched_workspace_bytes(count, total_nnz, 4, opts),
                     dtype=torch.uint8, device=dev)
    s = torch.cuda.Stream(dev)
    flush_l2 = _flusher(dev)
    torch.cuda.synchronize(dev)

    def batched(o=opts):
        C.check(C.ssspmv_csr_batched_f32(count, desc, total_nnz, opts=o, workspace=ws, stream=s),
                "ssspmv_csr_batched_f32")
    with torch.cuda.stream(s):
        for _ in range(args.warmup):
            batched()
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        batched()
    K = args.steps
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.25)
    with torch.cuda.stream(s):
        times = _timed_loop(g.replay, flush_l2, K, s)
    clocks = sampler.stop()
    ms = sum(times) / K
    value = nbytes / (ms / 1e3) / 1e9
    # stage split from direct (uncaptured) launches with the library's timer
    kst = min(K, 20)
    timer = C.ssspmv_timer_create(kst)
    ot = C.make_opts(W=args.tile_w, S=args.tile_s, variant=args.variant, timer=timer,
                     block_warps=bwarps)
    with torch.cuda.stream(s):
        _timed_loop(lambda: batched(ot), flush_l2, kst, s)
    st = C.ssspmv_timer_read(timer, kst)
    C.ssspmv_timer_destroy(timer)
    seg = sum(v[1] for v in st) / kst
    stage = {"setup_and_partition": round(sum(v[0] for v in st) / kst, 5), "segsum": round(seg, 5),
             "calibrate": round(sum(v[2] for v in st) / kst, 5)}
    # the same matrices as separate single calls: FP32, and the plain FP64 kernel
    big = max(C.ssspmv_workspace_bytes(A.m, A.nnz, 8, None) for A, _ in mats)
    ws1 = torch.empty(big, dtype=torch.uint8, device=dev)

    def separate_f32():
        for (A, _), d in zip(mats, dd):
            C.check(C.ssspmv_csr_f32(A.m, A.n, A.nnz, d["rp"], d["col"], d["val"], d["x"], d["y"],
                                     workspace=ws1, stream=s), "ssspmv_csr_f32")
    with torch.cuda.stream(s):
        separate_f32()
        t_sep = _timed_loop(separate_f32, flush_l2, 5, s)
    d64 = [dict(val=torch.as_tensor(A.val, device=dev), x=torch.as_tensor(x, device=dev),
                y=torch.empty(A.m, dtype=torch.float64, device=dev)) for A, x in mats]

    def separate_f64():
        for (A, _), d, e in zip(mats, dd, d64):
            C.check(C.ssspmv_csr_f64(A.m, A.n, A.nnz, d["rp"], d["col"], e["val"], e["x"], e["y"],
                                     workspace=ws1, stream=s), "ssspmv_csr_f64")
    with torch.cuda.stream(s):
        separate_f64()
        t64 = _timed_loop(separate_f64, flush_l2, 5, s)
    del d64
    ms_sep, ms64 = sum(t_sep) / len(t_sep), sum(t64) / len(t64)
    # end to end: every matrix's inputs from pinned host memory, the graph, every y back
    e2e = None
    if args.e2e_steps > 0:
        hosts = [(torch.from_numpy(A.row_ptr).pin_memory(), torch.from_numpy(A.col).pin_memory(),
                  d["val"].cpu().pin_memory(), d["x"].cpu().pin_memory(),
                  torch.empty(A.m, dtype=torch.float32).pin_memory()) for (A, _), d in zip(mats, dd)]
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            with torch.cuda.stream(s):
                for h, d in zip(hosts, dd):
                    d["rp"].copy_(h[0], non_blocking=True)
                    d["col"].copy_(h[1], non_blocking=True)
                    d["val"].copy_(h[2], non_blocking=True)
                    d["x"].copy_(h[3], non_blocking=True)
                g.replay()
                for h, d in zip(hosts, dd):
                    h[4].copy_(d["y"], non_blocking=True)
            s.synchronize()
        te = (time.perf_counter() - t0) / args.e2e_steps
        h2d = sum(sum(v.numel() * v.element_size() for v in h[:4]) for h in hosts)
        d2h = sum(h[4].numel() * 4 for h in hosts)
        e2e = {"value": round(nbytes / te / 1e9, 3), "unit": "GB/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": round(te * 1e3, 4)}
    status = C.ssspmv_device_status(ws, stream=s)
    if status:
        raise RuntimeError("device status bits %#x" % status)
    cpu = None
    if args.cpu_seconds > 0:
        rate, used, done, dt = _cpu_baseline(mats, args.cpu_seconds, f32_bytes)
        cpu = {"value": round(rate, 3), "unit": "GB/s", "cores": used, "kind": "oracle",
               "sample": "%d matrix products cycling through the batch in order, by the FP64 "
                         "oracle row loop (%d OpenMP threads), counted at FP32 bytes, %.1f s"
                         % (done, used, dt)}
    hbm, peak_kind = peaks()
    fams = {f: sum(1 for sp in specs if sp[0] == f) for f in synth.BATCH_FAMILIES}
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": 1, "steps": K,
        "warmup": args.warmup, "ms_per_step": round(ms, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "matrices": count, "families": fams,
                   "rows": sum(A.m for A, _ in mats), "nnz": total_nnz,
                   "bytes_per_step": nbytes, "hbm_frac": round(value / hbm, 4),
                   "W": C.ssspmv_plan_shape(1, 1, 4, opts)["W"],
                   "variant": ["default", "speculative", "exact", "rows"][args.variant],
                   "autotuned": tuned,
                   "launch": "one CUDA graph replay: set-up, partition, one persistent "
                             "segmented-sum launch over every bunch of every matrix, calibration",
                   "stage_ms": stage, "separate_f32_calls_ms": round(ms_sep, 4),
                   "speedup_vs_separate_f32_calls": round(ms_sep / ms, 3),
                   "separate_plain_f64_calls_ms": round(ms64, 4),
                   "speedup_vs_plain_f64": round(ms64 / ms, 3),
                   "generation_s": round(t_gen, 1),
                   "l2": "flushed between steps (512 MB write then read, outside the timed events)"},
        "roofline": {"bound": "hbm", "kernel": "segsum_kernel (batched)",
                     "achieved": round(nbytes / (seg / 1e3) / 1e9, 2), "peak": hbm,
                     "unit": "GB/s", "frac": round(nbytes / (seg / 1e3) / 1e9 / hbm, 4),
                     "peak_kind": peak_kind, "traffic": None},
        "clocks": clocks, "e2e": e2e, "gpu_launches": 4 * K, "cpu_baseline": cpu,
    }
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="stencil160")
    ap.add_argument("--tile-w", type=int, default=0)
    ap.add_argument("--tile-s", type=int, default=0)
    ap.add_argument("--select", action="store_true",
                    help="FP64: tile shape and variant chosen by the shipped selector network "
                         "(the default configuration is timed beside it)")
    ap.add_argument("--block-warps", type=int, default=0)
    ap.add_argument("--variant", type=int, default=0,
                    help="0 default, 1 speculative + calibration, 2 exact stores, 3 row-parallel")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--hot", action="store_true",
                    help="no L2 flush between steps (for workloads that fit in L2, e.g. uniform4096)")
    ap.add_argument("--configs", action=argparse.BooleanOptionalAction, default=True,
                    help="after the stencil160 FP64 headline, measure the other configurations "
                         "(uniform4096, rmat22 FP64/FP32/BF16, batch512, the selector) into the "
                         "line's `configs` object")
    ap.add_argument("--config-steps", type=int, default=100,
                    help="timed steps per configuration of `configs`")
    ap.add_argument("--config-cpu-seconds", type=float, default=3.0,
                    help="CPU-oracle budget per configuration of `configs`")
    ap.add_argument("--precision", choices=["f64", "f32", "bf16"], default="f64",
                    help="f32: FP32 val/x/y; bf16: BF16 val, FP32 x/y (compensated FP32 sums)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload.startswith("batch"):
        return run_batch(args)
    if args.precision != "f64":
        return run_precision(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
