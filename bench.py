"""Benchmark of the iALS++ epoch on GB300 (one JSON line on stdout).

A step is one epoch of Algorithm 3 (residual recompute, then for every block
the user pass and the item pass) over the ML20M-shaped synthetic workload:
136,000 users x 20,000 items, 10M binary positives (Zipf(1.05) items,
lognormal(3.7, 1.1) user lengths clipped to [5, 8000]), d = 128, b = 32,
alpha0 = 0.1, lambda = 1e-3 scaled by (1 + nu |S_r|) with nu = 1.

Metric: row-block solves per second, (|U| + |I|) * d / b per epoch.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision fp32|bf16] [--no-cpu-baseline]

--impl reference times the FP64 CPU oracle (the reference arm of this
project: the paper ships no code) on a bounded sample of the same workload.
Under torchrun each rank trains an independent replica on its own GPU
(replicas only; no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "ml20m_136k"
WORKLOADS = {
    "ml20m_136k": ("ML20M-shaped synthetic: 136,000 users x 20,000 items, 10,000,000 positives, "
                   "Zipf(1.05) items, lognormal(3.7,1.1) lengths in [5,8000], d=128, b=32, "
                   "alpha0=0.1, lambda=1e-3, nu=1, seed 0"),
    "skewed_136k": ("ML20M shape with skewed users: 136,000 users x 20,000 items, 10,000,000 "
                    "positives, Zipf(1.05) items, Zipf(1.3) user activity (rows capped at all "
                    "20,000 items), d=128, b=32, alpha0=0.1, lambda=1e-3, nu=1, seed 0"),
    "msd_570k": ("MSD-shaped synthetic: 570,000 users x 41,000 items, 34,000,000 positives, "
                 "Zipf(0.9) items, lognormal(3.5,1.2) lengths in [1,41000], d=1024, b=128, "
                 "alpha0=0.02, lambda=2e-3, nu=1, seed 0"),
}
WORKLOAD_DESC = WORKLOADS[WORKLOAD]
METRIC = "iALS++ epoch throughput (row-block solves/s = (|U|+|I|)*d/b per epoch)"

# DRAM bytes (read + write) per launch of the dominant kernel, from the ncu capture
# summarised under profiles/ (per precision); valid only for the workload (name, d, b)
# and the kernel sources it was taken on (sha256 of the listed files, concatenated,
# first 16 hex digits).
NCU_TRAFFIC = {
    ("sparse", "bf16"): {"workload": ("ml20m_136k", 128, 32),
                         "sources": ["paper_2110_14044_gb300/csrc/k_sparse_bf16.cuh",
                                     "paper_2110_14044_gb300/csrc/k_sparse_impl.cuh"],
                         "sha256_16": "c5cac084ed942636", "bytes_per_launch": 283.9e6},
    ("sparse", "fp32"): {"workload": ("ml20m_136k", 128, 32),
                         "sources": ["paper_2110_14044_gb300/csrc/k_sparse_impl.cuh"],
                         "sha256_16": "ae0d25ab32b93899", "bytes_per_launch": 183.4e6},
}


def sources_hash(paths):
    import hashlib
    h = hashlib.sha256()
    for p in paths:
        h.update(open(os.path.join(ROOT, p), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(kind, precision, workload=None):
    """The recorded DRAM bytes per launch, if they were taken on this workload (name, d, b)
    and on the kernel sources as they are now; else None."""
    rec = NCU_TRAFFIC.get((kind, precision))
    if not rec or not rec["bytes_per_launch"]:
        return None
    if workload is not None and tuple(workload) != tuple(rec["workload"]):
        return None
    try:
        h = sources_hash(rec["sources"])
    except OSError:
        return None
    return rec["bytes_per_launch"] if h == rec["sha256_16"] else None


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


# ----------------------------------------------------------------- multi-rank aggregation
# Under torchrun every rank trains an independent replica (no collective on the
# data path); the only exchanges are the barriers around the timed region and
# the maximum of the per-rank times.  These helpers take the device so that the
# same code runs over NCCL (CUDA tensors) and over gloo (CPU tensors, in tests).
def rank_barrier(world, device):
    import torch
    if device.startswith("cuda"):
        torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        if device.startswith("cuda"):
            torch.cuda.synchronize()


def max_over_ranks(x, world, device):
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, ms_max):
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / (ms_max / 1e3)


# ----------------------------------------------------------------- error against stored oracle traces
GOLDEN = os.path.join(ROOT, "tests", "golden")


def inputs_fingerprint(data, W0, H0):
    """sha256 (first 16 hex) of the inputs a stored oracle trace was computed on."""
    import hashlib
    h = hashlib.sha256()
    for a in (data.u_indptr, data.u_items, W0, H0):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()[:16]


def load_trace(name):
    try:
        return json.load(open(os.path.join(GOLDEN, name)))
    except OSError:
        return None


def trace_errors(data, d, b, alpha0, lam, nu, W0, H0, precision, trace_name, stream=None):
    """Relative objective error per epoch of a fresh CUDA-graph run from (W0, H0)
    against the FP64 oracle's stored trace (written by tests/golden/make_oracle_trace.py,
    oracle and generator only), or the reason there is none."""
    import paper_2110_14044_gb300 as ials
    rec = load_trace(trace_name)
    if rec is None:
        return {"trace": trace_name, "missing": True}
    pr = rec["problem"]
    if (pr["d"], pr["b"], pr["n_users"], pr["nnz"]) != (d, b, data.n_users, int(data.u_indptr[-1])) or \
            inputs_fingerprint(data, W0, H0) != rec["inputs_sha256_16"]:
        return {"trace": trace_name, "skipped": "inputs differ from those the trace was computed on"}
    m = ials.Model(data, d, b, alpha0, lam, nu, precision=precision, graph=True, stream=stream,
                   W0=W0, H0=H0)
    rel = []
    for ref in rec["objective_after_epoch"]:
        o, _ = m.epoch(1, objective=True)
        rel.append(abs(o - ref) / abs(ref))
    m.close()
    return {"trace": trace_name, "epochs": len(rel), "rel_objective_error_per_epoch": rel,
            "max": max(rel) if rel else None}


def launches_per_epoch(kern, steps, bf16, b):
    """Kernel launches per epoch from the profiled intervals ({kind: (ms, marks)}).

    Every interval holds one kernel except the Gramian and row-term ones: the
    FP32 Gramian is a tile kernel and a reduction, the FP32 row terms one
    kernel; on the BF16 path each 32-column slab (one for b = 16, 32; b / 32
    above) is a tcgen05 kernel plus a reduction (Gramian) or plus the G
    transpose-split (row terms)."""
    slabs = max(1, b // 32) if bf16 else 1
    per_mark = {"gram": 2 * slabs, "rowterm": 2 * slabs if bf16 else 1}
    return sum(c * per_mark.get(k, 1) for k, (_, c) in kern.items()) / steps


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- CPU oracle sample
def oracle_sample(prob, frac=0.1):
    """The FP64 oracle on the first `frac` of the users (all items): one user and
    one item block step per call.  Returns (callable, rows per call)."""
    import oracle
    from paper_2110_14044_gb300 import synth
    data = prob.data
    n_sub = max(1, int(data.n_users * frac))
    end = int(data.u_indptr[n_sub])
    u_ptr = data.u_indptr[:n_sub + 1].copy()
    u_idx = data.u_items[:end].copy()
    i_ptr, i_idx = synth.transpose_csr(n_sub, data.n_items, u_ptr, u_idx)
    P = oracle.Problem(n_sub, data.n_items, u_ptr, u_idx, i_ptr, i_idx, prob.d, prob.b,
                       prob.alpha0, prob.lam, prob.nu)
    W, H = P.factors(prob.W0[:n_sub], prob.H0)
    yhat = oracle.predict(P, W, H)
    state = {"k": 0}
    nb = prob.d // prob.b

    def step():
        k = state["k"] % nb
        oracle.halfstep(P, 0, k, W, H, yhat)
        oracle.halfstep(P, 1, k, W, H, yhat)
        state["k"] += 1

    who = (f"all {n_sub} users" if n_sub == data.n_users else f"the first {n_sub} users")
    desc = (f"FP64 oracle, one user + one item block step per call on {who} "
            f"({end} positives) x {data.n_items} items, d={prob.d}, b={prob.b}")
    return step, n_sub + data.n_items, desc, P.n_threads


def cpu_baseline(prob, budget_s=15.0, frac=0.1):
    step, rows, desc, threads = oracle_sample(prob, frac)
    t0 = time.perf_counter()
    n = 0
    while True:
        step()
        n += 1
        if time.perf_counter() - t0 >= budget_s or n >= 64:
            break
    dt = time.perf_counter() - t0
    return {"value": rows * n / dt, "unit": "rows/s", "cores": threads, "kind": "oracle",
            "sample": desc + f"; {n} calls in {dt:.1f} s"}


def cpu_full_epoch(prob):
    """One whole epoch of Algorithm 3 by the FP64 oracle on the host cores, from the
    bench's initial factors (the full problem, every block, both sides)."""
    import oracle
    P = oracle.Problem.from_data(prob.data, prob.d, prob.b, prob.alpha0, prob.lam, prob.nu)
    t0 = time.perf_counter()
    oracle.ialspp(P, 1, prob.W0, prob.H0)
    dt = time.perf_counter() - t0
    rows = (prob.data.n_users + prob.data.n_items) * (prob.d // prob.b)
    return {"value": rows / dt, "unit": "rows/s", "cores": P.n_threads, "kind": "oracle",
            "epoch_s": dt,
            "sample": f"FP64 oracle, one whole epoch of the workload ({prob.data.n_users} users x "
                      f"{prob.data.n_items} items, {prob.data.nnz} positives, d={prob.d}, b={prob.b}) "
                      f"in {dt:.1f} s"}


# ----------------------------------------------------------------- reference arm
def run_reference(args):
    rank, _, world = env_rank()
    if rank != 0:
        return
    from paper_2110_14044_gb300 import synth
    prob = synth.preset(args.workload, seed=0, **overrides(args))
    # the whole problem at d <= 256 (one user and one item block step of all rows per step,
    # about 1.7 s on 16 host cores at the ML20M shape); a 1% user sample at d = 1024
    step, rows, desc, threads = oracle_sample(prob, 1.0 if prob.d <= 256 else 0.01)
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = rows * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "rows/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": describe(args, prob), "sample": desc},
        "cpu_baseline": {"value": value, "unit": "rows/s", "cores": threads, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def kernel_rooflines(m, steps, prec, b, precision_name, workload_key, peaks):
    """Per-kernel-kind device time over `steps` eager epochs (CUDA events around every
    launch, on the context's stream) against the algorithmic work of the context's own
    decomposition: the dominant kernel's `roofline` and every kind's fractions."""
    from paper_2110_14044_gb300 import _abi
    kern, prof_total, _ = _abi.ials_profile_epochs(m.ctx, steps)
    work = _abi.ials_work_model(m.ctx)
    n_launch_epoch = launches_per_epoch(kern, steps, prec == _abi.PREC_BF16, b)
    dom = max(("sparse", "gram", "rowterm", "residual", "split_solve", "split_resid"),
              key=lambda k: kern[k][0])
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    dms, dcnt = kern[dom]
    dbytes = work[dom][0] * steps  # bytes over all profiled launches
    achieved = dbytes / (dms / 1e3) / 1e9
    roofline = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm_peak,
                "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": measured_traffic(dom, precision_name, workload_key),
                "peak_source": peak_src,
                "bytes_per_launch": dbytes / max(dcnt, 1), "ms_per_launch": dms / max(dcnt, 1),
                "gflops": work[dom][1] * steps / (dms / 1e3) / 1e9}
    # every kernel kind against its own roofline: algorithmic bytes / event time against the
    # measured copy bandwidth; FLOPs against the tensor peak (BF16 tensor-core kernels: the
    # measured burst bf16 peak) or the FP32 FMA peak (152 SMs x 128 FMA x 2 x max SM clock)
    fma_peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    # (the BF16 path's row statistics at b = 128 run on FP32 register tiles)
    tensor_kinds = (("gram", "rowterm") + (("sparse",) if b != 128 else ())) if prec == _abi.PREC_BF16 else ()
    per_kind = {}
    for k, (kms, kcnt) in kern.items():
        if kms <= 0 or k == "objective":
            continue
        gbs = work[k][0] * steps / (kms / 1e3) / 1e9
        tfs = work[k][1] * steps / (kms / 1e3) / 1e12
        fpk = peaks.get("bf16_tflops", 1900.0) if k in tensor_kinds else fma_peak
        per_kind[k] = {"ms_per_epoch": kms / steps, "GB/s": gbs, "hbm_frac": gbs / hbm_peak,
                       "TFLOP/s": tfs, "flop_peak": fpk, "flop_frac": tfs / fpk}
    return roofline, per_kind, kern, prof_total, n_launch_epoch


# ----------------------------------------------------------------- our arm
def run_ours(args):
    rank, local_rank, world = env_rank()
    msd_job = sweep_job = None
    default_run = args.workload == WORKLOAD and not (args.d or args.b)
    if rank == 0 and args.d1024 and default_run:
        # the d = 1024 workload's interaction set is drawn in a spawned process (no CUDA
        # in it) while the d = 128 measurements run
        msd_job = start_generation(MSD)
    if rank == 0 and args.sweep and default_run:
        sweep_job = start_generation(SWEEP)
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    from paper_2110_14044_gb300 import _abi, build, synth
    if rank == 0:
        build.build()   # one rank builds (a no-op when the library is up to date) ...
    if world > 1:
        torch.distributed.barrier()  # ... before any rank loads it
    import paper_2110_14044_gb300 as ials

    prob = synth.preset(args.workload, seed=0, **overrides(args))
    data = prob.data
    prec = _abi.PREC_BF16 if args.precision == "bf16" else _abi.PREC_FP32
    stream = torch.cuda.Stream()
    m = ials.Model(data, prob.d, prob.b, prob.alpha0, prob.lam, prob.nu, precision=prec,
                   graph=not args.no_graph, stream=stream, W0=prob.W0, H0=prob.H0)
    rows_per_epoch = (data.n_users + data.n_items) * (prob.d // prob.b)

    def barrier():
        rank_barrier(world, "cuda")

    # warm-up
    for _ in range(args.warmup):
        m.epoch(1)
    obj_before = m.objective()

    # timed region: K epochs, device-resident inputs (working set > L2)
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    _, st = m.epoch(args.steps)
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    ms = max_over_ranks(ms, world, "cuda")
    obj_after = m.objective()
    ms_per_step = ms / args.steps
    value = job_throughput(rows_per_epoch * args.steps, world, ms)

    # per-kernel device times over the same number of eager epochs (events per launch)
    peaks = load_peaks()
    roofline, per_kind, kern, prof_total, n_launch_epoch = kernel_rooflines(
        m, args.steps, prec, prob.b, args.precision, (args.workload, prob.d, prob.b), peaks)

    # end to end through the public API: factors in from pinned host memory,
    # one epoch, factors back to pinned host memory, every step
    Wp = torch.from_numpy(prob.W0).pin_memory()
    Hp = torch.from_numpy(prob.H0).pin_memory()
    e2e_steps = max(1, min(args.steps, 20))
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    for _ in range(e2e_steps):
        _abi.ials_set_factors(m.ctx, Wp, Hp)
        _abi.ials_epoch(m.ctx, 1)
        _abi.ials_get_factors(m.ctx, Wp, Hp)
    e1.record(stream)
    barrier()
    wall = time.perf_counter() - t0
    e2e_ms = max_over_ranks(max(e0.elapsed_time(e1), wall * 1e3), world, "cuda") / e2e_steps
    fb = (prob.W0.nbytes + prob.H0.nbytes)

    line = {
        "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == _abi.PREC_FP32 else "bf16",
        "data": "synthetic (seeded; no dataset in the container)",
        "config": {"workload": describe(args, prob), "precision": args.precision,
                   "graph": not args.no_graph,
                   "l2": "inputs larger than L2 (factors + residuals + CSR > 126 MB; no flush needed)",
                   "parallelism": f"replicas x{world}"},
        "epoch_s": ms_per_step / 1e3,
        "rows_per_s_plain": (data.n_users + data.n_items) / (ms_per_step / 1e3),
        "objective": {"before": obj_before, "after": obj_after, "status": st},
        "kernels_ms_per_epoch": {k: v[0] / args.steps for k, v in kern.items()},
        "profiled_epoch_ms": prof_total / args.steps,
        "roofline": roofline,
        "kernels_roofline": per_kind,
        "e2e": {"value": job_throughput(rows_per_epoch, world, e2e_ms), "unit": "rows/s",
                "h2d_bytes_per_step": fb, "d2h_bytes_per_step": fb, "ms_per_step": e2e_ms},
        "gpu_launches": int(round(n_launch_epoch * args.steps)),
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the whole problem when an oracle epoch fits the baseline's time bound (d <= 256),
        # else a user sample
        line["cpu_baseline"] = (cpu_full_epoch(prob) if prob.d <= 256
                                else cpu_baseline(prob, frac=0.01))
    if rank == 0 and args.variants:
        # the other precision on the same data, same timing
        other = "fp32" if args.precision == "bf16" else "bf16"
        oprec = _abi.PREC_FP32 if other == "fp32" else _abi.PREC_BF16
        m2 = ials.Model(data, prob.d, prob.b, prob.alpha0, prob.lam, prob.nu, precision=oprec,
                        graph=not args.no_graph, stream=stream, W0=prob.W0, H0=prob.H0)
        for _ in range(args.warmup):
            m2.epoch(1)
        o0 = m2.objective()
        barrier()
        ev0.record(stream)
        m2.epoch(args.steps)
        ev1.record(stream)
        barrier()
        ms2 = ev0.elapsed_time(ev1) / args.steps
        o_after2 = m2.objective()
        roof2, kinds2, _, _, _ = kernel_rooflines(m2, args.steps, oprec, prob.b, other,
                                                  (args.workload, prob.d, prob.b), peaks)
        line["variants"] = {
            args.precision: {"epoch_s": ms_per_step / 1e3, "rows_per_s": value / world,
                             "objective_after": obj_after},
            other: {"epoch_s": ms2 / 1e3, "rows_per_s": rows_per_epoch / (ms2 / 1e3),
                    "objective_before": o0, "objective_after": o_after2,
                    "roofline": roof2, "kernels_roofline": kinds2},
        }
        m2.close()
    if rank == 0 and args.workload == WORKLOAD and not (args.d or args.b):
        # error of every precision against the FP64 oracle, epoch by epoch, from the same
        # initial factors as the oracle's stored 16-epoch trace of this workload
        line["error_vs_oracle"] = {
            name: trace_errors(data, prob.d, prob.b, prob.alpha0, prob.lam, prob.nu, prob.W0, prob.H0,
                               pr, "ml20m_trace.json", stream)
            for name, pr in (("fp32", _abi.PREC_FP32), ("bf16", _abi.PREC_BF16))}
    if msd_job is not None:
        line["d1024"] = run_msd(msd_job, args, stream, peaks)
    if rank == 0 and args.foldin:
        line["foldin"] = run_foldin(cpu_sample=0 if args.no_cpu_baseline else 40)
    conv = args.convergence if args.convergence is not None else (6 if default_run else 0)
    if rank == 0 and conv:
        line["convergence"] = run_convergence(prob, conv, stream)
    if sweep_job is not None:
        line["sweep_skewed"] = run_sweep(sweep_job, stream)
    if rank == 0 and args.autotune:
        from paper_2110_14044_gb300 import autotune
        tuned = {}
        for name, pr in (("fp32", _abi.PREC_FP32), ("bf16", _abi.PREC_BF16)):
            best, table = autotune.autotune_block_size(data, prob.d, prob.alpha0, prob.lam, prob.nu,
                                                       precision=pr, W0=prob.W0, H0=prob.H0)
            tuned[name] = {"best_b": best, "epoch_s_by_b": {str(k): v for k, v in table.items()}}
        line["autotune"] = tuned
    if rank == 0:
        print(json.dumps(line), flush=True)
    m.close()
    if world > 1:
        torch.distributed.destroy_process_group()


# ----------------------------------------------------------------- the d = 1024 workload
MSD = "msd_570k"
MSD_BLOCKS = (32, 64, 128)   # the autotuner's candidates at d = 1024 (b = 128 is the stated one)


def _draw_preset(name, out_dir):
    """Child process: draw a preset's interaction set (seed 0) and save its CSR views."""
    from paper_2110_14044_gb300 import synth
    c = synth.PRESETS[name]
    data = synth.make_interactions(c["n_users"], c["n_items"], c["nnz"], c["zipf_s"], c["ln_mu"],
                                   c["ln_sigma"], c["len_min"], c["len_max"], 0, c.get("user_zipf"))
    for k in ("u_indptr", "u_items", "i_indptr", "i_users"):
        np.save(os.path.join(out_dir, k + ".npy"), getattr(data, k))


def start_generation(name):
    """Draw a preset's interactions in a spawned process (no CUDA in it) while the
    GPU measures something else; collect with `collect_generation`."""
    import multiprocessing as mp
    out_dir = tempfile.mkdtemp(prefix=name + "_")
    proc = mp.get_context("spawn").Process(target=_draw_preset, args=(name, out_dir))
    proc.start()
    return name, proc, out_dir


def collect_generation(job):
    import shutil
    from paper_2110_14044_gb300 import synth
    name, proc, out_dir = job
    proc.join()
    if proc.exitcode != 0:
        shutil.rmtree(out_dir, ignore_errors=True)
        raise RuntimeError(f"generator process for {name} exited with {proc.exitcode}")
    arrs = {k: np.load(os.path.join(out_dir, k + ".npy")) for k in ("u_indptr", "u_items", "i_indptr", "i_users")}
    shutil.rmtree(out_dir, ignore_errors=True)
    c = synth.PRESETS[name]
    return synth.Interactions(c["n_users"], c["n_items"], **arrs)


def run_msd(job, args, stream, peaks):
    """The metric's d = 1024 half: the MSD-shaped workload (570,000 x 41,000, 34M
    positives, d = 1024), FP32 and BF16 side by side at the stated b = 128 and at every
    autotuner candidate (the fastest is the autotuned b), with the rooflines of the
    stated and autotuned configurations and the per-epoch error against the FP64
    oracle on the 1% user subsample (stored traces; b = 128 and b = 32)."""
    import torch
    import paper_2110_14044_gb300 as ials
    from paper_2110_14044_gb300 import _abi, autotune, synth
    data = collect_generation(job)
    c = synth.PRESETS[MSD]
    d = c["d"]
    rows_plain = data.n_users + data.n_items
    out = {"workload": WORKLOADS[MSD], "initial_factors": "the library's seeded N(0, (0.1/sqrt(d))^2) draw",
           "steps": args.d1024_steps, "warmup": 1, "stated_b": c["b"], "configs": {}}
    K = max(1, args.d1024_steps)
    best = {}
    for pname, prec in (("bf16", _abi.PREC_BF16), ("fp32", _abi.PREC_FP32)):
        for b in MSD_BLOCKS:
            if not autotune.admissible(d, b, prec):
                continue
            m = ials.Model(data, d, b, c["alpha0"], c["lam"], c["nu"], precision=prec, graph=True,
                           stream=stream)
            m.epoch(1)
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            _, st = m.epoch(K)
            ev1.record(stream)
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1) / K
            rec = {"precision": pname, "b": b, "epoch_s": ms / 1e3,
                   "rows_per_s": rows_plain * (d // b) / (ms / 1e3), "rows_per_s_plain": rows_plain / (ms / 1e3),
                   "objective_after": m.objective(), "status": st}
            if b == c["b"]:
                rec["roofline"], rec["kernels_roofline"], _, _, _ = kernel_rooflines(
                    m, 1, prec, b, pname, (MSD, d, b), peaks)
            out["configs"][f"{pname}_b{b}"] = rec
            if pname not in best or ms < out["configs"][f"{pname}_b{best[pname]}"]["epoch_s"] * 1e3:
                best[pname] = b
            m.close()
    out["autotuned_b"] = best
    for pname, b in best.items():
        key = f"{pname}_b{b}"
        if "roofline" not in out["configs"][key]:
            prec = _abi.PREC_BF16 if pname == "bf16" else _abi.PREC_FP32
            m = ials.Model(data, d, b, c["alpha0"], c["lam"], c["nu"], precision=prec, stream=stream)
            m.epoch(1)
            out["configs"][key]["roofline"], out["configs"][key]["kernels_roofline"], _, _, _ = \
                kernel_rooflines(m, 1, prec, b, pname, (MSD, d, b), peaks)
            m.close()
    # error against the FP64 oracle on the 1% user subsample, epoch by epoch
    err = {"sample": "1% user subsample of the same generator: 5,700 users x 41,000 items, "
                     "340,000 positives, d = 1024, seeded W0/H0; FP64 oracle traces stored in tests/golden"}
    for b, tname in ((128, "msd_subsample_trace.json"), (32, "msd_subsample_b32_trace.json")):
        sub = synth.preset(MSD, seed=0, n_users=c["n_users"] // 100, nnz=c["nnz"] // 100, b=b)
        for pname, prec in (("fp32", _abi.PREC_FP32), ("bf16", _abi.PREC_BF16)):
            err[f"{pname}_b{b}"] = trace_errors(sub.data, d, b, sub.alpha0, sub.lam, sub.nu, sub.W0, sub.H0,
                                                prec, tname, stream)
    out["error_vs_oracle"] = err
    return out


def run_convergence(prob, epochs, stream):
    """Objective (Eq. 2, FP64) after each of `epochs` epochs for every admissible
    block size, in both precisions, from the same initial factors (the analogue,
    on the training objective, of the paper's quality-vs-b study, Section 5.2.2),
    with the device time of each epoch: b = 1 is iCD (Algorithm 2), b = d is iALS
    (Algorithm 1), so the table is also the three-way runtime comparison at this d."""
    import torch
    import paper_2110_14044_gb300 as ials
    from paper_2110_14044_gb300 import _abi, autotune
    out = {"epochs": epochs, "d": prob.d,
           "desc": "objective before and after each epoch and epoch seconds (graph replay; the "
                   "first epoch includes the capture); same W0, H0 for every run"}
    for name, prec in (("fp32", _abi.PREC_FP32), ("bf16", _abi.PREC_BF16)):
        res = {}
        for b in autotune.CANDIDATES:
            if not autotune.admissible(prob.d, b, prec):
                continue
            m = ials.Model(prob.data, prob.d, b, prob.alpha0, prob.lam, prob.nu, precision=prec,
                           graph=True, W0=prob.W0, H0=prob.H0, stream=stream)
            objs, secs = [m.objective()], []
            for _ in range(epochs):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                m.epoch(1)
                e1.record(stream)
                objs.append(m.objective())
                secs.append(e0.elapsed_time(e1) / 1e3)
            res[str(b)] = {"objective": objs, "epoch_s": secs,
                           "epoch_s_median_after_first": float(np.median(secs[1:])) if len(secs) > 1 else secs[0]}
            m.close()
        out[name] = res
    return out


# ------------------------------------------------------- the skewed-activity d sweep
SWEEP = "skewed_136k"
SWEEP_DIMS = (64, 256, 512, 2048)
SWEEP_BLOCKS = (1, 8, 16, 32, 64, 128, 256)   # b = 1 (iCD) timed where d <= 256
SWEEP_SPLITS = (512, 8192)                    # split lengths tried at the fastest b (0 = library's)


def run_sweep(job, stream):
    """Block size and work decomposition autotuned per d on the skewed-activity shape
    (Zipf(1.3) users): d in {64, 256, 512, 2048}, FP32 and BF16 side by side, every
    admissible b timed (one graph-replayed epoch after a warm-up epoch that captures
    the graph), then the split length tuned at the fastest b.  Where b = 1 and b = d
    are timed (iCD up to d = 256, iALS up to d = 512) the table holds the three-way
    comparison iCD / iALS++ / iALS."""
    from paper_2110_14044_gb300 import _abi, autotune, synth
    data = collect_generation(job)
    c = synth.PRESETS[SWEEP]
    lens = np.diff(data.u_indptr)
    out = {"workload": WORKLOADS[SWEEP].replace("d=128, b=32, ", ""),
           "max_user_row": int(lens.max()), "max_item_row": int(np.diff(data.i_indptr).max()),
           "users_over_1000": int((lens > 1000).sum()),
           "initial_factors": "the library's seeded N(0, (0.1/sqrt(d))^2) draw",
           "timing": "1 epoch (graph replay) after 1 warm-up epoch, CUDA events", "dims": {}}
    rows = data.n_users + data.n_items
    for d in SWEEP_DIMS:
        rec = {}
        for pname, prec in (("fp32", _abi.PREC_FP32), ("bf16", _abi.PREC_BF16)):
            by_b = {}
            # iALS (b = d) is timed up to d = 512; b = 1 (iCD) up to d = 256
            for b in SWEEP_BLOCKS + ((d,) if 256 < d <= 512 else ()):
                if not autotune.admissible(d, b, prec) or (b == 1 and d > 256):
                    continue
                by_b[b] = autotune.time_epoch(data, d, b, c["alpha0"], c["lam"], c["nu"], prec,
                                              epochs=1, stream=stream)
            best = min(by_b, key=by_b.get)
            by_split = {0: by_b[best]}
            for sl in SWEEP_SPLITS:
                by_split[sl] = autotune.time_epoch(data, d, best, c["alpha0"], c["lam"], c["nu"], prec,
                                                   epochs=1, split_len=sl, stream=stream)
            best_sl = min(by_split, key=by_split.get)
            rec[pname] = {"epoch_s_by_b": {str(k): v for k, v in by_b.items()},
                          "epoch_s_by_split_len": {str(k): v for k, v in by_split.items()},
                          "autotuned": {"b": best, "split_len": best_sl, "epoch_s": by_split[best_sl],
                                        "rows_per_s": rows * (d // best) / by_split[best_sl]}}
        f = rec["fp32"]["epoch_s_by_b"]
        rec["three_way_fp32"] = {"icd_b1_s": f.get("1"), "ialspp_s": rec["fp32"]["autotuned"]["epoch_s"],
                                 "ialspp_b": rec["fp32"]["autotuned"]["b"], "ials_bd_s": f.get(str(d))}
        out["dims"][str(d)] = rec
    return out


def run_ncu_step(args):
    """One user and one item block step (block 0) on the bench workload, for ncu."""
    import torch
    from paper_2110_14044_gb300 import _abi, build, synth
    build.build()
    import paper_2110_14044_gb300 as ials
    o = overrides(args)
    if args.ncu_frac < 1.0:  # a user sample of the workload (same shapes otherwise), for short captures
        c = synth.PRESETS[args.workload]
        o.update(n_users=max(1, int(c["n_users"] * args.ncu_frac)), nnz=max(1, int(c["nnz"] * args.ncu_frac)))
    prob = synth.preset(args.workload, seed=0, **o)
    prec = _abi.PREC_BF16 if args.precision == "bf16" else _abi.PREC_FP32
    m = ials.Model(prob.data, prob.d, prob.b, prob.alpha0, prob.lam, prob.nu, precision=prec,
                   W0=prob.W0, H0=prob.H0)
    for side in (0, 1):
        assert m.block_step(side, 0) == 0
    torch.cuda.synchronize()
    m.close()
    print("ncu-step done")


def run_ncu_foldin(n_req=16, seed=0):
    """A few fold-in requests of the serving workload (for profiler captures)."""
    import paper_2110_14044_gb300 as ials
    from paper_2110_14044_gb300 import build
    build.build()
    rng = np.random.Generator(np.random.Philox(key=[seed, 7]))
    n_items, d = 41000, 256
    H = rng.normal(0.0, 0.05, (n_items, d)).astype(np.float32)
    srv = ials.FoldinServer(H, d, 64, 0.1, 1e-3, 1.0, sweeps=4, workspace_bytes=1 << 30)
    tickets = []
    for _ in range(n_req):
        n = int(np.exp(rng.uniform(0.0, np.log(5000.0))))
        tickets.append(srv.submit(rng.choice(n_items, n, replace=False).astype(np.int32)))
    for t in tickets:
        srv.result(t)
    srv.close()
    print("ncu-foldin done")


# ----------------------------------------------------------------- fold-in serving
FOLDIN_DESC = ("fold-in: frozen H 41,000 x 256 ~ N(0, 0.05^2), b=64, 4 sweeps, alpha0=0.1, "
               "lambda=1e-3, nu=1; open loop: Poisson arrivals at each rate; closed loop: C "
               "clients, one request outstanding each; history lengths log-uniform on "
               "[1, 5000] over Zipf(1.0) items; 4 GB workspace")


def foldin_requests(rng, n_items, n_req, cdf):
    """History lengths log-uniform on [1, 5000] over Zipf(1.0) items (distinct per request)."""
    lens = np.exp(rng.uniform(0.0, np.log(5000.0), n_req)).astype(np.int64)
    reqs = []
    for n in lens:
        draw = np.unique(np.minimum(np.searchsorted(cdf, rng.random(2 * n + 8)), n_items - 1))
        reqs.append(rng.permutation(draw)[:n].astype(np.int32))
    return reqs


def run_foldin(rates=(2000, 5000, 10000, 20000, 50000), n_req=3000, closed_clients=(16, 128),
               cpu_sample=0, seed=0):
    """Fold-in serving.  Open loop: Poisson arrivals at each rate, latency = submit ->
    result in host memory (measured inside the library).  Closed loop: C clients that
    each submit their next request when the previous result arrives.  Optionally the
    FP64 oracle's per-request latency on a sample of the same requests (host cores)."""
    import threading
    import paper_2110_14044_gb300 as ials
    from paper_2110_14044_gb300 import _abi
    rng = np.random.Generator(np.random.Philox(key=[seed, 7]))
    n_items, d, b, sweeps = 41000, 256, 64, 4
    alpha0, lam, nu = 0.1, 1e-3, 1.0
    H = rng.normal(0.0, 0.05, (n_items, d)).astype(np.float32)
    ranks = np.arange(1, n_items + 1, dtype=np.float64)
    p = ranks ** -1.0
    p /= p.sum()
    perm = rng.permutation(n_items)
    cdf = np.cumsum(p[np.argsort(perm)])
    cdf[-1] = 1.0
    srv = ials.FoldinServer(H, d, b, alpha0, lam, nu, sweeps=sweeps, workspace_bytes=4 << 30)
    out = {"desc": FOLDIN_DESC, "rates": [], "closed_loop": []}
    for rate in rates:
        reqs = foldin_requests(rng, n_items, n_req, cdf)
        lens = np.array([r.size for r in reqs])
        sched = np.cumsum(rng.exponential(1.0 / rate, n_req))
        lat = np.zeros(n_req)
        done_t = np.zeros(n_req)
        tickets = [0] * n_req
        ready = threading.Event()

        def collector():
            ready.wait()
            w = np.empty(d, np.float32)
            for k in range(n_req):
                while tickets[k] == 0:
                    time.sleep(0)
                while True:
                    st, us = _abi.ials_foldin_poll_timed(srv.srv, tickets[k], w, 2000)
                    if st == _abi.OK or st == _abi.ENOTPD:
                        break
                lat[k] = us / 1e3
                done_t[k] = time.perf_counter()

        th = threading.Thread(target=collector)
        th.start()
        t0 = time.perf_counter()
        ready.set()
        for k in range(n_req):
            while time.perf_counter() - t0 < sched[k]:
                pass
            tickets[k] = srv.submit(reqs[k])
        th.join()
        span = done_t.max() - t0
        out["rates"].append({"offered_req_s": rate, "achieved_req_s": n_req / span,
                             "p50_ms": float(np.percentile(lat, 50)),
                             "p99_ms": float(np.percentile(lat, 99)), "requests": n_req,
                             "mean_len": float(lens.mean())})
    for clients in closed_clients:
        reqs = foldin_requests(rng, n_items, n_req, cdf)
        lat = np.zeros(n_req)
        nxt = [0]
        lock = threading.Lock()

        def client():
            w = np.empty(d, np.float32)
            while True:
                with lock:
                    k = nxt[0]
                    nxt[0] += 1
                if k >= n_req:
                    return
                t = srv.submit(reqs[k])
                while True:
                    st, us = _abi.ials_foldin_poll_timed(srv.srv, t, w, 2000)
                    if st == _abi.OK or st == _abi.ENOTPD:
                        break
                lat[k] = us / 1e3

        ths = [threading.Thread(target=client) for _ in range(clients)]
        t0 = time.perf_counter()
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        span = time.perf_counter() - t0
        out["closed_loop"].append({"clients": clients, "achieved_req_s": n_req / span,
                                   "p50_ms": float(np.percentile(lat, 50)),
                                   "p99_ms": float(np.percentile(lat, 99)), "requests": n_req})
    srv.close()
    if cpu_sample:
        import oracle
        reqs = foldin_requests(rng, n_items, cpu_sample, cdf)
        G = oracle.gramian(H)  # formed once, as the server does
        ms = []
        for items in reqs:
            t0 = time.perf_counter()
            oracle.foldin(H, d, b, alpha0, lam, nu, sweeps, items, G=G)
            ms.append((time.perf_counter() - t0) * 1e3)
        out["cpu_oracle"] = {"kind": "oracle", "requests": cpu_sample, "cores": 1,
                             "p50_ms": float(np.percentile(ms, 50)),
                             "p99_ms": float(np.percentile(ms, 99)),
                             "mean_len": float(np.mean([r.size for r in reqs])),
                             "note": "FP64 oracle, one request at a time, one thread, G^I = H^T H "
                                     "formed once beforehand (as the server does)"}
    return out


def overrides(args):
    o = {}
    if args.d:
        o["d"] = args.d
    if args.b:
        o["b"] = args.b
    return o


def describe(args, prob):
    desc = WORKLOADS[args.workload]
    if args.d or args.b:
        desc += f" (overridden: d={prob.d}, b={prob.b})"
    return desc


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--d", type=int, default=0, help="override the embedding dimension")
    ap.add_argument("--b", type=int, default=0, help="override the block size")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16"])
    ap.add_argument("--no-variants", dest="variants", action="store_false",
                    help="do not also time the other precision")
    ap.add_argument("--no-foldin", dest="foldin", action="store_false",
                    help="do not run the fold-in serving measurement")
    ap.add_argument("--autotune", action="store_true",
                    help="also time every admissible block size per precision (b sweep)")
    ap.add_argument("--convergence", type=int, default=None, metavar="E",
                    help="record the objective over E epochs for every admissible b (0: skip; "
                         "default 6 on the default workload, else 0)")
    ap.add_argument("--no-sweep", dest="sweep", action="store_false",
                    help="do not run the skewed-activity d x b sweep")
    ap.add_argument("--no-d1024", dest="d1024", action="store_false",
                    help="do not also measure the MSD-shaped d = 1024 workload")
    ap.add_argument("--d1024-steps", type=int, default=3,
                    help="timed epochs per configuration of the d = 1024 workload")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ncu-frac", type=float, default=1.0,
                    help="with --ncu-step: use this fraction of the workload's users and positives")
    ap.add_argument("--ncu-step", action="store_true",
                    help="run one user and one item block step only (for profiler captures)")
    ap.add_argument("--ncu-foldin", action="store_true",
                    help="serve a few fold-in requests only (for profiler captures)")
    args = ap.parse_args()
    if args.ncu_step:
        run_ncu_step(args)
    elif args.ncu_foldin:
        run_ncu_foldin()
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
