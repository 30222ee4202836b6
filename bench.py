#!/usr/bin/env python3
"""Benchmark: modular coefficient MACs/s of dense polynomial multiplication
mod p = 469762049 on one GB300.  Parity with the CPU oracle is the tests'
job; here the oracle runs only in the cpu_baseline legs (which also compare
their products with the GPU's results word for word) and in the reference
arm, and every other result is cross-checked on the GPU (tensor-core against
plain, plain against transform, graph against direct, a division against
a = q b + r, a gcd against its planted factor, a transform product at a
random point).

Headline step: the batched tensor-core product of 1024 pairs of degree 4095
(1024 * 4096^2 = 1.72e10 modular multiply-adds), one polymul_batched call
with PM_TENSOR (a planning launch and one persistent tcgen05 kernel).  Each
timed step is bracketed by CUDA events on the launching stream and preceded
by a 256 MiB write that flushes the 129 MB L2 (outside the events).  The
roofline is the tensor one: the bf16 limb products of the encoding per modular MAC (2 flops
each) over the measured bf16 peak.  The one-pair degree-16383 product of
the s-blocked plain kernel (the paper's Section 5 form) is the row
`plain_single`, with its own ALU roofline, e2e and CPU baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-rows]

Prints one JSON line.  With N > 1 (torchrun) every rank runs its own replica
of the step (the work is not sharded here) and rank 0 reports the job total
over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1402_0264_gb300 import inputs  # noqa: E402

P = inputs.P_DEFAULT
METRIC = "modular coefficient MACs/s (n*m per product), bit-exact vs oracle"
UNIT = "MAC/s"
BATCH_T, DEG_T = 1024, 4095
MACS_T = BATCH_T * (DEG_T + 1) ** 2        # 1.718e10 modular multiply-adds per step
WORKLOAD = ("batched tensor-core polymul mod p=469762049: 1024 pairs of degree 4095, uint32 coefficients "
            "uniform in [0,p), bf16 limbs on tcgen05 with exact fp32 accumulation and a fused mod-p epilogue")
N_SINGLE = 16384
MACS_SINGLE = N_SINGLE * N_SINGLE
WORKLOAD_SINGLE = "plain polymul mod p=469762049, one pair of degree 16383, uint32 coefficients uniform in [0,p)"
FLUSH_BYTES = 256 << 20
SMS = 152
IMAD_PER_CLK_SM = 32      # nominal 32x32->64 multiply-add issue rate (half the 32-bit IMAD rate); the bench measures it
SM_MAX_MHZ = 2070.0
L2_NOTE = "flushed between steps (256 MiB write outside the timed events)"


def headline_config(world: int) -> dict:
    return {"workload": WORKLOAD, "batch": BATCH_T, "deg": DEG_T, "p": P, "mode": "PM_TENSOR",
            "parallelism": "replicas" if world > 1 else "single", "l2": L2_NOTE}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return pk, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": SM_MAX_MHZ}, "fallback"


def alu_peak_macs(rate=IMAD_PER_CLK_SM, mhz=SM_MAX_MHZ):
    """Plain-path ceiling: one 32x32->64 multiply-add per modular MAC, `rate` per SM per clock."""
    return SMS * rate * mhz * 1e6


def source_hash(*names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_1402_0264_gb300", "csrc", n), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_for(kernel: str, *src: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel is unchanged since."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            t = json.load(fh)
    except OSError:
        return None
    ent = t.get(kernel)
    if not ent or ent.get("source_sha") != source_hash(*src):
        return None
    return ent.get("bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    def __init__(self, index):
        self.index = index  # nvidia-smi --id value (UUID of the CUDA device)
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.15)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        mhz = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(mhz) if mhz else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    # NCCL reduces device tensors; gloo (the reference arm, CPU tests) host ones
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def division_model_ratio(n: int, m: int, s: int, ell: int, U: float) -> float:
    """T_1 / T_s of Section 3 (Corollary 1 with K_1 = m / l, K_s = m / (2 s)): the naive division
    (N_1 / K_1 = n - m + 1, L_1 = n - m + 1, C_1 = 3 + 5U) over the optimized one
    (N_s = (n - m + 1) m / (2 s^2), L_s = (n - m + 1) / s, C_s = 3 s + 9 U); a has n terms, b m."""
    mu = n - m + 1
    t1 = (mu * m / ell / (m / ell) + mu) * (3 + 5 * U)
    ts = (mu * m / (2 * s * s) / (m / (2 * s)) + mu / s) * (3 * s + 9 * U)
    return t1 / ts


def gcd_model_ratio(n: int, m: int, s: int, ell: int, U: float) -> float:
    """T_1 / T_s of Section 6 (Corollary 1 with K_1 = m / l, K_s = m / s): the naive gcd
    (N_1 = m (n + l + 1) / l, L_1 = n + m - 2, C_1 = 3 + 5U) over the optimized one
    (N_s = m n / s^2 + m / s, L_s = (n + m) / s, C_s = 3 s + 8 U); a has n terms, b m."""
    t1 = (m * (n + ell + 1) / ell / (m / ell) + n + m - 2) * (3 + 5 * U)
    ts = ((m * n / (s * s) + m / s) / (m / s) + (n + m) / s) * (3 * s + 8 * U)
    return t1 / ts


def fit_model_U(model_predict, points, n: int, m: int, P: float, rate: float, mhz: float) -> dict:
    """Calibrates the model's U on measured times (the paper's U is a machine parameter
    it leaves unvalued).  points: (s, l, ms) of one product with a n-term a and a m-term b.
    The model's time is T_thm of Theorem 1 in units of one local operation of a block
    (l / (rate * clock) seconds); the measured time is taken as kappa * T_thm, and U and
    kappa minimise the squared error of log(time) over the points (U on a log grid from 1/4
    to 64, kappa in closed form for each U).  Returns U, kappa, the rms log error and the
    s the fitted model picks for each l."""
    clk = mhz * 1e6
    grid = [0.25 * 2 ** (i / 16) for i in range(16 * 8 + 1)]
    best = None
    for U in grid:
        lp = [math.log(model_predict(n, m, s, ell, U, P)["T_thm"] * ell / (rate * clk)) for s, ell, _ in points]
        lm = [math.log(ms * 1e-3) for _, _, ms in points]
        lk = sum(b - a for a, b in zip(lp, lm)) / len(lp)
        err = math.sqrt(sum((b - a - lk) ** 2 for a, b in zip(lp, lm)) / len(lp))
        if best is None or err < best[0]:
            best = (err, U, math.exp(lk))
    err, U, kappa = best
    picks = {}
    for ell in sorted({e for _, e, _ in points}):
        ss = [s for s, e, _ in points if e == ell]
        picks[str(ell)] = min(ss, key=lambda s_: model_predict(n, m, s_, ell, U, P)["T_thm"])
    return {"U_fit": U, "kappa": kappa, "rms_log_err": err, "best_s_fitted": picks}


def eval_mod(poly, r: int, p: int) -> int:
    """poly(r) mod p on the host with numpy (a spot check of a product: c(r) = a(r) b(r) mod p
    for a product c = a b, the Schwartz-Zippel test).  Powers r^i as r^(i mod B) (r^B)^(i div B)."""
    c = np.asarray(poly, dtype=np.uint64)
    B = 4096
    pw = np.empty(B, dtype=np.uint64)
    pw[0] = 1
    for i in range(1, B):
        pw[i] = pw[i - 1] * r % p
    rb = int(pw[-1]) * r % p
    nb = (len(c) + B - 1) // B
    blk = np.empty(nb, dtype=np.uint64)
    blk[0] = 1
    for j in range(1, nb):
        blk[j] = blk[j - 1] * rb % p
    idx = np.arange(len(c))
    w = pw[idx % B] * blk[idx // B] % p
    return int((c * w % p).sum() % p)


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle as it stands
# ---------------------------------------------------------------------------

def run_reference(args, world, rank):
    """The oracle on the host cores: the 1024 pairs of degree 4095 by the long-multiplication
    definition, the pairs shared out over all host threads (OpenMP).  Each step is the whole
    batch when K+W of them fit in about two minutes, else the first `pairs` pairs of it (a
    bounded sample of the same workload; the MAC count is that of the pairs done)."""
    if rank != 0:
        return 0
    import oracle
    tp = inputs.workload_tensor()
    a_data, a_off, b_data, b_off, c_off = tp
    threads = oracle.omp_threads()
    t0 = time.perf_counter()
    oracle.polymul_batch_omp(a_data, a_off[:9], b_data, b_off[:9], c_off[:9], P)  # build, load, time 8 pairs
    t8 = time.perf_counter() - t0
    budget = 120.0 / max(1, args.steps + args.warmup)
    pairs = BATCH_T if t8 / 8 * BATCH_T <= budget else max(threads, int(budget / (t8 / 8)) // threads * threads)
    pairs = min(pairs, BATCH_T)
    sub = (a_data, a_off[:pairs + 1], b_data, b_off[:pairs + 1], c_off[:pairs + 1])
    for _ in range(args.warmup):
        oracle.polymul_batch_omp(*sub, P)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.polymul_batch_omp(*sub, P)
    dt = time.perf_counter() - t0
    macs = pairs * (DEG_T + 1) ** 2
    value = macs * args.steps / dt
    sample = (f"{args.steps} runs of the whole batch" if pairs == BATCH_T else
              f"{args.steps} runs of the first {pairs} of the 1024 pairs")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": headline_config(world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "cpu": cpu_model(),
                             "sample": sample + " (C schoolbook with 128-bit accumulation, pairs over "
                                                f"{threads} OpenMP threads)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def tc_issued_flops(a_off, b_off, enc: dict) -> float:
    """bf16 flops the tensor kernel issues for a batch (padding included): per tile of
    32 tile_blocks outputs and per shift it meets (K-groups included), 2 MMAs of 128 x N x 16 with
    N = tile_blocks * na, the tile's full width."""
    nb_t = enc["tile_blocks"]
    n_all = np.diff(a_off)
    m_all = np.diff(b_off)
    tot = 0
    for n_, m_ in zip(n_all.tolist(), m_all.tolist()):
        if m_ > n_:
            n_, m_ = m_, n_
        na = (n_ + 31) // 32
        dmax = (m_ + 30) // 32
        for t_ in range((n_ + m_ - 1 + 32 * nb_t - 1) // (32 * nb_t)):
            I0 = nb_t * t_
            tot += min(dmax, I0 + nb_t - 1) - max(0, I0 - na + 1) + 1
    return float(tot) * 2 * 2 * 128 * 16 * nb_t * enc["na"]


def run_ours(args, world, rank, local):
    import torch

    from paper_1402_0264_gb300 import build as pbuild
    from paper_1402_0264_gb300 import polymul as pm

    if not os.path.exists(pm.LIB_PATH):
        pbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    flush_buf = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def flush():
        flush_buf.zero_()

    tp = inputs.workload_tensor()
    tt = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in tp]
    total = int(tp[4][-1])
    out = torch.empty(total, dtype=torch.uint32, device=dev)

    def step():
        pm.batched(tt[0], tt[1], tt[2], tt[3], tt[4], max_deg=DEG_T, mode=pm.PM_TENSOR, out=out, total=total)

    # warm-up; the warmed result agrees with the plain CUDA-core form on the same batch (the oracle
    # itself runs in the cpu_baseline leg below, which also checks this result word for word)
    for _ in range(args.warmup):
        step()
    plain_out = pm.batched(tt[0], tt[1], tt[2], tt[3], tt[4], max_deg=DEG_T, mode=pm.PM_PLAIN, s=8, total=total)
    torch.cuda.synchronize()
    assert torch.equal(out, plain_out), "bench: the tensor-core and plain forms disagree"
    del plain_out
    assert pm.sync_status() == 0

    K = args.steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    launches0 = pm.launch_count()
    try:
        smi_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        smi_id = str(local)
    sampler = ClockSampler(smi_id)
    with sampler:
        barrier(world)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for i in range(K):
            flush()
            starts[i].record(stream)
            step()
            ends[i].record(stream)
        torch.cuda.synchronize()
        barrier(world)
        wall = time.perf_counter() - w0
    launches = pm.launch_count() - launches0
    clocks = sampler.summary()
    step_ms = [s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)]
    total_ms = max_over_ranks(sum(step_ms), world)
    value = world * MACS_T * K / (total_ms * 1e-3)
    ms_per_step = total_ms / K
    assert pm.sync_status() == 0

    # end to end through the C ABI from pinned host buffers (polymul_batched_host): every step
    # copies its inputs (both coefficient arrays and the three offset arrays) in, runs the product
    # and copies the 1024 products out, all inside the events; the library cuts the batch into
    # chunks whose copies overlap the products of the others
    hosts = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in tp]
    out_h = torch.empty(total, dtype=torch.uint32).pin_memory()
    e2e_step = lambda: pm.batched_host(*hosts, out_h, max_deg=DEG_T, mode=pm.PM_TENSOR, stream=stream)
    for _ in range(max(1, args.warmup)):
        e2e_step()
    e_starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    e_ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    barrier(world)
    torch.cuda.synchronize()
    for i in range(K):
        flush()
        e_starts[i].record(stream)
        e2e_step()
        e_ends[i].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    e2e_ms = max_over_ranks(sum(s_.elapsed_time(e_) for s_, e_ in zip(e_starts, e_ends)), world)
    assert pm.sync_status() == 0
    gpu_result = out_h.numpy().view(np.uint32).copy()
    assert np.array_equal(gpu_result, out.cpu().numpy().view(np.uint32)), \
        "bench: the host-buffer products differ from the device result"

    if rank != 0:
        return 0

    pk, pk_kind = peaks()
    enc = pm.tensor_limbs()
    achieved = MACS_T * 2 * enc["limb_products"] / (ms_per_step * 1e-3) / 1e12
    issued = tc_issued_flops(tp[1], tp[3], enc) / (ms_per_step * 1e-3) / 1e12
    peak = pk["bf16_tflops"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "products_per_s": value / MACS_T * BATCH_T,
        "config": headline_config(world),
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "peak_basis": f"measured bf16 dense GEMM, burst ({pk_kind}): the step is one short "
                                   "kernel timed alone",
                     "achieved_basis": f"useful work only: {enc['limb_products']} bf16 limb products "
                                       f"({2 * enc['limb_products']} flops) per modular MAC ({enc['na']} balanced "
                                       f"base-{enc['base_a']} limbs of a x {enc['nb']} base-{enc['base_b']} limbs "
                                       "of b), n*m MACs per pair, no tile padding; over the CUDA-event time of "
                                       "the whole call (planning launch included)",
                     "encoding": enc,
                     "issued_tflops": issued, "issued_frac": issued / peak,
                     "kernel": "tc_batched_kernel",
                     "traffic": traffic_for("tc_batched_kernel", "tensor.cu", "common.cuh")},
        "e2e": {"value": world * MACS_T * K / (e2e_ms * 1e-3), "unit": UNIT,
                "basis": "polymul_batched_host from pinned host buffers, copies in and out inside the events",
                "ms_per_step": e2e_ms / K,
                "h2d_bytes_per_step": int(sum(h_.numel() * h_.element_size() for h_ in hosts)),
                "d2h_bytes_per_step": int(out_h.numel() * 4)},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "wall_s_timed_region": wall,
        "peaks_source": pk_kind,
    }
    if world == 1 and not args.no_rows:
        line["rows"] = measure_rows(pm, torch, dev, flush, clocks, pk, args)
        line["vs_plain_same_batch"] = line["rows"]["tensor_vs_plain"]
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_batch(tp, gpu_result)
    print(json.dumps(line), flush=True)
    return 0


def median_ms(fn, reps, flush, stream):
    import torch
    ts = []
    for _ in range(reps):
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def measure_rows(pm, torch, dev, flush, clocks, pk, args):
    stream = torch.cuda.current_stream()
    rows = {}
    mhz = clocks.get("sm_mhz") or SM_MAX_MHZ

    # --- the ceiling of the plain path, measured: 32x32->64 multiply-adds per clock per SM ---
    # (the roofline's peak is the unit-count figure, 32 per clock per SM: never below the measured rate)
    rate = pm.probe_mac_rate(threads=256, blocks_per_sm=4, iters=20000)
    mhz_max = pk.get("sm_max_mhz") or SM_MAX_MHZ
    alu_peak = alu_peak_macs(max(IMAD_PER_CLK_SM, rate), mhz_max)
    rows["alu_probe"] = {"imad_wide_per_clk_per_sm": rate, "nominal_per_clk_per_sm": IMAD_PER_CLK_SM, "sms": SMS,
                         "sm_max_mhz": mhz_max, "measured_peak_macs_per_s": alu_peak_macs(rate, mhz_max),
                         "peak_macs_per_s": alu_peak,
                         "how": "polymul_probe_mac_rate: 4 x 152 blocks of 256 threads, 16 independent "
                                "64-bit sums per thread, per-SM cycle counters around the loops"}

    # --- the one-pair degree-16383 product of the s-blocked kernel (Section 5), tuned s ---
    rows["plain_single"] = plain_single_row(pm, torch, dev, flush, stream, alu_peak, rate, pk, args)
    rows["plain_single"]["roofline"]["frac_of_measured_rate"] = (rows["plain_single"]["macs_per_s"] /
                                                                 alu_peak_macs(rate, mhz_max))

    # --- s sweep on the degree-16383 pair with the cost model beside each point ---
    a_np, b_np = inputs.workload_single()
    a = torch.from_numpy(a_np).to(dev)
    b = torch.from_numpy(b_np).to(dev)
    c = torch.empty(2 * N_SINGLE - 1, dtype=torch.uint32, device=dev)
    ell = 256
    # U: time to move one 4-byte word per SM (HBM share) over the time of one
    # local multiply-add, both per SM: (ops/clk/SM * 4 B * clk * SMs) / (HBM bytes/s),
    # with the multiply-add rate measured by the probe above
    U = 4.0 * rate * SM_MAX_MHZ * 1e6 * SMS / (pk["hbm_gbs"] * 1e9)
    unit_s = ell / (rate * SM_MAX_MHZ * 1e6)         # one local op of a whole block
    sweep = []
    for s in pm.S_CANDIDATES:
        ms = median_ms(lambda: pm.plain(a, b, s=s, out=c), 20, flush, stream)
        pred = pm.model_predict(N_SINGLE, N_SINGLE, s, ell, U, float(SMS))
        sweep.append({"s": s, "ms": ms, "macs_per_s": MACS_SINGLE / (ms * 1e-3),
                      "alu_frac": MACS_SINGLE / (ms * 1e-3) / alu_peak,
                      "model_T_thm_s": pred["T_thm"] * unit_s, "model_T_cor_s": pred["T_cor"] * unit_s,
                      "model_W": pred["W"], "model_O": pred["O"]})
    rows["plain_s_sweep"] = {"workload": "degree-16383 pair", "ell": ell, "U": U, "P": SMS,
                             "time_unit_s": unit_s, "points": sweep,
                             "best_measured_s": min(sweep, key=lambda r: r["ms"])["s"],
                             "best_thm_s": min(sweep, key=lambda r: r["model_T_thm_s"])["s"],
                             "best_cor_s": min(sweep, key=lambda r: r["model_T_cor_s"])["s"]}

    # --- block-size study: l = 128 and 512 threads per block beside l = 256 ---
    ell_rows = {256: [{"s": r["s"], "ms": r["ms"], "model_T_thm_s": r["model_T_thm_s"],
                       "model_T_cor_s": r["model_T_cor_s"]} for r in sweep]}
    ref = c.clone()
    for el in (128, 512):
        u_el = el / (rate * SM_MAX_MHZ * 1e6)
        pts = []
        for s in pm.S_CANDIDATES:
            ms = median_ms(lambda: pm.plain_ell(a, b, s, el, out=c), 20, flush, stream)
            assert torch.equal(c, ref), f"l = {el}, s = {s} disagrees with l = 256"
            pred = pm.model_predict(N_SINGLE, N_SINGLE, s, el, U, float(SMS))
            pts.append({"s": s, "ms": ms, "model_T_thm_s": pred["T_thm"] * u_el,
                        "model_T_cor_s": pred["T_cor"] * u_el})
        ell_rows[el] = pts
    best = {el: min(p_, key=lambda r: r["ms"]) for el, p_ in ell_rows.items()}
    rows["plain_ell_study"] = {
        "workload": "degree-16383 pair", "U": U, "P": SMS,
        "points": {str(el): p_ for el, p_ in ell_rows.items()},
        "best_measured": {str(el): {"s": r["s"], "ms": r["ms"]} for el, r in best.items()},
        "best_thm": {str(el): min(p_, key=lambda r: r["model_T_thm_s"])["s"] for el, p_ in ell_rows.items()}}
    # U calibrated on the 21 measured points of the study (the derived U beside it)
    fit = fit_model_U(pm.model_predict, [(r["s"], el, r["ms"]) for el, p_ in ell_rows.items() for r in p_],
                      N_SINGLE, N_SINGLE, float(SMS), rate, SM_MAX_MHZ)
    fit["U_derived"] = U
    rows["plain_ell_study"]["model_fit"] = fit

    # --- degree-1023 pair (latency bound) ---
    a0, b0 = inputs.workload_small()
    da0, db0 = torch.from_numpy(a0).to(dev), torch.from_numpy(b0).to(dev)
    c0 = torch.empty(2047, dtype=torch.uint32, device=dev)
    s0 = pm.tune_plain(da0, db0, reps=10, out=c0)[0]
    ms0 = median_ms(lambda: pm.plain(da0, db0, s=s0, out=c0), 50, flush, stream)
    assert torch.equal(c0, pm.ntt(da0, db0)), "plain and transform paths disagree"
    rows["plain_small"] = {"workload": "degree-1023 pair", "s": s0, "ms": ms0,
                           "macs_per_s": 1024 * 1024 / (ms0 * 1e-3)}

    # --- batched: 4096 pairs, degrees log-uniform in [16, 2048], one graph launch; (s, Q) by the autotuner ---
    packed = inputs.workload_batched()
    a_data, a_off, b_data, b_off, c_off = packed
    na_ = a_off[1:] - a_off[:-1]
    nb_ = b_off[1:] - b_off[:-1]
    macs = int((na_ * nb_).sum())
    ta = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in packed]
    outb = torch.empty(int(c_off[-1]), dtype=torch.uint32, device=dev)
    s_b, q_b, tune_b = pm.tune_batched(ta[0], ta[1], ta[2], ta[3], ta[4], max_deg=2048, reps=10, out=outb,
                                       total=outb.numel())
    # the model of Section 5 for the batch (Theorem 1 over all pairs' thread-blocks: N = sum of N_s,
    # the span the longest pair's), in the time unit of one local operation of a block
    model_b = {}
    for s in sorted({sv for sv, _ in tune_b}):
        n_tot, l_max, c_s = 0.0, 0.0, 0.0
        for n_i, m_i in zip(na_.tolist(), nb_.tolist()):
            nn_, mm_ = max(n_i, m_i), min(n_i, m_i)
            if s > mm_:
                continue
            pr = pm.model_predict(nn_, mm_, s, 256, 4.0 * rate * SM_MAX_MHZ * 1e6 * SMS / (pk["hbm_gbs"] * 1e9),
                                  float(SMS))
            n_tot += pr["N"]
            l_max = max(l_max, pr["L"])
            c_s = pr["C"]
        model_b[s] = (n_tot / SMS + l_max) * c_s * 256 / (rate * SM_MAX_MHZ * 1e6)
    run_b = lambda: pm.batched(ta[0], ta[1], ta[2], ta[3], ta[4], max_deg=2048, mode=pm.PM_PLAIN, s=0, out=outb,
                               total=outb.numel())
    run_b()
    ms_direct = median_ms(run_b, 20, flush, stream)
    g = torch.cuda.CUDAGraph()
    gs = torch.cuda.Stream()
    with torch.cuda.stream(gs):
        pm.batched(ta[0], ta[1], ta[2], ta[3], ta[4], max_deg=2048, mode=pm.PM_PLAIN, s=0, out=outb,
                   total=outb.numel(), stream=gs)
        gs.synchronize()
        with torch.cuda.graph(g, stream=gs):
            pm.batched(ta[0], ta[1], ta[2], ta[3], ta[4], max_deg=2048, mode=pm.PM_PLAIN, s=0,
                       out=outb, total=outb.numel(), stream=gs)
    ms_g = median_ms(g.replay, 20, flush, stream)
    want = outb.clone()  # the graph replay's result; the forms below must agree with it
    # the tensor-core form on the whole batch
    run_bt = lambda: pm.batched(ta[0], ta[1], ta[2], ta[3], ta[4], max_deg=2048, mode=pm.PM_TENSOR, out=outb,
                                total=outb.numel())
    run_bt()
    ms_bt = median_ms(run_bt, 10, flush, stream)
    assert torch.equal(outb, want), "batched: tensor and plain forms disagree"
    # PM_AUTO: each pair by its size (shorter operand of 128 terms or more to the tensor cores)
    run_ba = lambda: pm.batched(ta[0], ta[1], ta[2], ta[3], ta[4], max_deg=2048, mode=pm.PM_AUTO, out=outb,
                                total=outb.numel())
    run_ba()
    ms_ba = median_ms(run_ba, 20, flush, stream)
    assert torch.equal(outb, want), "batched: PM_AUTO and the plain form disagree"
    rows["batched_plain"] = {"workload": "4096 pairs, degrees log-uniform in [16,2048]", "s": s_b, "q": q_b,
                             "form": "warp-level units (degrees below 4096)",
                             "tuner": "polymul_tune_batched: flushed medians of 10 calls per (s, Q)",
                             "sweep": [{"s": sv, "q": qv, "ms": ms_, "macs_per_s": macs / (ms_ * 1e-3),
                                        "model_T_thm_s": model_b.get(sv)}
                                       for (sv, qv), ms_ in sorted(tune_b.items())],
                             "tensor_form_ms_same_batch": ms_bt,
                             "auto_ms_same_batch": ms_ba, "auto_macs_per_s": macs / (ms_ba * 1e-3),
                             "auto_form": "PM_AUTO: pairs whose shorter operand has >= 128 terms on the tensor "
                                          "cores, the others on the warp-level plain form",
                             "macs": macs, "ms_graph": ms_g, "ms_direct": ms_direct,
                             "macs_per_s": macs / (ms_g * 1e-3), "products_per_s": 4096 / (ms_g * 1e-3),
                             "alu_frac": macs / (ms_g * 1e-3) / alu_peak}
    del ta, outb, want

    # --- the headline batch through the plain CUDA-core form (the comparison the tensor form must win) ---
    tp = inputs.workload_tensor()
    macs_t = int(((tp[1][1:] - tp[1][:-1]) * (tp[3][1:] - tp[3][:-1])).sum())
    tt = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in tp]
    outt = torch.empty(int(tp[4][-1]), dtype=torch.uint32, device=dev)
    run_t = lambda: pm.batched(tt[0], tt[1], tt[2], tt[3], tt[4], max_deg=4095, mode=pm.PM_TENSOR,
                               out=outt, total=outt.numel())
    run_t()
    ms_t = median_ms(run_t, 10, flush, stream)
    want_t = outt.clone()
    run_tp = lambda: pm.batched(tt[0], tt[1], tt[2], tt[3], tt[4], max_deg=4095, mode=pm.PM_PLAIN, s=8,
                                out=outt, total=outt.numel())
    run_tp()
    ms_tp = median_ms(run_tp, 5, flush, stream)
    assert torch.equal(outt, want_t), "tensor and plain forms disagree on the 1024-pair batch"
    rows["tensor_vs_plain"] = {"workload": "1024 pairs of degree 4095", "macs": macs_t, "tensor_ms": ms_t,
                               "tensor_macs_per_s": macs_t / (ms_t * 1e-3), "plain_s8_ms": ms_tp,
                               "plain_s8_macs_per_s": macs_t / (ms_tp * 1e-3),
                               "plain_s8_alu_frac": macs_t / (ms_tp * 1e-3) / alu_peak,
                               "speedup_tensor_over_plain": ms_tp / ms_t}
    del tt, outt, want_t

    # --- transform path: one pair of degree 2^22 - 1, and the plain/transform crossover ---
    an, bn = inputs.workload_ntt()
    dan, dbn = torch.from_numpy(an).to(dev), torch.from_numpy(bn).to(dev)
    cn = torch.empty(2 * len(an) - 1, dtype=torch.uint32, device=dev)
    pm.ntt(dan, dbn, out=cn)
    ms_n = median_ms(lambda: pm.ntt(dan, dbn, out=cn), 20, flush, stream)
    rr = 123456789  # c(r) = a(r) b(r) mod p at a fixed point (Schwartz-Zippel)
    assert eval_mod(cn.cpu().numpy(), rr, P) == eval_mod(an, rr, P) * eval_mod(bn, rr, P) % P
    nn = len(an)
    algo_bytes = 4 * (2 * nn + 2 * nn - 1)  # read a and b, write c
    rows["ntt"] = {"workload": "one pair of degree 2^22-1 (transform length 2^23)", "ms": ms_n,
                   "schoolbook_equiv_macs_per_s": nn * nn / (ms_n * 1e-3),
                   "products_per_s": 1.0 / (ms_n * 1e-3),
                   "algorithmic_bytes": algo_bytes,
                   "algorithmic_gbs": algo_bytes / (ms_n * 1e-3) / 1e9,
                   "hbm_frac_algorithmic": algo_bytes / (ms_n * 1e-3) / 1e9 / pk["hbm_gbs"]}
    sweep = []
    for logn in range(10, 23):
        n_ = 1 << logn
        a_, b_ = inputs.workload_ntt(deg=n_ - 1, seed=inputs.SEED_BASE + 40 + logn)
        da_, db_ = torch.from_numpy(a_).to(dev), torch.from_numpy(b_).to(dev)
        c_ = torch.empty(2 * n_ - 1, dtype=torch.uint32, device=dev)
        pm.ntt(da_, db_, out=c_)
        t_ntt = median_ms(lambda: pm.ntt(da_, db_, out=c_), 7, flush, stream)
        t_plain = None
        if logn <= 18:
            pm.plain(da_, db_, s=8, out=c_)
            t_plain = median_ms(lambda: pm.plain(da_, db_, s=8, out=c_), 5 if logn <= 16 else 3, flush, stream)
        sweep.append({"deg": n_ - 1, "ms_ntt": t_ntt, "ms_plain_s8": t_plain})
    cross = next((r["deg"] for r in sweep if r["ms_plain_s8"] is not None and r["ms_ntt"] < r["ms_plain_s8"]), None)
    rows["ntt_crossover"] = {"points": sweep, "first_deg_where_ntt_wins": cross}
    # --- division (Section 3, Algorithms 3-4): a of degree 32767 by b of degree 16383 ---
    def division_holds(a_t, b_t, q_t, r_t):
        """a == q b + r, with the product from the library's own plain path."""
        qb = pm.plain(q_t, b_t).cpu().numpy().astype(np.uint64)
        qb[: r_t.numel()] = (qb[: r_t.numel()] + r_t.cpu().numpy().astype(np.uint64)) % P
        return np.array_equal(qb.astype(np.uint32), a_t.cpu().numpy())

    ad, bd = inputs.poly_pair(32767, 16383, inputs.SEED_BASE + 5)
    if bd[-1] == 0:
        bd[-1] = 1
    ta_d, tb_d = torch.from_numpy(ad).to(dev), torch.from_numpy(bd).to(dev)
    qd = torch.empty(len(ad) - len(bd) + 1, dtype=torch.uint32, device=dev)
    rd = torch.empty(len(bd) - 1, dtype=torch.uint32, device=dev)
    n_d, m_d = len(ad), len(bd)
    work_d = (n_d - m_d + 1) * m_d  # one multiply-subtract per coefficient of b per step
    sweep = []
    for s_d in (32, 64, 128, 256):
        pm.divide(ta_d, tb_d, s=s_d, q=qd, r=rd)
        ms = median_ms(lambda s_d=s_d: pm.divide(ta_d, tb_d, s=s_d, q=qd, r=rd), 5, flush, stream)
        assert pm.sync_status() == 0 and division_holds(ta_d, tb_d, qd, rd), f"division s={s_d}: a != q b + r"
        sweep.append({"s": s_d, "ms": ms, "launches": 1 + -(-(n_d - m_d + 1) // s_d),
                      "mac_per_s": work_d / (ms * 1e-3)})
    # s = 1 (the naive division, one step per launch) against s = 256 on a smaller pair, with the
    # paper's running-time ratio R = T_1 / T_s of Section 3 (Corollary 1, K_1 = m / l, K_s = m / (2 s))
    a1, b1 = inputs.poly_pair(4095, 2047, inputs.SEED_BASE + 6)
    if b1[-1] == 0:
        b1[-1] = 1
    t1a, t1b = torch.from_numpy(a1).to(dev), torch.from_numpy(b1).to(dev)
    q1 = torch.empty(len(a1) - len(b1) + 1, dtype=torch.uint32, device=dev)
    r1 = torch.empty(len(b1) - 1, dtype=torch.uint32, device=dev)
    small = {}
    for s_d in (1, 256):
        pm.divide(t1a, t1b, s=s_d, q=q1, r=r1)
        assert pm.sync_status() == 0 and division_holds(t1a, t1b, q1, r1), f"division s={s_d}: a != q b + r"
        small[s_d] = median_ms(lambda s_d=s_d: pm.divide(t1a, t1b, s=s_d, q=q1, r=r1), 3, flush, stream)
    U = 4.0 * rate * SM_MAX_MHZ * 1e6 * SMS / (pk["hbm_gbs"] * 1e9)
    div_ratio = division_model_ratio(len(a1), len(b1), 256, 256, U)
    rows["division"] = {"workload": "a of degree 32767 divided by b of degree 16383",
                        "work_macs": work_d, "s_sweep": sweep,
                        "best_s": min(sweep, key=lambda e: e["ms"])["s"],
                        "naive_vs_s256_deg4095_by_2047": {"ms_s1": small[1], "ms_s256": small[256],
                                                         "measured_ratio": small[1] / small[256],
                                                         "model_ratio_T1_over_Ts": div_ratio, "U": U}}

    # --- gcd (Section 6, Algorithms 10-11): a of degree 9999, b of degree 8999, planted gcd of degree 1000 ---
    def planted_on_gpu(g_np, u_np, v_np):
        """a = g u and b = g v formed by the library's own product (gcd(u, v) = 1 for these seeds)."""
        tg, tu, tv = (torch.from_numpy(x).to(dev) for x in (g_np, u_np, v_np))
        return pm.plain(tg, tu), pm.plain(tg, tv), tg

    g_np, u_np, v_np = inputs.workload_gcd()
    ga, gb, tg = planted_on_gpu(g_np, u_np, v_np)
    gout = torch.empty(max(ga.numel(), gb.numel()), dtype=torch.uint32, device=dev)
    # the normal remainder sequence lowers one degree by one per step, from (9999, 8999) to (1000, -1)
    steps_g = (ga.numel() - 1 - 1000) + (gb.numel() - 1 - 1000) + 1
    sweep = []
    for s_g in (32, 64, 128, 256):
        res = pm.gcd(ga, gb, s=s_g, out=gout)
        assert pm.sync_status() == 0 and torch.equal(res, tg), f"gcd s={s_g}: not the planted gcd"
        ms = median_ms(lambda s_g=s_g: pm.gcd(ga, gb, s=s_g, out=gout), 5, flush, stream)
        sweep.append({"s": s_g, "ms": ms, "us_per_step": ms * 1e3 / steps_g})
    # s = 1 (the naive gcd of Algorithms 8-9, one step per launch) against s = 256 on the smallest size of
    # the paper's gcd timings (degrees 1999 and 1499), with the running-time ratio T_1 / T_s of Corollary 1
    g1, u1, v1 = inputs.gcd_cofactors(200, 1799, 1299, inputs.SEED_BASE + 8)
    sa, sb, sg = planted_on_gpu(g1, u1, v1)
    sout = torch.empty(max(sa.numel(), sb.numel()), dtype=torch.uint32, device=dev)
    small = {}
    for s_g in (1, 256):
        res = pm.gcd(sa, sb, s=s_g, out=sout)
        assert pm.sync_status() == 0 and torch.equal(res, sg), f"gcd s={s_g}: not the planted gcd"
        small[s_g] = median_ms(lambda s_g=s_g: pm.gcd(sa, sb, s=s_g, out=sout), 3, flush, stream)
    gcd_ratio = gcd_model_ratio(sa.numel(), sb.numel(), 256, 256, U)
    rows["gcd"] = {"workload": "a of degree 9999, b of degree 8999, planted gcd of degree 1000",
                   "division_steps": steps_g, "s_sweep": sweep,
                   "best_s": min(sweep, key=lambda e: e["ms"])["s"],
                   "naive_vs_s256_deg1999_and_1499": {"ms_s1": small[1], "ms_s256": small[256],
                                                      "measured_ratio": small[1] / small[256],
                                                      "model_ratio_T1_over_Ts": gcd_ratio, "U": U}}
    return rows


def run_case(args):
    """One kernel family on its workload: W warm-up and K timed steps (CUDA events, L2 flushed)."""
    import torch

    from paper_1402_0264_gb300 import build as pbuild
    from paper_1402_0264_gb300 import polymul as pm

    if not os.path.exists(pm.LIB_PATH):
        pbuild.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    flush_buf = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    s = args.s or 8
    if args.case == "plain":
        a, b = inputs.workload_single()
        ta, tb = torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)
        out = torch.empty(len(a) + len(b) - 1, dtype=torch.uint32, device=dev)
        step = lambda: pm.plain(ta, tb, s=s, out=out)
        check = lambda: torch.equal(out, pm.ntt(ta, tb))  # the transform path agrees
        macs, name = len(a) * len(b), "degree-16383 pair, plain s=%d" % s
    elif args.case == "divide":
        a, b = inputs.poly_pair(32767, 16383, inputs.SEED_BASE + 5)
        if b[-1] == 0:
            b[-1] = 1
        ta, tb = torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)
        qo = torch.empty(len(a) - len(b) + 1, dtype=torch.uint32, device=dev)
        out = torch.empty(len(b) - 1, dtype=torch.uint32, device=dev)
        sd = args.s or 0
        step = lambda: pm.divide(ta, tb, s=sd, q=qo, r=out)

        def check():  # a == q b + r through the library's own product
            qb = pm.plain(qo, tb).cpu().numpy().astype(np.uint64)
            qb[: out.numel()] = (qb[: out.numel()] + out.cpu().numpy().astype(np.uint64)) % P
            return np.array_equal(qb.astype(np.uint32), a)
        macs, name = (len(a) - len(b) + 1) * len(b), "degree 32767 divided by degree 16383, s=%d" % sd
    elif args.case == "gcd":
        g_np, u_np, v_np = inputs.workload_gcd()
        tg, tu, tv = (torch.from_numpy(x).to(dev) for x in (g_np, u_np, v_np))
        ta, tb = pm.plain(tg, tu), pm.plain(tg, tv)
        out = torch.empty(max(ta.numel(), tb.numel()), dtype=torch.uint32, device=dev)
        sg = args.s or 0
        res = {}
        def step():
            res["g"] = pm.gcd(ta, tb, s=sg, out=out)
        check = lambda: torch.equal(res["g"], tg)  # the planted factor
        macs, name = 0, "gcd of degrees 9999 and 8999 (planted gcd of degree 1000), s=%d" % sg
    elif args.case == "ntt":
        a, b = inputs.workload_ntt()
        ta, tb = torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)
        out = torch.empty(len(a) + len(b) - 1, dtype=torch.uint32, device=dev)
        step = lambda: pm.ntt(ta, tb, out=out)
        check = lambda: (eval_mod(out.cpu().numpy(), 123456789, P) ==
                         eval_mod(a, 123456789, P) * eval_mod(b, 123456789, P) % P)  # c(r) = a(r) b(r)
        macs, name = len(a) * len(b), "degree 2^22-1 pair, transform"
    else:
        packed = (inputs.workload_batched(batch=args.batch or 4096) if args.case == "batched"
                  else inputs.workload_tensor(batch=args.batch or 1024))
        max_deg = 2048 if args.case == "batched" else 4095
        mode = pm.PM_PLAIN if args.case == "batched" else pm.PM_TENSOR
        t = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in packed]
        out = torch.empty(int(packed[4][-1]), dtype=torch.uint32, device=dev)
        step = lambda: pm.batched(t[0], t[1], t[2], t[3], t[4], max_deg=max_deg, mode=mode, s=s,
                                  out=out, total=out.numel())
        other = pm.PM_TENSOR if args.case == "batched" else pm.PM_PLAIN  # the other form must agree
        check = lambda: torch.equal(out, pm.batched(t[0], t[1], t[2], t[3], t[4], max_deg=max_deg, mode=other,
                                                    total=out.numel()))
        macs = int(((packed[1][1:] - packed[1][:-1]) * (packed[3][1:] - packed[3][:-1])).sum())
        name = ("%d pairs, degrees log-uniform in [16,2048], plain s=%d" % (len(packed[1]) - 1, s)
                if args.case == "batched" else "%d pairs of degree 4095, tensor cores" % (len(packed[1]) - 1))
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert check(), "the two paths disagree"
    ts = []
    for _ in range(args.steps):
        flush_buf.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    assert pm.sync_status() == 0
    ms = sum(ts) / len(ts)
    print(json.dumps({"case": args.case, "workload": name, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": ms, "macs_per_s": macs / (ms * 1e-3) if macs else None, "unit": UNIT}),
          flush=True)
    return 0


def cpu_baseline_batch(tp, gpu_result):
    """The oracle on all host cores (the pairs of the headline batch shared out over OpenMP
    threads) for about 10 s of whole batches, plus one core on a sample of pairs; its products are
    compared word for word with the GPU's."""
    import oracle
    a_data, a_off, b_data, b_off, c_off = tp
    threads = oracle.omp_threads()
    reps, t0 = 0, time.perf_counter()
    while True:
        want = oracle.polymul_batch_omp(a_data, a_off, b_data, b_off, c_off, P)
        reps += 1
        dt = time.perf_counter() - t0
        if dt > 10.0 or reps >= 50:
            break
    assert np.array_equal(gpu_result, want), "bench: the GPU's batch differs from the oracle"
    k1 = 8  # one core: the first 8 pairs
    t1 = time.perf_counter()
    oracle.polymul_batch(a_data, a_off[:k1 + 1], b_data, b_off[:k1 + 1], c_off[:k1 + 1], P)
    dt1 = time.perf_counter() - t1
    return {"value": MACS_T * reps / dt, "unit": UNIT, "cores": threads, "kind": "oracle", "cpu": cpu_model(),
            "sample": f"{reps} runs of the whole 1024-pair batch ({dt:.1f} s), C schoolbook with 128-bit "
                      f"accumulation, pairs over {threads} OpenMP threads",
            "single_core_value": k1 * (DEG_T + 1) ** 2 / dt1,
            "single_core_sample": f"the first {k1} pairs on one thread ({dt1:.2f} s)"}


def cpu_baseline_single(a_np, b_np, gpu_result):
    """The oracle on the degree-16383 pair: one thread for about 10 s of full products (its product is
    compared word for word with the GPU's), then all host threads for about 5 s."""
    import oracle
    oracle.polymul(a_np[:8], b_np[:8], P)
    reps, t0 = 0, time.perf_counter()
    while True:
        want = oracle.polymul(a_np, b_np, P)
        reps += 1
        dt = time.perf_counter() - t0
        if dt > 10.0 or reps >= 100:
            break
    assert np.array_equal(gpu_result, want), "bench: the GPU result differs from the oracle"
    threads = oracle.omp_threads()
    r2, t2 = 0, time.perf_counter()
    while True:
        oracle.polymul_omp(a_np, b_np, P)
        r2 += 1
        dt2 = time.perf_counter() - t2
        if dt2 > 5.0 or r2 >= 1000:
            break
    return {"value": MACS_SINGLE * r2 / dt2, "unit": UNIT, "cores": threads, "kind": "oracle", "cpu": cpu_model(),
            "sample": f"{r2} full products of the degree-16383 pair, coefficients over {threads} OpenMP "
                      f"threads ({dt2:.1f} s)",
            "single_core_value": MACS_SINGLE * reps / dt,
            "single_core_sample": f"{reps} full products on one thread ({dt:.1f} s)"}


def plain_single_row(pm, torch, dev, flush, stream, alu_peak, rate, pk, args):
    """The one-pair degree-16383 product of the s-blocked kernel at the tuned s: per-step CUDA
    events after an L2 flush, the ALU roofline, end to end from pinned host buffers, the oracle."""
    a_np, b_np = inputs.workload_single()
    a = torch.from_numpy(a_np).to(dev)
    b = torch.from_numpy(b_np).to(dev)
    c = torch.empty(2 * N_SINGLE - 1, dtype=torch.uint32, device=dev)
    if args.s:
        s, tune_ms = args.s, {}
    else:  # flushed medians of 20 calls per s; near-ties go to the smaller s
        s, tune_ms = pm.tune_plain(a, b, reps=20, out=c)
    for _ in range(3):
        pm.plain(a, b, s=s, out=c)
    torch.cuda.synchronize()
    assert torch.equal(c, pm.ntt(a, b)), "bench: the plain and transform paths disagree"
    K = max(20, min(args.steps, 200))
    st = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    en = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    l0 = pm.launch_count()
    for i in range(K):
        flush()
        st[i].record(stream)
        pm.plain(a, b, s=s, out=c)
        en[i].record(stream)
    torch.cuda.synchronize()
    launches = pm.launch_count() - l0
    ms = [x.elapsed_time(y) for x, y in zip(st, en)]
    mean = sum(ms) / K
    a_h = torch.from_numpy(a_np).pin_memory()
    b_h = torch.from_numpy(b_np).pin_memory()
    c_h = torch.empty(2 * N_SINGLE - 1, dtype=torch.uint32).pin_memory()
    for i in range(K):
        flush()
        st[i].record(stream)
        a.copy_(a_h, non_blocking=True)
        b.copy_(b_h, non_blocking=True)
        pm.plain(a, b, s=s, out=c)
        c_h.copy_(c, non_blocking=True)
        en[i].record(stream)
    torch.cuda.synchronize()
    e2e_ms = sum(x.elapsed_time(y) for x, y in zip(st, en)) / K
    res = c_h.numpy().view(np.uint32).copy()
    assert np.array_equal(res, c.cpu().numpy().view(np.uint32))
    achieved = MACS_SINGLE / (mean * 1e-3)
    mhz = pk.get("sm_max_mhz") or SM_MAX_MHZ
    row = {"workload": WORKLOAD_SINGLE, "s": s, "steps": K, "ms_per_step": mean,
           "ms_median": statistics.median(ms), "macs_per_s": achieved, "gpu_launches": int(launches),
           "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "MAC/s",
                        "frac": achieved / alu_peak,
                        "peak_basis": f"derived: {IMAD_PER_CLK_SM} 32x32->64 multiply-adds (IMAD.WIDE.U32, half "
                                      f"the 32-bit IMAD rate) per clk per SM x {SMS} SMs x {mhz:.0f} MHz max SM "
                                      f"clock, one per modular MAC; measured in-tree {rate:.2f} per clk per SM "
                                      "(polymul_probe_mac_rate)",
                        "kernel": f"plain_sk_kernel<{s}>",
                        "traffic": traffic_for(f"plain_sk_kernel<{s}>", "plain.cu", "common.cuh")},
           "e2e": {"value": MACS_SINGLE / (e2e_ms * 1e-3), "unit": UNIT,
                   "h2d_bytes_per_step": int(a_h.numel() * 4 + b_h.numel() * 4),
                   "d2h_bytes_per_step": int(c_h.numel() * 4)},
           "tune_ms": {str(k): v for k, v in tune_ms.items()}}
    if not args.no_cpu_baseline:
        row["cpu_baseline"] = cpu_baseline_single(a_np, b_np, res)
    return row


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-rows", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--s", type=int, default=0, help="fix the block parameter (skip the tuner)")
    ap.add_argument("--case", choices=["plain", "batched", "tensor", "ntt", "divide", "gcd"], default=None,
                    help="time one kernel family alone (profiling runs); prints one JSON line")
    ap.add_argument("--batch", type=int, default=0,
                    help="with --case batched/tensor: the first pairs of the workload only (0 = all)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        rc = run_reference(args, world, rank)
    elif args.case:
        rc = run_case(args)
    else:
        rc = run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
