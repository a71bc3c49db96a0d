#!/usr/bin/env python3
"""Benchmark: multiplicative-update sweeps per second of the fused sweep.

Workload: dense CP 'ir,jr,kr->ijk' 512 x 512 x 512 (134,217,728 entries),
rank 64, Y = Poisson counts from Gamma(0.3, 1) ground-truth factors (seed 0),
no missing entries, KL loss ((alpha, beta) = (1, 0) of App. B), init
U(0.5, 1.5).  One step = one sweep of Algorithm 1 (three factor updates).
Y (537 MB) is larger than the 129 MB L2, so no flush is needed between steps.

Arms:
  --impl ours       the tensor-core (BF16 operands, FP32 accumulation) sweep,
                    plus the plain FP32 CUDA-core sweep as a variant
  --impl reference  the FP64 CPU oracle on the host cores (a bounded slab of the
                    same workload per step, scaled to sweeps/s)

Multi-GPU (torchrun): every rank fits its own replica of the workload (the
problems are independent; no collective on the data path): weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MU sweeps/sec at oracle-matched loss; % of HBM/tensor roofline; mixed vs plain FP32"
UNIT = "sweeps/s"
WORKLOAD = "cp ir,jr,kr->ijk 512x512x512 rank 64, KL (alpha,beta)=(1,0), Poisson/Gamma(0.3,1), no mask"
N_ENTRIES = 512 ** 3
SLAB_ROWS = 16          # rows of factor A updated per reference step
CPU_BASELINE_ROWS = 512  # rows of factor A updated by the cpu_baseline leg (all of them at 512^3)
CPU_BASELINE_REPS = 2    # timed repetitions of that update (about 10 s of oracle work at 512^3)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=512, help="cube side (512 = the benchmark workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--workload", default="cp_kl",
                    choices=["cp_kl", "cp_beta05", "custom4", "small", "batched", "uber", "icews", "losses",
                             "foldin", "uber_mesh"],
                    help="cp_kl: the benchmark line (default); the others print one measurement "
                         "line each for the other workloads")
    ap.add_argument("--batched-problems", type=int, default=48)
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the planner's default column splits (for profiler runs, where the "
                         "autotuner's event timings include the profiler's own overhead)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, world, device="cpu"):
    """The maximum of x over all ranks of the default process group (x itself
    when world == 1): every rank's timed region is bracketed by barriers, and the
    job's time is the slowest rank's."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps, ms):
    """Units per second of the whole job: every rank ran `steps` steps of its own
    replica and `ms` is the slowest rank's time."""
    return world * steps / (ms / 1e3)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


def kernel_hash():
    h = hashlib.sha256()
    for f in ("k_view_tc.cuh", "k_view_tc.cu", "k_view_tc_inst.cuh"):
        with open(os.path.join(ROOT, "paper_2602_02759_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_traffic():
    """DRAM bytes per launch of the fused pass from the committed ncu summary,
    or None when the kernel source changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "fused_pass_traffic.txt")
    try:
        d = {}
        with open(path) as fh:
            for line in fh:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    d[k.strip()] = v.strip()
        if d.get("kernel_hash") == kernel_hash():
            return float(d["bytes_per_launch_full"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []          # (receive time, line)
        self.window = None

    def start(self, wait_s: float = 5.0):
        """Start sampling every 20 ms and wait (up to wait_s) for the first sample."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < wait_s and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, t_begin: float, t_end: float):
        """Host wall-clock bounds of the timed region."""
        self.window = (t_begin, t_end)

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.05)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        lines = self.lines
        if self.window:
            inside = [x for x in lines if self.window[0] <= x[0] <= self.window[1] + 0.025]
            if not inside:  # region shorter than the sampling interval: the first sample after it began
                inside = [x for x in lines if x[0] >= self.window[0]][:1]
            lines = inside
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, ln in lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- oracle legs

def oracle_slab_seconds(p, rows):
    """Time the oracle's update of rows [0, rows) of factor A: that update only
    involves Y[0:rows], A[0:rows], B and C, so it is exactly those rows of the
    full update."""
    import numpy as np
    from oracle import OracleModel
    import oracle
    dims = dict(p.dims)
    dims["i"] = rows
    m = OracleModel(p.model_str, dims)
    y = np.ascontiguousarray(p.y[:rows], dtype=np.float64)
    init = [np.ascontiguousarray(p.inits[0][0][:rows], np.float64),
            p.inits[0][1].astype(np.float64), p.inits[0][2].astype(np.float64)]
    t0 = time.perf_counter()
    m.update_factor(0, y, None, init, p.alpha, p.beta)
    return time.perf_counter() - t0, oracle.num_threads()


def sweep_fraction(rows, n):
    # a sweep updates 3 factors of n rows each
    return rows / (3.0 * n)


def foldin_variant(nef, torch, stream, train_sweeps=100, steps=200, lr=1e-3):
    """The fold-in workload (CP 2048x128x128 rank 32, KL): MU fit of the 1536
    training slices, encoder training on (slice, component count mass) pairs,
    then the 512 held-out slices folded in from the encoder's loadings and from
    the plain initialisation, with k MU passes on mode 0 (B, C fixed)."""
    import numpy as np
    import synth
    p = synth.config5()
    n, J, K = p.y.shape
    R = p.dims["r"]
    n_tr = 1536
    n_te = n - n_tr
    d = J * K
    y = torch.from_numpy(p.y).cuda()
    ytr, yte = y[:n_tr].contiguous(), y[n_tr:].contiguous()
    A0, B0, C0 = (torch.from_numpy(f).cuda() for f in p.inits[0])
    fs = [A0[:n_tr].contiguous(), B0.clone(), C0.clone()]
    fit = nef.Plan(p.model_str, dict(i=n_tr, j=J, k=K, r=R), precision="bf16", stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fit.fit(ytr, None, fs, 1.0, 0.0, train_sweeps)
    e1.record(stream)
    torch.cuda.synchronize()
    t_fit = e0.elapsed_time(e1) / 1e3
    A_tr, B, C = fs
    mass = (B.sum(0) * C.sum(0))[None, :]
    targets = (A_tr * mass).contiguous()
    xs = ytr.reshape(n_tr, d).contiguous()
    enc = nef.FoldIn(d, 512, R, n_tr, torch.from_numpy(nef.pack_params(synth.mlp_params((d, 512, 512, R), 3))).cuda(),
                     stream=stream)
    l0 = enc.train_step(xs, targets, lr)
    # half the timed steps pass the slices (features recomputed every step), the other
    # half use the batch kept by nef_foldin_load_batch (full-batch training computes
    # the features once); both give the same parameters bit for bit
    half = (steps - 2) // 2
    e0.record(stream)
    for _ in range(half):
        enc.train_step(xs, targets, lr, want_loss=False)
    e1.record(stream)
    torch.cuda.synchronize()
    t_train_feat = e0.elapsed_time(e1) / 1e3 / half
    enc.load_batch(xs)
    e0.record(stream)
    for _ in range(steps - 2 - half):
        enc.train_step(None, targets, lr, want_loss=False)
    e1.record(stream)
    l_end = enc.train_step(None, targets, lr)
    t_train = e0.elapsed_time(e1) / 1e3 / (steps - 2 - half)
    # products per Adam step: the first layer's forward product and weight gradient (its
    # input gradient is not needed), three each for the other two layers
    flops = 2.0 * n_tr * (2 * d * 512 + 3 * 512 * 512 + 3 * 512 * R)
    ref = nef.Plan(p.model_str, dict(i=n_te, j=J, k=K, r=R), precision="fp32", stream=stream)
    x_te = yte.reshape(n_te, d).contiguous()
    for _ in range(3):  # warm-up
        enc.predict(x_te)
    torch.cuda.synchronize()
    n_pred = 20
    e0.record(stream)
    for _ in range(n_pred):
        out_te = enc.predict(x_te)
    e1.record(stream)
    torch.cuda.synchronize()
    t_pred = e0.elapsed_time(e1) / 1e3 / n_pred
    A_enc = (out_te / mass).contiguous()

    def gaps(A, ks):
        fs2 = [A.clone(), B, C]
        out, done = {}, 0
        for k in ks:
            for _ in range(k - done):
                ref.update(0, yte, None, fs2, 1.0, 0.0)
            done = k
            out[k] = ref.loss(yte, None, fs2, 1.0, 0.0)[0]
        return out

    ks = [0, 1, 2, 5, 10, 20]
    full = gaps(A0[n_tr:].contiguous(), [500])[500]
    g_enc = gaps(A_enc, ks)
    g_pl = gaps(A0[n_tr:].contiguous(), ks)
    return {"workload": p.note + ", KL; encoder 16384->512->512->32, targets = loading x column-sum mass",
            "mu_fit_train": {"sweeps": train_sweeps, "seconds": t_fit},
            "encoder_train": {"adam_steps": steps, "batch": n_tr, "loss_first": l0, "loss_last": l_end,
                              "ms_per_step": t_train * 1e3, "tflops": flops / t_train / 1e12,
                              "ms_per_step_features_every_step": t_train_feat * 1e3,
                              "note": "ms_per_step: full-batch steps on the batch kept by "
                                      "nef_foldin_load_batch; the other figure passes the slices "
                                      "every step (log1p features recomputed)"},
            "predict_ms": t_pred * 1e3,
            "predict_note": f"{n_te} held-out slices per call, mean of {n_pred} calls after 3 warm-up calls",
            "heldout_gap_vs_full_mu_foldin": {"k_passes": ks,
                                              "encoder": [g_enc[k] / full - 1 for k in ks],
                                              "plain_init": [g_pl[k] / full - 1 for k in ks],
                                              "full_foldin_passes": 500}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import synth
    p = synth.config2(n=args.n)
    rows = min(SLAB_ROWS, args.n)
    for _ in range(args.warmup):
        oracle_slab_seconds(p, rows)
    ts = []
    cores = 1
    for _ in range(args.steps):
        t, cores = oracle_slab_seconds(p, rows)
        ts.append(t)
    total = sum(ts)
    value = args.steps * sweep_fraction(rows, args.n) / total
    sample = (f"per step: oracle update of rows 0..{rows - 1} of factor A (Y[0:{rows}], exact rows "
              f"of the full update) = {sweep_fraction(rows, args.n):.5f} sweep")
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "l2_flush": "inputs larger than L2"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm

def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2602_02759_gb300 as nef
    import synth

    p = synth.config2(n=args.n)
    # cpu_baseline before any heavy GPU work (rank 0, N = 1 only)
    cpu_base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rows = min(CPU_BASELINE_ROWS, args.n)
        t = 0.0
        for _ in range(CPU_BASELINE_REPS):
            ti, cores = oracle_slab_seconds(p, rows)
            t += ti
        frac = sweep_fraction(rows, args.n)
        cpu_base = {"value": CPU_BASELINE_REPS * frac / t, "unit": UNIT, "cores": cores,
                    "kind": "oracle",
                    "sample": f"{CPU_BASELINE_REPS} x the oracle update of rows 0..{rows - 1} of factor A "
                              f"(exact rows of the full update; {frac:.5f} sweep each), {t:.1f} s"}

    dims = p.dims
    stream = torch.cuda.current_stream()
    Y = torch.from_numpy(p.y).cuda()
    init = [torch.from_numpy(f).cuda() for f in p.inits[0]]

    def fresh():
        return [f.clone() for f in init]

    sampler = ClockSampler(local)
    sampler.start()
    # timed region: one nef_fit call of K sweeps (sweeps 3.. replay a captured
    # CUDA graph of one sweep); warm-up: W sweeps the same way
    plan = nef.Plan(p.model_str, dims, precision="bf16", stream=stream)
    fs = fresh()
    splits = None if args.no_autotune else plan.autotune(Y, None, fs, p.alpha, p.beta)  # plan setup
    plan.fit(Y, None, fs, p.alpha, p.beta, args.warmup)
    plan.check()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    t_begin = time.time()
    ev0.record(stream)
    plan.fit(Y, None, fs, p.alpha, p.beta, args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    sampler.mark(t_begin, time.time())
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    plan.check()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, device="cuda")
    value = whole_job_rate(world, args.steps, ms)

    # kernel durations: the same sweeps launched eagerly with a CUDA event pair
    # around every fused-pass launch (on the plan's stream)
    n_prof = min(args.steps, 100)
    pplan = nef.Plan(p.model_str, dims, precision="bf16", profile=True, stream=stream)
    gp = fresh()
    if not args.no_autotune:
        pplan.autotune(Y, None, gp, p.alpha, p.beta)
    pplan.fit(Y, None, gp, p.alpha, p.beta, 2)
    pplan.profile(reset=True)
    torch.cuda.synchronize()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    pplan.fit(Y, None, gp, p.alpha, p.beta, n_prof)
    e3.record(stream)
    torch.cuda.synchronize()
    pplan.check()
    ms_prof = e2.elapsed_time(e3)
    prof = pplan.profile(reset=True)
    del pplan, gp

    # roofline of the dominant kernel: the tensor-core fused pass
    hbm, bf16, src = load_peaks()
    tc_ms, tc_n = prof["tcgen05"]
    roof = None
    if tc_n:
        avg_s = tc_ms / tc_n / 1e3
        alg_bytes = 4.0 * p.y.size   # one FP32 read of Y per pass
        ach = alg_bytes / avg_s / 1e9
        traffic = load_traffic()
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": traffic, "peak_source": f"hbm_gbs of {src}",
                "kernel": "k_view_tc (tcgen05 fused pass)", "avg_launch_us": avg_s * 1e6,
                "algorithmic_bytes_per_launch": alg_bytes,
                "share_of_step": tc_ms / ms_prof,
                "timing": f"CUDA events around each fused-pass launch in {n_prof} eagerly launched sweeps "
                          f"right after the timed region"}
    launches_per_sweep = plan.launches(False)
    loss_bf16 = plan.loss(Y, None, fs, p.alpha, p.beta)[0]

    variants = {}
    if rank == 0 and not args.no_variants:
        # plain FP32 CUDA-core sweep from the same start, same number of sweeps
        plan32 = nef.Plan(p.model_str, dims, precision="fp32", stream=stream)
        g = fresh()
        plan32.fit(Y, None, g, p.alpha, p.beta, args.warmup)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan32.fit(Y, None, g, p.alpha, p.beta, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        plan32.check()
        ms32 = e0.elapsed_time(e1)
        loss32 = plan32.loss(Y, None, g, p.alpha, p.beta)[0]
        variants["fp32_plain"] = {"value": args.steps / (ms32 / 1e3), "unit": UNIT,
                                  "ms_per_step": ms32 / args.steps, "loss": loss32}
        variants["bf16_vs_fp32_speedup"] = (args.steps / (ms / 1e3)) / variants["fp32_plain"]["value"]
        variants["loss_check"] = {"bf16": loss_bf16, "fp32": loss32,
                                  "rel_diff": abs(loss_bf16 - loss32) / loss32,
                                  "sweeps": args.warmup + args.steps,
                                  "note": "the FP32 sweep matches the FP64 oracle to 1e-5 (parity tests)"}
        del plan32
        # the same BF16 sweeps with the per-sweep loss trace (loss summed inside the first
        # pass); the warm-up call uses the same trace buffer, so the timed call replays the
        # sweep graph captured with the trace and its loss kernels are already loaded
        n_lt = min(args.steps, 200)
        g = fresh()
        tr = torch.full((n_lt + 1,), float("nan"), dtype=torch.float64, device="cuda")
        plan.fit(Y, None, g, p.alpha, p.beta, 3, loss_trace=tr)
        torch.cuda.synchronize()
        e0.record(stream)
        plan.fit(Y, None, g, p.alpha, p.beta, n_lt, loss_trace=tr)
        e1.record(stream)
        torch.cuda.synchronize()
        plan.check()
        ms_lt = e0.elapsed_time(e1)
        last = float(tr[-1].item())
        ref_last = plan.loss(Y, None, g, p.alpha, p.beta)[0]
        variants["bf16_loss_trace"] = {"value": n_lt / (ms_lt / 1e3), "unit": UNIT, "sweeps": n_lt,
                                       "vs_plain_sweep": (n_lt / (ms_lt / 1e3)) / value,
                                       "final_trace_vs_nef_loss_rel": abs(last - ref_last) / ref_last}
        # nef_loss: one call (tensor-core loss pass, FP64 reduction, copy to the host), host clock
        for _ in range(3):
            plan.loss(Y, None, g, p.alpha, p.beta)
        t0 = time.perf_counter()
        for _ in range(20):
            plan.loss(Y, None, g, p.alpha, p.beta)
        loss_ms = (time.perf_counter() - t0) / 20 * 1e3
        variants["nef_loss_call"] = {"ms": loss_ms, "vs_fused_pass": loss_ms / (roof["avg_launch_us"] / 1e3)
                                     if roof else None,
                                     "note": "host time of one synchronising nef_loss call, mean of 20"}

    if rank == 0 and not args.no_variants:
        variants["foldin"] = foldin_variant(nef, torch, stream)

    e2e = None
    if not args.no_e2e:
        Yh = torch.from_numpy(p.y).pin_memory()
        Fh = [f.clone().cpu().pin_memory() for f in init]
        Fo = [torch.empty_like(f).pin_memory() for f in Fh]
        Yd = torch.empty_like(Y)
        fd = fresh()
        torch.cuda.synchronize()
        h2d = Yh.numel() * 4 + sum(f.numel() * 4 for f in Fh)
        d2h = sum(f.numel() * 4 for f in Fo)
        for it in range(args.warmup + args.steps):
            if it == args.warmup:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
            Yd.copy_(Yh, non_blocking=True)
            for a, b in zip(fd, Fh):
                a.copy_(b, non_blocking=True)
            plan.fit(Yd, None, fd, p.alpha, p.beta, 1)
            for a, b in zip(Fo, fd):
                a.copy_(b, non_blocking=True)
            torch.cuda.current_stream().synchronize()
        el = max_over_ranks(time.perf_counter() - t0, world, device="cuda")
        e2e = {"value": whole_job_rate(world, args.steps, el * 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}
        del Yd, Yh

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16 operands, fp32 accumulate",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "bf16 (tcgen05)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2_flush": "inputs larger than L2 (Y = 537 MB)",
                       "column_splits": splits},
            "roofline": roof, "cpu_baseline": cpu_base, "e2e": e2e,
            "gpu_launches": launches_per_sweep * args.steps,
            "clocks": clocks, "loss": loss_bf16, "variants": variants,
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def time_fit(nef, torch, p, precision, sweeps, warmup, stream, eager=False, autotune=True):
    """Seconds per sweep of one nef_fit call of `sweeps` sweeps (after `warmup`
    sweeps), and the final loss, from p.inits[0]."""
    dt = torch.float64 if precision == "fp64" else torch.float32

    def dev(a):
        return a if torch.is_tensor(a) else torch.from_numpy(a).cuda()

    Y = dev(p.y).to(dt)
    M = None if p.mask is None else dev(p.mask)
    fs = [dev(f).to(dt).clone() for f in p.inits[0]]  # every fit starts from the same inits
    lk = dict(loss=getattr(p, "loss", "ab"), loss_par=getattr(p, "loss_par", 0.0))
    plan = nef.Plan(p.model_str, p.dims, precision=precision, stream=stream, eager=eager, **lk)
    if autotune:
        plan.autotune(Y, M, fs, p.alpha, p.beta)  # plan setup, outside the timed region
    plan.fit(Y, M, fs, p.alpha, p.beta, warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.fit(Y, M, fs, p.alpha, p.beta, sweeps)
    e1.record(stream)
    torch.cuda.synchronize()
    plan.check()
    sec = e0.elapsed_time(e1) / 1e3 / sweeps
    loss = plan.loss(Y, M, fs, p.alpha, p.beta)[0]
    # per-family kernel time in two profiled sweeps
    pp = nef.Plan(p.model_str, p.dims, precision=precision, stream=stream, profile=1, **lk)
    gs = [f.clone() for f in fs]
    if autotune:
        pp.autotune(Y, M, gs, p.alpha, p.beta)
    pp.fit(Y, M, gs, p.alpha, p.beta, 2)
    prof = pp.profile(reset=True)
    info = plan.info()
    del plan, pp, Y, M
    return sec, loss, prof, info


def uber_mesh_problem(torch, dims=(27, 7, 24, 400, 400), r=10, k=6, seed=0):
    """The Uber model 'wr,dr,hr,irk,jrk->wdhij' at the 400 x 400 pick-up mesh of the
    paper's largest Uber tensor (27 x 7 x 24 x 400 x 400 = 725.8 M entries), R = 10,
    K = 6: the recipe of synth.config_uber (Gamma(0.3,1) truth, Poisson data, no mask,
    KL, inits U(0.5,1.5)) drawn on the GPU with a seeded torch generator, since numpy
    would take minutes at this size."""
    from types import SimpleNamespace
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    w, d, h, i, j = dims
    shapes = [(w, r), (d, r), (h, r), (i, r, k), (j, r, k)]
    truth = [torch._standard_gamma(torch.full(s, 0.3, device="cuda"), generator=g) for s in shapes]
    mean = torch.einsum("wr,dr,hr,irk,jrk->wdhij", *truth)
    y = torch.poisson(mean, generator=g).contiguous()
    del mean, truth
    inits = [[(0.5 + torch.rand(s, device="cuda", generator=g)).contiguous() for s in shapes]]
    return SimpleNamespace(model_str="wr,dr,hr,irk,jrk->wdhij",
                           dims={"w": w, "d": d, "h": h, "i": i, "j": j, "r": r, "k": k}, y=y, mask=None,
                           inits=inits, alpha=1.0, beta=0.0, factor_shapes=lambda: shapes,
                           note=f"uber-mesh wr,dr,hr,irk,jrk->wdhij {dims} R{r} K{k} KL (data drawn on the GPU)")


def run_workload(args):
    """Measurement lines for the workloads other than the benchmark line."""
    import numpy as np
    import torch
    import paper_2602_02759_gb300 as nef
    import synth
    hbm, _, src = load_peaks()
    stream = torch.cuda.current_stream()
    sweeps = max(3, args.steps)
    if args.workload == "foldin":
        # the learned fold-in workload alone (the benchmark line carries it as a variant)
        out = foldin_variant(nef, torch, stream)
        out["peak_source"] = f"hbm_gbs {hbm} of {src}"
        print(json.dumps(out), flush=True)
        return 0
    if args.workload == "losses":
        # the 512^3 rank-64 CP workload under each further loss family (App. B), BF16
        # and the plain FP32 sweep, the same sweeps from the same start
        n_el = args.n ** 3
        bytes_sweep = 3 * 4.0 * n_el
        out = {"workload": f"cp {args.n}^3 R64, loss families of App. B beyond KL", "entries": n_el,
               "algorithmic_bytes_per_sweep": bytes_sweep, "sweeps": sweeps, "families": {}}
        for kind in synth.LOSS_WORKLOADS:
            p = synth.config2_loss(kind, n=args.n)
            fam = {"note": p.note, "loss": p.loss, "loss_par": p.loss_par, "alpha_beta": [p.alpha, p.beta]}
            for prec in ("bf16", "fp32"):
                sec, loss, prof, info = time_fit(nef, torch, p, prec, sweeps if prec == "bf16" else 3,
                                                 args.warmup if prec == "bf16" else 1, stream)
                fam[prec] = {"sweeps_per_s": 1.0 / sec, "ms_per_sweep": sec * 1e3,
                             "hbm_frac": bytes_sweep / sec / 1e9 / hbm, "loss": loss,
                             "fused_pass_ms": {k: v[0] / max(1, v[1]) for k, v in prof.items() if v[1]}}
            fam["bf16_vs_fp32_speedup"] = fam["bf16"]["sweeps_per_s"] / fam["fp32"]["sweeps_per_s"]
            out["families"][kind] = fam
            del p
        out["note"] = ("the BF16 and FP32 losses come from different sweep counts (FP32: 1 + 3 sweeps); "
                       "parity with the oracle is in tests/test_gpu_losses.py")
        out["peak_source"] = f"hbm_gbs {hbm} of {src}"
        print(json.dumps(out), flush=True)
        return 0
    if args.workload in ("cp_beta05", "custom4", "small", "uber", "icews", "uber_mesh"):
        p = {"cp_beta05": lambda: synth.config2(beta=-0.5, n=args.n),
             "custom4": synth.config3, "small": synth.config1,
             "uber": synth.config_uber, "icews": synth.config_icews,
             "uber_mesh": lambda: uber_mesh_problem(torch)}[args.workload]()
        n_el = p.y.numel() if torch.is_tensor(p.y) else p.y.size
        n_fac = len(p.factor_shapes())
        bytes_sweep = n_fac * (4.0 * n_el + (n_el / 8.0 if p.mask is not None else 0.0))
        out = {"workload": p.note, "alpha_beta": [p.alpha, p.beta], "entries": int(n_el),
               "algorithmic_bytes_per_sweep": bytes_sweep, "sweeps": sweeps}
        precs = ["bf16", "fp32"] + (["fp64"] if args.workload == "small" else [])
        for prec in precs:
            sec, loss, prof, info = time_fit(nef, torch, p, prec, sweeps, args.warmup, stream,
                                             autotune=not args.no_autotune)
            if prec == "bf16":
                out["plan"] = info.strip().splitlines()
            out[prec] = {"sweeps_per_s": 1.0 / sec, "ms_per_sweep": sec * 1e3,
                         "hbm_frac": bytes_sweep / sec / 1e9 / hbm, "loss": loss,
                         "fused_pass_ms": {k: v[0] / max(1, v[1]) for k, v in prof.items() if v[1]},
                         "fused_pass_launches_per_2_sweeps": {k: v[1] for k, v in prof.items()}}
        out["bf16_vs_fp32_loss_rel"] = abs(out["bf16"]["loss"] - out["fp32"]["loss"]) / out["fp32"]["loss"]
        out["bf16_vs_fp32_speedup"] = out["bf16"]["sweeps_per_s"] / out["fp32"]["sweeps_per_s"]
        out["peak_source"] = f"hbm_gbs {hbm} of {src}"
        print(json.dumps(out), flush=True)
        return 0
    # batched: the batched workload (the first --batched-problems of its 512 problems),
    # every problem with 8 restarts
    specs = synth.batched_specs()[: args.batched_problems]
    restarts = 8
    if len(specs) <= 48:
        probs = [synth.batched_problem(shape, r, seed=1000 + q, restarts=restarts)
                 for q, (shape, r) in enumerate(specs)]
        Ys = [torch.from_numpy(q.y).cuda() for q in probs]
        Ms = [torch.from_numpy(q.mask).cuda() for q in probs]
        inits = [[[torch.from_numpy(f).cuda() for f in q.inits[k]] for k in range(restarts)] for q in probs]
        gen_note = "numpy (synth.batched_problem)"
    else:
        # the same recipe drawn on the GPU with a seeded torch generator (numpy would take
        # minutes for 3.7e9 entries): Gamma(0.3, 1) truth, Poisson counts, 10% missing,
        # inits U(0.5, 1.5)
        gg = torch.Generator(device="cuda")
        gg.manual_seed(1000)
        Ys, Ms, inits = [], [], []
        for (i, j, k), r in specs:
            tr = [torch._standard_gamma(torch.full((n, r), 0.3, device="cuda"), generator=gg) for n in (i, j, k)]
            mean = torch.einsum("ir,jr,kr->ijk", *tr)
            Ys.append(torch.poisson(mean, generator=gg).contiguous())
            Ms.append((torch.rand(mean.shape, device="cuda", generator=gg) >= 0.1).to(torch.uint8).contiguous())
            del mean, tr
            inits.append([[(0.5 + torch.rand((n, r), device="cuda", generator=gg)).contiguous() for n in (i, j, k)]
                          for _ in range(restarts)])
        probs = None
        gen_note = "torch CUDA generator, seed 1000 (same recipe as synth.batched_problem)"

    def fresh(count=None):
        src = inits if count is None else inits[:count]
        return [[[f.clone() for f in fk] for fk in fp] for fp in src]

    n_sum = sum(y.numel() for y in Ys)
    bytes_sweep = 3 * n_sum * (4.0 + 1.0 / 8.0)
    fits = len(Ys) * restarts
    facs = fresh()
    # the work-item size, tuned on this workload (outside the timed region)
    tiles, tile_ms = nef.fit_batched_tune(Ys, Ms, facs, 1.0, 0.0)
    nef.fit_batched(Ys, Ms, facs, 1.0, 0.0, args.warmup, losses=False, tiles=tiles)
    torch.cuda.synchronize()
    # the fit: one call of `sweeps` sweeps (set-up included), no loss evaluation
    t0 = time.perf_counter()
    nef.fit_batched(Ys, Ms, facs, 1.0, 0.0, sweeps, losses=False, tiles=tiles)
    torch.cuda.synchronize()
    t_b = time.perf_counter() - t0
    # the call's fixed cost, and the loss of every fit (0 sweeps: set-up + loss pass)
    t0 = time.perf_counter()
    nef.fit_batched(Ys, Ms, facs, 1.0, 0.0, 0, losses=False, tiles=tiles)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    losses = nef.fit_batched(Ys, Ms, facs, 1.0, 0.0, 0, tiles=tiles)
    t_loss = time.perf_counter() - t0 - t_setup
    # one plain FP32 plan per (problem, restart), the same sweeps (at most the first 48 problems)
    n_cmp = min(48, len(Ys))
    facs2 = fresh(n_cmp)
    t1 = time.perf_counter()
    loss_fp32 = []
    for qi in range(n_cmp):
        i, j, k3 = Ys[qi].shape
        R = int(inits[qi][0][0].shape[1])
        plan = nef.Plan("ir,jr,kr->ijk", dict(i=i, j=j, k=k3, r=R), precision="fp32", stream=stream)
        for k in range(restarts):
            plan.fit(Ys[qi], Ms[qi], facs2[qi][k], 1.0, 0.0, args.warmup + sweeps)
        torch.cuda.synchronize()
        loss_fp32.append([plan.loss(Ys[qi], Ms[qi], facs2[qi][k], 1.0, 0.0)[0] for k in range(restarts)])
        del plan
    t_s = time.perf_counter() - t1
    sweeps_fp32 = n_cmp * restarts * (args.warmup + sweeps)
    rel = [abs(losses[a][b] - loss_fp32[a][b]) / loss_fp32[a][b] for a in range(n_cmp) for b in range(restarts)]
    # the issue side: every restart's epilogue work runs per entry, so the engine is bound by
    # instruction issue, not by HBM; the instructions per entry-update are the ncu count of
    # k_batched_persistent on the first 8 problems (36.3 warp instructions per 32)
    eu_per_s = 3.0 * n_sum * restarts * sweeps / t_b
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    issue_peak = n_sm * 4 * 2070e6  # 4 schedulers per SM, one warp instruction per clock, 2070 MHz
    issue = {"entry_updates_per_s": eu_per_s, "warp_instructions_per_32_entry_updates": 36.3,
             "achieved_warp_instructions_per_s": eu_per_s * 36.3 / 32, "peak_warp_instructions_per_s": issue_peak,
             "frac": eu_per_s * 36.3 / 32 / issue_peak,
             "note": "instruction count per entry-update from one ncu capture of the first 8 problems; "
                     "peak = SMs x 4 issue slots x 2070 MHz"}
    out = {"workload": f"batched CP: {'all' if len(Ys) == 512 else 'first ' + str(len(Ys)) + ' of the'} 512 "
                       f"problems (dims U{{20..300}}^3, ranks U{{4..32}}, 10% missing), {restarts} restarts each, KL",
           "data": gen_note, "entries": int(n_sum), "fits": fits, "sweeps": sweeps,
           "batched_bf16": {"fit_sweeps_per_s": fits * sweeps / t_b, "seconds": t_b,
                            "ms_per_all_problem_sweep": t_b / sweeps * 1e3,
                            "hbm_frac": bytes_sweep * sweeps / t_b / 1e9 / hbm,
                            "call_setup_ms": t_setup * 1e3, "loss_pass_ms": t_loss * 1e3,
                            "tiles_per_item": tiles, "issue": issue,
                            "tune_ms_2_sweeps": {str(k): v for k, v in tile_ms.items()},
                            "note": "wall clock of one nef_fit_batched call of all the sweeps without the "
                                    "final loss evaluation (one persistent launch per bond width, "
                                    "graph-captured); call_setup_ms is a 0-sweep call, loss_pass_ms the "
                                    "extra time of the losses of every fit; bytes count Y and the mask bits "
                                    "once per problem and mode, not once per restart"},
           "per_fit_fp32": {"fit_sweeps_per_s": sweeps_fp32 / t_s, "seconds": t_s, "problems": n_cmp,
                            "note": "one NEF_FP32 plan per problem, restarts fitted one after another"},
           "speedup": (fits * sweeps / t_b) / (sweeps_fp32 / t_s),
           "loss_rel_batched_vs_fp32": {"max": max(rel), "median": float(np.median(rel)),
                                        "p90": float(np.quantile(rel, 0.9)), "problems": n_cmp},
           "peak_source": f"hbm_gbs {hbm} of {src}"}
    print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "cp_kl":
        return run_workload(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
