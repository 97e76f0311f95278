"""Benchmark: PGA tensor completion (Algorithm 5) on one GB300 per rank.

Workload (one "step"): one call of lt_pga_complete -- 100 PGA iterations of the
144 x 176 x 3 x 32 low-L-rank completion problem (L-rank 10, Gaussian noise 1e-3, 30%
observed, L_3 = DCT 3, L_4 = DCT 32, tau = 0.5, step 1), cold start X^0 = X^1 = 0.
Every iteration runs all hot-path steps: momentum + masked gradient step fused into the
forward transform, per-slice Jacobi SVD + shrink + reconstruction, inverse transform
with the fused residual, device-side scalar update.

value     PGA iterations per second of the plain FP64 path, summed over ranks, inputs
          resident in HBM.  L2 is flushed (a 512 MiB write) between timed steps.  The
          completion contexts run with the warm-started SVT (LT_OPT_WARM_START: period 8
          for FP64, 4 for FP32 / LT_MIXED; --warm / --warm32, 0 turns it off).
e2e       the same metric through the C ABI with host buffers: the pinned-host mask and
          observations are copied in and the result copied out inside every step.
mixed     the LT_MIXED path on the same inputs with the library's defaults (FP32 data;
          modes below 64 stay in the fused SIMT transform passes, so on this workload it
          runs the FP32 kernels: tc_launches_per_step = 0), with its relative error
          against the FP64 result of the same run; mixed_tc32: LT_MIXED with the mode-32
          products on the tcgen05 tensor cores (LT_OPT_TC_MODE_MIN = 32); fp32: the same
          for the LT_FP32 context.
svt       L-SVT slices/s (lt_svt, transforms included, and the Jacobi launch alone):
          the 96 144x176 slices of P_Omega(M) (FP64, FP32) and the 2048 256x256 slices
          of the fifth-order tensor (FP64, FP32, LT_MIXED) with errors against FP64.
batched   the 64 uneven completion problems in LT_MIXED (those with I4 = 64 put their
          mode-4 products on the tcgen05 tensor cores) as one graph-captured call.
product_256x256x16x16x8  the fifth-order *_L-product (LT_MIXED and FP32): the face-wise
          GEMM on the tcgen05 tensor cores (split TF32 x 3) against the HBM roofline,
          and the error of each against the FP64 product of the same operands.
roofline  the Jacobi SVT kernel (dominant): executed-flop count reported by the kernel
          / its CUDA-event time over the timed steps, against the FP64 FMA peak derived
          from SMs x max SM clock x 2 DFMA/clk/SM (ALU-bound: the FP64 pipe), with the
          fraction of the throughput lt_measure_fma_peak measures at start-up beside it.
autotune  the SVT kernel form each context runs, picked by lt_autotune_svt (timings of
          every form on the observations, outside the timed region).
cpu_baseline  the FP64 oracle (numpy/LAPACK) on the host cores, a bounded sample of
          the same workload (a few PGA iterations).

Multi-GPU (torchrun): every rank solves its own independent problem (replicas: one
completion problem does not shard without an all-to-all); value = all ranks'
iterations / max-over-ranks time.  `--impl reference` times the oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PGA iters/s & L-SVT slices/s, mixed vs FP64 at rel-err<=1e-5; %roofline"
WORKLOAD = "pga_completion_144x176x3x32_fp64"
# Peaks of the ALU-bound rooflines in GFLOP/s, derived from unit counts and clocks:
# SMs x maximum SM clock x FMA units per SM per clock x 2 (FP64: 2 DFMA per SM per clock,
# the part's nominal 1.25 TFLOP/s; FP32: 128 FFMA).  Beside them, the FMA throughput
# that lt_measure_fma_peak measures at start-up (eight independent FMA chains per
# thread, four 512-thread CTAs per SM): on GB300 FP32 reaches 97.6 % of the derived peak
# and FP64 84 % (1057.8 GFLOP/s at 2070 MHz, the same for every chain, unroll and
# occupancy variant tried).
FMA_PER_CLK = {"fp64": 2, "fp32": 128}
FMA_PEAKS = {}
DERIVED_PEAKS = {}
PEAK_SOURCE = ("derived: SMs x max SM clock x FMA per SM per clock x 2 (FP64 2, FP32 128 "
               "FMA/clk/SM); measured_peak = lt_measure_fma_peak at start-up")


def max_sm_mhz():
    try:
        r = subprocess.run(["nvidia-smi", "-i", str(int(os.environ.get("LOCAL_RANK", "0"))),
                            "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                           capture_output=True, text=True, timeout=20)
        return float(r.stdout.strip().splitlines()[0])
    except Exception:
        return 2070.0


def fma_peak(name):
    """Derived FMA peak ("fp64" or "fp32") of this GPU in GFLOP/s (cached)."""
    if name not in DERIVED_PEAKS:
        import torch
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        DERIVED_PEAKS[name] = round(sms * max_sm_mhz() * 1e6 * FMA_PER_CLK[name] * 2 / 1e9, 1)
    return DERIVED_PEAKS[name]


def measured_peak(name):
    """FMA throughput measured by lt_measure_fma_peak ("fp64" or "fp32"), GFLOP/s."""
    if name not in FMA_PEAKS:
        from paper_2202_02870_gb300 import lt
        prec = lt.LT_FP64 if name == "fp64" else lt.LT_FP32
        FMA_PEAKS[name] = round(max(lt.lt_measure_fma_peak(prec) for _ in range(2)), 1)
    return FMA_PEAKS[name]


def alu_roofline(achieved, name, **extra):
    """Roofline entry of an ALU-bound kernel: achieved GFLOP/s against the derived peak,
    with the fraction of the measured FMA throughput beside it."""
    peak, meas = fma_peak(name), measured_peak(name)
    return dict({"bound": "alu", "achieved": round(achieved, 2), "peak": peak, "unit": "GFLOP/s",
                 "frac": round(achieved / peak, 4), "peak_source": PEAK_SOURCE,
                 "measured_peak": meas, "frac_of_measured": round(achieved / meas, 4)}, **extra)
ORACLE_ITERS_PER_STEP = 3


# Source files of the FP64 Jacobi SVT kernel.  A committed ncu summary under profiles/
# carries a "traffic-record:" line with the DRAM bytes per launch it measured and the
# sha256 of these files at capture time; the bench line reports that traffic only while
# the files still hash the same (else null: the counters describe another kernel).
JACOBI_FP64_SOURCES = [f"paper_2202_02870_gb300/csrc/{f}" for f in (
    "lt_jacobi_svt.cuh", "lt_jacobi_common.cuh", "lt_internal.cuh", "lt_jacobi.cu",
    "lt_jacobi_f64_a.cu", "lt_jacobi_f64_b.cu", "lt_jacobi_f64_c.cu",
    "lt_jacobi_cluster.cuh", "lt_jacobi_cl.cu")]


def sources_sha256(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(kernel):
    import glob
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as fh:
            for line in fh:
                if not line.startswith("traffic-record:"):
                    continue
                try:
                    rec = json.loads(line.split(":", 1)[1])
                    if rec["kernel"] == kernel and rec["sources_sha256"] == sources_sha256(rec["files"]):
                        return int(rec["dram_bytes_per_launch"])
                except Exception:
                    continue
    return None


# HBM copy bandwidth of a GB300 as recorded in MEASURED_PEAKS.json (hbm_gbs) before this
# code was tuned; used when that file is not present.
HBM_GBS_RECORDED = 6799.6


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def hbm_peak():
    """(GB/s, source) of the HBM roofline."""
    v = load_peaks().get("hbm_gbs")
    if v:
        return float(v), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    return HBM_GBS_RECORDED, "MEASURED_PEAKS.json hbm_gbs as recorded in bench.py (of measured)"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws, device):
    """The largest value of x over the ranks of the process group (x itself at N = 1):
    the job's step time is the slowest rank's."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, ws, step_ms):
    """Whole-job throughput: the units every rank processed in a step over the slowest
    rank's step time (ms)."""
    return ws * units_per_rank / (step_ms / 1e3)


def problem_inputs(rank):
    """Seeded config-2 problem; rank r uses problem index r."""
    from paper_2202_02870_gb300 import synth
    c = synth.completion_case(2, 144, 176, (3, 32), rank=10, rho=0.3, problem=rank)
    c.update(tau=0.5, step=1.0, iters=100)
    return c


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.out.close()

    def summary(self):
        res = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if not self.path or not os.path.exists(self.path):
            return res
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            res = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                   "reasons": sorted(reasons), "samples": len(sm)}
        return res


def run_ours(args):
    import torch
    import torch.distributed as dist
    from oracle import lt_oracle as O  # used by the cpu_baseline leg only
    from paper_2202_02870_gb300 import lt

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    c = problem_inputs(rank)
    shape = (144, 176, 3, 32)
    tshape = tuple(reversed(shape))
    N = int(np.prod(shape))
    iters = c["iters"]

    def ctx_for(prec):
        ctx = lt.Context([3, 32], [lt.lt_make_dct(3), lt.lt_make_dct(32)], prec)
        warm = args.warm if prec == lt.LT_FP64 else args.warm32
        if warm:
            lt.lt_ctx_set_option(ctx, lt.LT_OPT_WARM_START, warm)
        return ctx

    ctx64 = ctx_for(lt.LT_FP64)
    # ground truth X = U *_L V^T with the library's own product (a10), then obs on host
    to_dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a.ravel(order="F"))).to(dt).reshape(
        tuple(reversed(a.shape))).to(dev)
    Ud = to_dev(c["U"], torch.float64)
    Vt = np.asfortranarray(np.swapaxes(c["V"], 0, 1))
    Vd = to_dev(Vt, torch.float64)
    Xtrue = torch.empty(tshape, dtype=torch.float64, device=dev)
    lt.lt_product(ctx64, Ud, Vd, Xtrue)
    torch.cuda.synchronize()
    xt = Xtrue.cpu().numpy().reshape(-1).reshape(shape, order="F")
    obs_np = c["mask"] * (xt + c["noise"])
    mask_d = torch.from_numpy(np.ascontiguousarray(c["mask"].ravel(order="F"))).reshape(tshape).to(dev)
    obs64 = to_dev(obs_np, torch.float64)
    obs32 = obs64.float()

    # autotuner: the SVT kernel form of each context is picked by timing the forms on the
    # first iterate's thresholding input (the observations, step * tau), outside the
    # timed region
    tuned = {}

    def tune(ctx, obs, name):
        D = torch.empty_like(obs)
        rep = lt.lt_autotune_svt(ctx, obs, c["tau"] * c["step"], D)
        tuned[name] = {"jacobi_group": rep.jacobi_group, "jacobi_block": rep.jacobi_block,
                       "forms_timed": rep.candidates, "best_ms": round(rep.best_ms, 3),
                       "default_ms": round(rep.default_ms, 3)}
        return ctx

    tune(ctx64, obs64, "fp64")
    for name in ("fp64", "fp32"):
        fma_peak(name)
        measured_peak(name)

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def run_path(ctx, obs, dt, K, W, profile):
        """W warm-up steps, then K timed steps; with `profile` the library brackets every
        kernel launch of the timed steps with CUDA events on its stream (per-kernel times
        and rooflines over the timed region)."""
        X = torch.zeros(tshape, dtype=dt, device=dev)
        wsb = torch.empty(lt.lt_workspace_size(ctx, lt.LT_OP_PGA, 144, 176), dtype=torch.uint8, device=dev)
        rep = lt.lt_pga_report()
        for _ in range(W):
            X.zero_()
            lt.lt_pga_complete(ctx, mask_d, obs, c["tau"], c["step"], iters, X, report=rep, ws=wsb)
        torch.cuda.synchronize()
        lt.lt_ctx_get_stats(ctx, reset=True)
        lt.lt_ctx_set_option(ctx, lt.LT_OPT_PROFILE, 1 if profile else 0)
        st = torch.cuda.current_stream()
        times = []
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(K):
            flush.zero_()
            X.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            lt.lt_pga_complete(ctx, mask_d, obs, c["tau"], c["step"], iters, X, report=rep, ws=wsb)
            e1.record(st)
            times.append((e0, e1))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if ws > 1:
            dist.barrier()
        ms = [a.elapsed_time(b) for a, b in times]
        stats = lt.lt_ctx_get_stats(ctx, reset=True)
        lt.lt_ctx_set_option(ctx, lt.LT_OPT_PROFILE, 0)
        stats["timed_launches"] = sum(stats[f]["launches"] for f in ("transform", "jacobi", "gemm", "aux"))
        return X, ms, wall, stats, rep

    # ---------------- FP64 path (value) with clocks and the Jacobi roofline
    with ClockSampler(local) as clk:
        X64, ms64, wall64, st64, rep64 = run_path(ctx64, obs64, torch.float64, args.steps,
                                                  args.warmup, True)
    clocks = clk.summary()
    step_ms = max_over_ranks(statistics.mean(ms64), ws, dev)
    value = job_rate(iters, ws, step_ms)

    jac = st64["jacobi"]
    tra = st64["transform"]
    jac_launches = max(jac["launches"], 1)
    jac_ms_avg = jac["ms"] / jac_launches
    jac_flops_avg = jac["flops"] / jac_launches
    achieved = jac_flops_avg / (jac_ms_avg / 1e3) / 1e9 if jac_ms_avg > 0 else 0.0
    families = ("transform", "jacobi", "gemm", "aux")
    gpu_launches = st64["timed_launches"]  # launches of the K timed steps
    slices_per_s = 96 / (jac_ms_avg / 1e3) if jac_ms_avg > 0 else 0.0

    # ---------------- FP32 and mixed (LT_MIXED: tensor-core mode-32 passes) paths on the
    # same inputs
    def single_leg(prec, label, tc_mode_min=None):
        name = {lt.LT_FP32: "fp32", lt.LT_MIXED: "mixed"}[prec]
        ctxp = ctx_for(prec)
        if tc_mode_min is not None:
            lt.lt_ctx_set_option(ctxp, lt.LT_OPT_TC_MODE_MIN, tc_mode_min)
            name += f"_tc{tc_mode_min}"
        ctxp = tune(ctxp, obs32, name)
        Xp, msp, _, stp, repp = run_path(ctxp, obs32, torch.float32, args.steps, args.warmup, True)
        mean_ms = statistics.mean(msp)
        relp = float(torch.linalg.norm(Xp.double() - X64) / torch.linalg.norm(X64))
        jp = stp["jacobi"]
        jp_ms = jp["ms"] / max(jp["launches"], 1)
        jp_flops = jp["flops"] / max(jp["launches"], 1)
        jp_ach = jp_flops / (jp_ms / 1e3) / 1e9 if jp_ms > 0 else 0.0
        tr = stp["transform"]
        return {"dtype": label, "value": round(ws * iters / (mean_ms / 1e3), 3),
                "unit": "iters/s", "ms_per_step": round(mean_ms, 3),
                "rel_err_vs_fp64": relp,
                "svt_slices_per_s": round(96 / (jp_ms / 1e3), 1) if jp_ms > 0 else None,
                "transform_ms_per_step": round(tr["ms"] / args.steps, 3),
                "tc_launches_per_step": stp["tc_launches"] / args.steps,
                "max_sweeps": repp.max_sweeps_used,
                "jacobi_flops_per_launch": jp_flops,
                "roofline": alu_roofline(jp_ach, "fp32", kernel="jacobi_svt (FP32)")}

    fp32_leg = single_leg(lt.LT_FP32, "f32")
    # LT_MIXED with the library's defaults: modes 3 and 32 are below LT_OPT_TC_MODE_MIN
    # (64), so this workload runs the FP32 kernels (tc_launches_per_step = 0)
    mixed_leg = single_leg(lt.LT_MIXED, "f32 (LT_MIXED defaults: no mode of this workload "
                                        "reaches the tensor cores)")
    # LT_MIXED with the mode-32 products on the tcgen05 tensor cores (split TF32 x 3)
    mixed_tc_leg = single_leg(lt.LT_MIXED, "f32 + mode-32 products on the tensor cores "
                                           "(split tf32x3)", tc_mode_min=32)

    # ---------------- the Fourier operator (TNN-PGA-F, Sec. 5) on the same observations
    fourier = None
    if args.fourier_steps > 0:
        fourier = fourier_leg(args, dev, ws, mask_d, obs64, c, flush,
                              rank == 0 and ws == 1 and not args.no_cpu)

    # ---------------- batched: the 64 uneven problems of one batch, FP32
    batched = None
    if args.batched_steps > 0:
        batched = run_batched_leg(args, dev, ws)

    # ---------------- L-SVT slices/s (config 2 with transforms; config 3's 2048 slices)
    svt = None
    if args.svt_steps > 0 and rank == 0:
        svt = svt_legs(dev, obs64, c, flush, args.svt_steps)

    # ---------------- the fifth-order *_L-product (face-wise GEMM on the tensor cores)
    product = None
    if args.product_steps > 0 and rank == 0:
        product = product5_leg(["mixed", "fp32"], args.product_steps, 2)

    # ---------------- e2e: host buffers through the C ABI, copies inside each step
    mask_h = torch.from_numpy(np.ascontiguousarray(c["mask"].ravel(order="F"))).reshape(tshape).pin_memory()
    obs_h = obs64.cpu().pin_memory()
    out_h = torch.empty(tshape, dtype=torch.float64).pin_memory()
    mask_e = torch.empty_like(mask_d)
    obs_e = torch.empty_like(obs64)
    Xe = torch.empty_like(X64)
    wse = torch.empty(lt.lt_workspace_size(ctx64, lt.LT_OP_PGA, 144, 176), dtype=torch.uint8, device=dev)
    e2e_ms = []
    st = torch.cuda.current_stream()
    lt.lt_ctx_set_option(ctx64, lt.LT_OPT_PROFILE, 1)  # same conditions as the timed steps
    for _ in range(max(1, args.steps // 2)):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        mask_e.copy_(mask_h, non_blocking=True)
        obs_e.copy_(obs_h, non_blocking=True)
        Xe.zero_()
        lt.lt_pga_complete(ctx64, mask_e, obs_e, c["tau"], c["step"], iters, Xe, ws=wse)
        out_h.copy_(Xe, non_blocking=True)
        e1.record(st)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    lt.lt_ctx_set_option(ctx64, lt.LT_OPT_PROFILE, 0)
    lt.lt_ctx_get_stats(ctx64, reset=True)
    e2e_step = max_over_ranks(statistics.mean(e2e_ms), ws, dev)

    # ---------------- CPU baseline: the oracle on the host cores (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        Ms = [O.dct_matrix(3), O.dct_matrix(32)]
        t0 = time.perf_counter()
        O.pga(c["mask"], obs_np, c["tau"], c["step"], args.cpu_iters, Ms)
        dt = time.perf_counter() - t0
        cpu = {"value": args.cpu_iters / dt, "unit": "iters/s", "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": f"{args.cpu_iters} PGA iterations of the same 144x176x3x32 problem "
                         f"({dt:.1f} s), numpy/LAPACK FP64, BLAS threads = all host cores",
               "single_thread": oracle_single_thread(obs_np, c, 3)}

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": round(value, 5),
            "unit": "iters/s",
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(step_ms, 3),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f64",
            "data": "synthetic: seeded low-L-rank tensor X = U *_L V^T (N(0,1) factors, "
                    "rank 10) + N(0,1e-3) noise, Bernoulli(0.3) mask; stands in for the "
                    "paper's colour videos",
            "config": {"workload": WORKLOAD, "shape": [144, 176, 3, 32], "transforms": ["dct3", "dct32"],
                       "tau": 0.5, "step": 1.0, "iters_per_step": iters, "rank": 10, "observed": 0.3,
                       "warm_start_period": {"fp64": args.warm, "fp32_mixed": args.warm32},
                       "l2": "flushed between steps (512 MiB write)",
                       "parallelism": f"replicas x{ws}"},
            "svt_slices_per_s": round(slices_per_s, 1),
            "mixed": mixed_leg,
            "mixed_tc32": mixed_tc_leg,
            "fp32": fp32_leg,
            "autotune": tuned,
            "fma_peaks_gflops": {"derived": DERIVED_PEAKS, "measured": FMA_PEAKS,
                                 "source": PEAK_SOURCE},
            "batched": batched,
            "fourier": fourier,
            "product_256x256x16x16x8": product,
            "svt": svt,
            "roofline": alu_roofline(achieved, "fp64", kernel="jacobi_svt (FP64)",
                                     traffic=profiled_traffic("jacobi_svt_fp64"),
                                     flops_per_launch=jac_flops_avg,
                                     ms_per_launch=round(jac_ms_avg, 4)),
            "kernels": {f: {"launches": st64[f]["launches"], "ms": round(st64[f]["ms"], 3),
                            "share": round(st64[f]["ms"] / max(sum(st64[x]["ms"] for x in families), 1e-9), 4)}
                        for f in families},
            "transform_roofline": {
                "bound": "alu", "achieved": round(tra["flops"] / max(tra["ms"], 1e-9) / 1e6, 2),
                "unit": "GFLOP/s", "peak": fma_peak("fp64"), "frac": round(
                    tra["flops"] / max(tra["ms"], 1e-9) / 1e6 / fma_peak("fp64"), 4),
                "hbm_gbs": round(tra["bytes"] / max(tra["ms"], 1e-9) / 1e6, 1),
                "hbm_peak_gbs": hbm_peak()[0]},
            "e2e": {"value": round(job_rate(iters, ws, e2e_step), 5), "unit": "iters/s",
                    "ms_per_step": round(e2e_step, 3),
                    "h2d_bytes_per_step": int(N + N * 8), "d2h_bytes_per_step": int(N * 8)},
            "gpu_launches": int(gpu_launches),
            "clocks": clocks,
            "report": {"iters_done": rep64.iters_done, "rel_residual": rep64.rel_residual,
                       "max_sweeps": rep64.max_sweeps_used, "device_status": rep64.device_status},
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


def oracle_single_thread(obs_np, c, iters):
    """The oracle's PGA on one host thread (BLAS and OpenMP pools set to 1 before numpy
    loads, in a child process), the setting of the paper's single-core timings: `iters`
    iterations of the same problem.  Returns {"value", "unit", "cores": 1, "sample"} or
    {"error": ...}; never raises."""
    with tempfile.TemporaryDirectory() as td:
        np.save(os.path.join(td, "obs.npy"), obs_np)
        np.save(os.path.join(td, "mask.npy"), c["mask"])
        code = (
            "import sys, time, json, numpy as np\n"
            f"sys.path.insert(0, {ROOT!r})\n"
            "from oracle import lt_oracle as O\n"
            f"obs = np.load({os.path.join(td, 'obs.npy')!r})\n"
            f"mask = np.load({os.path.join(td, 'mask.npy')!r})\n"
            "Ms = [O.dct_matrix(3), O.dct_matrix(32)]\n"
            "t0 = time.perf_counter()\n"
            f"O.pga(mask, obs, {c['tau']!r}, {c['step']!r}, {int(iters)}, Ms)\n"
            "print(json.dumps({'seconds': time.perf_counter() - t0}))\n")
        env = dict(os.environ)
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
                    "BLIS_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
            env[var] = "1"
        try:
            r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True,
                               text=True, timeout=300)
            sec = json.loads(r.stdout.strip().splitlines()[-1])["seconds"]
        except Exception as e:  # the baseline is a report, not part of the product path
            return {"error": f"{type(e).__name__}: {str(e)[:200]}"}
    return {"value": round(iters / sec, 4), "unit": "iters/s", "cores": 1,
            "sample": f"{iters} PGA iterations of the same problem ({sec:.1f} s), BLAS and "
                      "OpenMP pools of one thread"}


def fourier_leg(args, dev, ws, mask_d, obs64, c, flush, cpu):
    """TNN-PGA-F: PGA with M_3 = F_3 (t-product operator) and M_4 = DCT 32 on the
    144x176x3x32 observations (lt_ctx_create_fourier), FP64 and FP32; `--fourier-iters`
    iterations per step, 3 warm-up steps, `--fourier-steps` timed steps with CUDA
    events.  With `cpu` (rank 0, N = 1) the oracle's TNN-PGA-F is timed on a sample of
    two iterations of the same problem."""
    import torch
    from paper_2202_02870_gb300 import lt
    iters = args.fourier_iters
    out = {"operator": "F_3 (t-product) x DCT 32", "iters_per_step": iters,
           "slices": "32 real 144x176 + 32 realified 288x352 per iteration"}
    X64 = None
    for prec, label, dt in ((lt.LT_FP64, "f64", torch.float64), (lt.LT_FP32, "f32", torch.float32)):
        ctx = lt.lt_ctx_create_fourier([3, 32], [lt.lt_make_dct(32)], prec)
        obs = obs64.to(dt)
        X = torch.zeros_like(obs)
        wsb = torch.empty(lt.lt_workspace_size(ctx, lt.LT_OP_PGA, 144, 176), dtype=torch.uint8,
                          device=dev)
        rep = lt.lt_pga_report()
        for _ in range(3):
            X.zero_()
            lt.lt_pga_complete(ctx, mask_d, obs, c["tau"], c["step"], iters, X, report=rep, ws=wsb)
        torch.cuda.synchronize()
        lt.lt_ctx_get_stats(ctx, reset=True)
        lt.lt_ctx_set_option(ctx, lt.LT_OPT_PROFILE, 1)
        st = torch.cuda.current_stream()
        ms = []
        for _ in range(args.fourier_steps):
            flush.zero_()
            X.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            lt.lt_pga_complete(ctx, mask_d, obs, c["tau"], c["step"], iters, X, report=rep, ws=wsb)
            e1.record(st)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        stats = lt.lt_ctx_get_stats(ctx, reset=True)
        lt.lt_ctx_set_option(ctx, lt.LT_OPT_PROFILE, 0)
        step_ms = max_over_ranks(statistics.mean(ms), ws, dev)
        jac = stats["jacobi"]
        gflops = jac["flops"] / max(jac["ms"], 1e-9) / 1e6
        leg = {"value": round(job_rate(iters, ws, step_ms), 4), "unit": "iters/s",
               "ms_per_iter": round(step_ms / iters, 3),
               "jacobi_ms_per_iter": round(jac["ms"] / max(args.fourier_steps * iters, 1), 3),
               "roofline": alu_roofline(gflops, "fp64" if prec == lt.LT_FP64 else "fp32",
                                        kernel=f"jacobi_svt ({label.upper()})"),
               "rel_residual": rep.rel_residual, "device_status": rep.device_status}
        if X64 is None:
            X64 = X.double()
        else:
            leg["rel_err_vs_fp64"] = float(torch.linalg.norm(X.double() - X64) / torch.linalg.norm(X64))
        out[label] = leg
    if cpu:
        from oracle import lt_oracle as O  # the cpu_baseline sample only
        obs_np = obs64.cpu().numpy().reshape(-1).reshape((144, 176, 3, 32), order="F")
        t0 = time.perf_counter()
        O.pga(c["mask"], obs_np, c["tau"], c["step"], 2, [O.dct_matrix(32)], fourier=True)
        dtc = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": round(2 / dtc, 4), "unit": "iters/s",
                               "cores": os.cpu_count(), "kind": "oracle",
                               "sample": f"2 TNN-PGA-F iterations of the same problem ({dtc:.1f} s), "
                                         "numpy complex FFT + LAPACK SVD, FP64"}
    return out


def run_batched_leg(args, dev, ws):
    """The 64 independent completion problems of uneven sizes (I1 x I2 from 64 x 48 to
    512 x 384, I3 = 3, I4 in {8, 16, 32, 64}, DCT transforms) as one
    lt_pga_complete_batched call (a CUDA graph with a branch per problem):
    mixed  LT_MIXED, `--batched-iters` iterations per call, `--batched-steps` timed
           calls after one warm-up call, against the same problems issued one after the
           other; the Jacobi flops the kernels counted over the wall time against the
           derived FP32 FMA peak;
    fp64   the same problems in FP64, `--batched-iters-fp64` iterations, one timed call
           (no warm-up: a call takes seconds), and the relative error of the mixed
           iterates against the FP64 ones after the same iterations."""
    import torch
    from paper_2202_02870_gb300 import lt, synth
    shapes = synth.config4_shapes()
    rng = np.random.default_rng(4)
    masks, obs64 = [], []
    elems = 0
    for sh in shapes:
        full = (sh["I1"], sh["I2"]) + sh["trailing"]
        elems += int(np.prod(full))
        m = torch.from_numpy((rng.random(int(np.prod(full))) < sh["rho"]).astype(np.uint8))
        masks.append(m.reshape(tuple(reversed(full))).to(dev))
        obs64.append(masks[-1].double() * torch.randn(tuple(reversed(full)), device=dev,
                                                      dtype=torch.float64))
    n = len(shapes)
    out = {"problems": n, "elements": elems}
    finals = {}
    for name, prec, dt in (("mixed", lt.LT_MIXED, torch.float32), ("fp64", lt.LT_FP64, torch.float64)):
        iters = args.batched_iters if name == "mixed" else args.batched_iters_fp64
        steps = args.batched_steps if name == "mixed" else 1
        ctxs = [lt.Context(list(sh["trailing"]), [lt.lt_make_dct(k) for k in sh["trailing"]], prec)
                for sh in shapes]
        obss = [o.to(dt) for o in obs64]
        Xs = [torch.zeros_like(o) for o in obss]
        wsb = torch.empty(lt.lt_workspace_size_batched(ctxs, [x.shape[-1] for x in Xs],
                                                       [x.shape[-2] for x in Xs]),
                          dtype=torch.uint8, device=dev)

        def run():
            for x in Xs:
                x.zero_()
            lt.lt_pga_complete_batched(ctxs, masks, obss, [0.5] * n, [1.0] * n, iters, Xs, ws=wsb)

        if name == "mixed":
            run()
        torch.cuda.synchronize()
        for cx in ctxs:
            lt.lt_ctx_get_stats(cx, reset=True)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(steps):
            run()
        e1.record(st)
        torch.cuda.synchronize()
        ms_b = e0.elapsed_time(e1) / steps
        flops = sum(lt.lt_ctx_get_stats(cx, reset=True)["jacobi"]["flops"] for cx in ctxs) / steps
        leg = {"dtype": "f32 + split-tf32x3 tensor cores (I4 = 64 problems' mode-4 products)"
                        if name == "mixed" else "f64",
               "iters_per_step": iters, "steps": steps,
               "value": round(ws * n * iters / (ms_b / 1e3), 3), "unit": "problem-iters/s",
               "ms_per_step": round(ms_b, 2),
               "jacobi_roofline": alu_roofline(
                   flops / (ms_b / 1e3) / 1e9, "fp32" if name == "mixed" else "fp64",
                   note="Jacobi flops counted by the kernels over the whole batch call's "
                        "wall time")}
        if name == "mixed":
            # the same work, one problem after the other on one stream
            e0.record(st)
            for i in range(n):
                Xs[i].zero_()
                lt.lt_pga_complete(ctxs[i], masks[i], obss[i], 0.5, 1.0, iters, Xs[i])
            e1.record(st)
            torch.cuda.synchronize()
            ms_s = e0.elapsed_time(e1)
            leg["sequential_ms"] = round(ms_s, 2)
            leg["speedup_vs_sequential"] = round(ms_s / ms_b, 3)
            if args.batched_iters_fp64 != iters:
                # the mixed iterates at the FP64 leg's iteration count, for the error
                for x in Xs:
                    x.zero_()
                lt.lt_pga_complete_batched(ctxs, masks, obss, [0.5] * n, [1.0] * n,
                                           args.batched_iters_fp64, Xs, ws=wsb)
                torch.cuda.synchronize()
        finals[name] = [x.double() for x in Xs]
        out[name] = leg
        del ctxs, obss, Xs, wsb
        torch.cuda.empty_cache()
    num = sum(float(torch.linalg.norm(a - b) ** 2) for a, b in zip(finals["mixed"], finals["fp64"]))
    den = sum(float(torch.linalg.norm(b) ** 2) for b in finals["fp64"])
    out["mixed"]["rel_err_vs_fp64"] = (num / den) ** 0.5
    out["mixed"]["rel_err_iters"] = args.batched_iters_fp64
    out["mixed_over_fp64"] = round(out["mixed"]["value"] / out["fp64"]["value"], 2)
    return out


def svt_rate(ctx, G, tau, D, wsb, units, steps, warmup, flush):
    """Per-call time of lt_svt (transforms included) and of its Jacobi launch alone (the
    library's CUDA events), L2 flushed before every timed call."""
    import torch
    from paper_2202_02870_gb300 import lt
    for _ in range(warmup):
        lt.lt_svt(ctx, G, tau, D, ws=wsb)
    torch.cuda.synchronize()
    lt.lt_ctx_get_stats(ctx, reset=True)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_PROFILE, 1)
    st = torch.cuda.current_stream()
    ms = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        lt.lt_svt(ctx, G, tau, D, ws=wsb)
        e1.record(st)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    stats = lt.lt_ctx_get_stats(ctx, reset=True)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_PROFILE, 0)
    jac = stats["jacobi"]
    jms = jac["ms"] / max(jac["launches"], 1)
    call = statistics.mean(ms)
    return {"ms_per_call": round(call, 3), "slices_per_s": round(units / (call / 1e3), 1),
            "jacobi_ms_per_launch": round(jms, 3),
            "jacobi_slices_per_s": round(units / (jms / 1e3), 1) if jms > 0 else None,
            "jacobi_gflops_executed": round(jac["flops"] / max(jac["ms"], 1e-9) / 1e6, 1),
            "transform_ms_per_call": round(stats["transform"]["ms"] / steps, 3),
            "tc_launches_per_call": stats["tc_launches"] / steps}


def svt_legs(dev, obs64, c, flush, steps):
    """L-SVT slices/s (Algorithm 4, transforms included, and the Jacobi launch alone):
    config 2: the 96 transform-domain slices (144 x 176) of G = P_Omega(M), the first
              PGA iterate's input, tau 0.5, FP64 and FP32;
    config 3: the 256x256x16x16x8 tensor (U[-1,1], L_k = Q_k diag(d_k), cond 1e2 each),
              2048 slices of 256 x 256, tau = 0.1 x the median largest singular value
              of four sampled transform-domain slices, FP64, FP32 and LT_MIXED (its
              modes 16, 16, 8 are below LT_OPT_TC_MODE_MIN, so it runs the FP32 kernels),
              with the errors of FP32 / LT_MIXED against the FP64 result."""
    import torch
    from paper_2202_02870_gb300 import lt, synth
    out = {"config2_144x176x3x32": {}, "config3_256x256x16x16x8": {}}
    mats2 = [lt.lt_make_dct(3), lt.lt_make_dct(32)]
    for name, prec, dt in (("fp64", lt.LT_FP64, torch.float64), ("fp32", lt.LT_FP32, torch.float32)):
        ctx = lt.Context([3, 32], mats2, prec)
        G = obs64.to(dt)
        D = torch.empty_like(G)
        wsb = torch.empty(max(lt.lt_workspace_size(ctx, lt.LT_OP_SVT, 144, 176), 1),
                          dtype=torch.uint8, device=dev)
        leg = svt_rate(ctx, G, c["tau"], D, wsb, 96, steps, 2, flush)
        leg["jacobi_roofline"] = alu_roofline(leg["jacobi_gflops_executed"], name)
        out["config2_144x176x3x32"][name] = leg
    c3 = synth.config3()
    mats3 = [np.asarray(m) for _, m in c3["transforms"]]
    A64 = torch.from_numpy(np.ascontiguousarray(c3["A"].ravel(order="F"))).reshape(
        (8, 16, 16, 256, 256)).to(dev)
    ctx64 = lt.Context([16, 16, 8], mats3, lt.LT_FP64)
    Ah = torch.empty_like(A64)
    lt.lt_transform(ctx64, A64, Ah)
    samples = [0, 513, 1337, 2047]
    sl = Ah.reshape(2048, 256, 256)[samples]
    tau3 = 0.1 * float(torch.quantile(torch.linalg.matrix_norm(sl, ord=2), 0.5).item())
    del Ah, sl
    D64 = None
    for name, prec, dt in (("fp64", lt.LT_FP64, torch.float64), ("fp32", lt.LT_FP32, torch.float32),
                           ("mixed", lt.LT_MIXED, torch.float32)):
        ctx = ctx64 if prec == lt.LT_FP64 else lt.Context([16, 16, 8], mats3, prec)
        G = A64.to(dt)
        D = torch.empty_like(G)
        wsb = torch.empty(max(lt.lt_workspace_size(ctx, lt.LT_OP_SVT, 256, 256), 1),
                          dtype=torch.uint8, device=dev)
        n = 1 if prec == lt.LT_FP64 else max(1, min(steps, 3))
        leg = svt_rate(ctx, G, tau3, D, wsb, 2048, n, 1, flush)
        leg["jacobi_roofline"] = alu_roofline(leg["jacobi_gflops_executed"],
                                              "fp64" if prec == lt.LT_FP64 else "fp32")
        leg["device_status"] = lt.lt_last_device_status(ctx)
        if D64 is None:
            D64 = D.double()
        else:
            leg["rel_err_vs_fp64"] = float(torch.linalg.norm(D.double() - D64) / torch.linalg.norm(D64))
        out["config3_256x256x16x16x8"][name] = leg
        del G, D, wsb
    out["config3_256x256x16x16x8"]["tau"] = tau3
    del A64, D64
    torch.cuda.empty_cache()
    return out


def run_case(args):
    """Auxiliary single-operation runs used for profiling (not the benchmark line):
    --case svt     lt_svt (tau 0.5) of the 144x176x3x32 tensor G = P_Omega(M) of the
                   completion problem (what the first PGA iteration thresholds);
    --case product lt_product U *_L V^T of its 144x10x3x32 and 10x176x3x32 factors."""
    import torch
    from paper_2202_02870_gb300 import lt
    prec = {"fp64": lt.LT_FP64, "fp32": lt.LT_FP32, "mixed": lt.LT_MIXED}[args.precision]
    dt = torch.float64 if prec == lt.LT_FP64 else torch.float32
    c = problem_inputs(0)
    dev = torch.device("cuda", 0)
    to_dev = lambda a: torch.from_numpy(np.ascontiguousarray(a.ravel(order="F"))).to(dt).reshape(
        tuple(reversed(a.shape))).to(dev)
    ctx = lt.Context([3, 32], [lt.lt_make_dct(3), lt.lt_make_dct(32)], prec)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_JACOBI_GROUP, args.jacobi_group)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_JACOBI_BLOCK, args.jacobi_pairwise)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_JACOBI_CLUSTER, args.jacobi_cluster)
    if args.case == "svt":
        G = to_dev(c["mask"] * np.random.default_rng(1).standard_normal(c["mask"].shape))
        D = torch.empty_like(G)
        wsb = torch.empty(max(lt.lt_workspace_size(ctx, lt.LT_OP_SVT, 144, 176), 1),
                          dtype=torch.uint8, device=dev)
        run = lambda: lt.lt_svt(ctx, G, 0.5, D, ws=wsb)
        units, unit = 96, "slices"
    else:
        U = to_dev(c["U"])
        Vt = to_dev(np.asfortranarray(np.swapaxes(c["V"], 0, 1)))
        X = torch.empty((32, 3, 176, 144), dtype=dt, device=dev)
        run = lambda: lt.lt_product(ctx, U, Vt, X)
        units, unit = 1, "products"
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"case": args.case, "precision": args.precision,
                      "jacobi_group": args.jacobi_group, "jacobi_pairwise": args.jacobi_pairwise,
                      "jacobi_cluster": args.jacobi_cluster,
                      "ms_per_call": ms,
                      f"{unit}_per_s": units / (ms / 1e3)}))


def product5_leg(precisions, steps, warmup, tile_n=0):
    """The fifth-order *_L-product 256x256x16x16x8 times 256x128x16x16x8 (U[-1,1];
    L_k = Q_k diag(d_k), cond 1e2 each) through lt_product: three transforms (modes
    16, 16, 8) and the face-wise GEMM of 2048 slices of (256x256)(256x128).  Per
    precision: per-call time, per-family event times, and the GEMM kernel against the
    HBM roofline (algorithmic bytes: read L(A) and L(B) once, write L(C) once) with, for
    LT_MIXED, the tensor-pipe rate of the three TF32 products it issues."""
    import torch
    from paper_2202_02870_gb300 import lt, synth
    c = synth.config3()
    dev = torch.device("cuda", 0)
    hbm, hbm_src = hbm_peak()
    host = {"A": c["A"], "B": c["B"]}
    out = {}
    # the FP64 GPU product of the same operands: the reference of the other precisions'
    # errors (the FP64 path itself is pinned to the oracle by the parity tests)
    C64 = None
    if any(p in ("fp32", "mixed") for p in precisions):
        to64 = lambda a: torch.from_numpy(np.ascontiguousarray(a.ravel(order="F"))).reshape(
            tuple(reversed(a.shape))).to(dev)
        ctx64 = lt.Context([16, 16, 8], [np.asarray(m) for _, m in c["transforms"]], lt.LT_FP64)
        A64, B64 = to64(host["A"]), to64(host["B"])
        C64 = torch.empty((8, 16, 16, 128, 256), dtype=torch.float64, device=dev)
        lt.lt_product(ctx64, A64, B64, C64)
        torch.cuda.synchronize()
        del A64, B64, ctx64
    for name in precisions:
        prec = {"fp64": lt.LT_FP64, "fp32": lt.LT_FP32, "mixed": lt.LT_MIXED}[name]
        dt = torch.float64 if prec == lt.LT_FP64 else torch.float32
        to_dev = lambda a: torch.from_numpy(np.ascontiguousarray(a.ravel(order="F"))).to(dt).reshape(
            tuple(reversed(a.shape))).to(dev)
        A, B = to_dev(host["A"]), to_dev(host["B"])
        ctx = lt.Context([16, 16, 8], [np.asarray(m) for _, m in c["transforms"]], prec)
        if tile_n:
            lt.lt_ctx_set_option(ctx, lt.LT_OPT_TC_TILE_N, tile_n)
        Cd = torch.empty((8, 16, 16, 128, 256), dtype=dt, device=dev)
        ws = torch.empty(lt.lt_workspace_size(ctx, lt.LT_OP_PRODUCT, 256, 256, 128),
                         dtype=torch.uint8, device=dev)
        run = lambda: lt.lt_product(ctx, A, B, Cd, ws=ws)
        for _ in range(warmup):
            run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            run()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        lt.lt_ctx_get_stats(ctx, reset=True)
        lt.lt_ctx_set_option(ctx, lt.LT_OPT_PROFILE, 1)
        for _ in range(steps):
            run()
        st = lt.lt_ctx_get_stats(ctx, reset=True)
        g = st["gemm"]
        g_ms = g["ms"] / max(g["launches"], 1)
        gemm_bytes = g["bytes"] / max(g["launches"], 1)
        gemm_flops = g["flops"] / max(g["launches"], 1)
        tr = st["transform"]
        leg = {"ms_per_call": round(ms, 4), "products_per_s": round(1e3 / ms, 3),
               "kernels_ms_per_call": {k: round(st[k]["ms"] / steps, 4)
                                       for k in ("transform", "gemm", "aux")},
               "tc_launches_per_call": st["tc_launches"] / steps,
               "gemm_roofline": {"bound": "hbm", "achieved": round(gemm_bytes / g_ms / 1e6, 1),
                                 "peak": hbm, "unit": "GB/s", "peak_source": hbm_src,
                                 "frac": round(gemm_bytes / g_ms / 1e6 / hbm, 4),
                                 "algorithmic_bytes": gemm_bytes, "ms_per_launch": round(g_ms, 4),
                                 "tflops_algorithmic": round(gemm_flops / g_ms / 1e9, 2)},
               "transform_roofline": {"bound": "hbm",
                                      "achieved": round(tr["bytes"] / max(tr["ms"], 1e-9) / 1e6, 1),
                                      "peak": hbm, "unit": "GB/s", "peak_source": hbm_src,
                                      "frac": round(tr["bytes"] / max(tr["ms"], 1e-9) / 1e6 / hbm, 4),
                                      "tflops_algorithmic": round(tr["flops"] / max(tr["ms"], 1e-9) / 1e9, 2)}}
        if prec == lt.LT_MIXED:
            leg["gemm_roofline"]["tflops_issued_tf32x3"] = round(3 * gemm_flops / g_ms / 1e9, 2)
        if C64 is not None and prec != lt.LT_FP64:
            leg["rel_err_vs_fp64"] = float(torch.linalg.norm(Cd.double() - C64) / torch.linalg.norm(C64))
        out[name] = leg
        del A, B, Cd, ws, ctx
        torch.cuda.empty_cache()
    del C64
    torch.cuda.empty_cache()
    return out


def run_product5(args):
    """--case product5: the fifth-order product leg alone, one precision."""
    leg = product5_leg([args.precision], args.steps, args.warmup, args.tc_tile_n)[args.precision]
    print(json.dumps({"case": "product5", "precision": args.precision, **leg}))


def run_transform5(args):
    """--case transform5: lt_transform + lt_inverse of a 540x960x3x120 tensor (the large
    completion's shape; L_3 = DCT 3, L_4 = Q1 diag(d) Q2^T with cond 10), U[-1,1].
    Reports per-call times and the transform kernels against HBM (one read and one
    write of the tensor per pass) and the FP32 FMA rate."""
    import torch
    from paper_2202_02870_gb300 import lt, synth
    prec = {"fp64": lt.LT_FP64, "fp32": lt.LT_FP32, "mixed": lt.LT_MIXED}[args.precision]
    dt = torch.float64 if prec == lt.LT_FP64 else torch.float32
    rng = synth.rng_for(5, 1)
    M4 = synth.conditioned_matrix(rng, 120, 10.0, two_sided=True)
    ctx = lt.Context([3, 120], [lt.lt_make_dct(3), M4], prec)
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev)
    g.manual_seed(20220706)
    X = (torch.rand((120, 3, 960, 540), generator=g, device=dev, dtype=torch.float32) * 2 - 1).to(dt)
    Xh = torch.empty_like(X)
    run = lambda: (lt.lt_transform(ctx, X, Xh), lt.lt_inverse(ctx, Xh, Xh))
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    lt.lt_ctx_get_stats(ctx, reset=True)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_PROFILE, 1)
    for _ in range(args.steps):
        run()
    st = lt.lt_ctx_get_stats(ctx, reset=True)
    tr = st["transform"]
    print(json.dumps({"case": "transform5", "precision": args.precision,
                      "ms_per_transform_and_inverse": round(ms, 4),
                      "transform_kernel_ms": round(tr["ms"] / args.steps, 4),
                      "launches_per_call": tr["launches"] / args.steps,
                      "tc_launches_per_call": st["tc_launches"] / args.steps,
                      "gflops_algorithmic": round(tr["flops"] / max(tr["ms"], 1e-9) / 1e6, 1),
                      "hbm_gbs_algorithmic": round(tr["bytes"] / max(tr["ms"], 1e-9) / 1e6, 1),
                      "hbm_peak_gbs": hbm_peak()[0]}))


def run_pga5(args):
    """--case pga5: the large completion 540x960x3x120 (rank 15, noise 1e-3, 20%
    observed, L_3 = DCT 3, L_4 = Q1 diag(d) Q2^T with cond 10, tau 0.5, step 1), a few
    PGA iterations from a cold start on each path: FP64, FP32 and LT_MIXED (mode 120 on
    the tensor cores).  Reports ms per iteration, the Jacobi share, and the relative
    difference of the FP32 / mixed iterates from the FP64 one after the same iterations."""
    import torch
    from paper_2202_02870_gb300 import lt, synth
    c = synth.config5()
    dev = torch.device("cuda", 0)
    shape = (540, 960, 3, 120)
    tshape = tuple(reversed(shape))
    mats = [lt.lt_make_dct(3), np.asarray(c["transforms"][1][1])]
    ctx64 = lt.Context([3, 120], mats, lt.LT_FP64)
    to_dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a.ravel(order="F"))).to(dt).reshape(
        tuple(reversed(a.shape))).to(dev)
    U = to_dev(c["U"], torch.float64)
    Vt = to_dev(np.asfortranarray(np.swapaxes(c["V"], 0, 1)), torch.float64)
    Xt = torch.empty(tshape, dtype=torch.float64, device=dev)
    lt.lt_product(ctx64, U, Vt, Xt)
    mask = torch.from_numpy(np.ascontiguousarray(c["mask"].ravel(order="F"))).reshape(tshape).to(dev)
    obs64 = mask.double() * (Xt + to_dev(c["noise"], torch.float64))
    del U, Vt, Xt
    out = {"case": "pga5", "shape": list(shape), "iters": args.iters5}
    res = {}
    for name, prec in (("fp64", lt.LT_FP64), ("fp32", lt.LT_FP32), ("mixed", lt.LT_MIXED)):
        ctx = ctx64 if prec == lt.LT_FP64 else lt.Context([3, 120], mats, prec)
        dt = torch.float64 if prec == lt.LT_FP64 else torch.float32
        obs = obs64.to(dt)
        X = torch.zeros(tshape, dtype=dt, device=dev)
        wsb = torch.empty(lt.lt_workspace_size(ctx, lt.LT_OP_PGA, 540, 960), dtype=torch.uint8,
                          device=dev)
        lt.lt_ctx_get_stats(ctx, reset=True)
        lt.lt_ctx_set_option(ctx, lt.LT_OPT_PROFILE, 1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        lt.lt_pga_complete(ctx, mask, obs, 0.5, 1.0, args.iters5, X, ws=wsb)
        e1.record()
        torch.cuda.synchronize()
        st = lt.lt_ctx_get_stats(ctx, reset=True)
        ms = e0.elapsed_time(e1) / args.iters5
        res[name] = X.double()
        out[name] = {"ms_per_iter": round(ms, 2), "iters_per_s": round(1e3 / ms, 3),
                     "jacobi_share": round(st["jacobi"]["ms"] / max(sum(st[f]["ms"] for f in
                                           ("transform", "jacobi", "gemm", "aux")), 1e-9), 4),
                     "transform_ms_per_iter": round(st["transform"]["ms"] / args.iters5, 2),
                     "tc_launches": st["tc_launches"]}
        del X, wsb, obs
        torch.cuda.empty_cache()
    for name in ("fp32", "mixed"):
        out[name]["rel_diff_vs_fp64"] = float(torch.linalg.norm(res[name] - res["fp64"]) /
                                              torch.linalg.norm(res["fp64"]))
    if args.tol5 > 0:
        # run to the stopping test of Sec. 5 (r <= tol) on the chosen path, from a cold
        # start; FP64 time-to-residual extrapolated from its ms per iteration above
        name = args.precision if args.precision != "fp64" else "mixed"
        prec = {"fp32": lt.LT_FP32, "mixed": lt.LT_MIXED}[name]
        ctx = lt.Context([3, 120], mats, prec)
        obs = obs64.float()
        mu0 = 0.0
        if args.mu0_frac > 0:
            # continuation of Algorithm 5 with the paper's settings: mu_0 = nu ||M||_F,
            # nu = 0.9, mu_bar = tau
            mu0 = args.mu0_frac * float(torch.linalg.norm(obs64))
            lt.lt_ctx_set_option(ctx, lt.LT_OPT_MU0, mu0)
            lt.lt_ctx_set_option(ctx, lt.LT_OPT_NU, 0.9)
        X = torch.zeros(tshape, dtype=torch.float32, device=dev)
        wsb = torch.empty(lt.lt_workspace_size(ctx, lt.LT_OP_PGA, 540, 960), dtype=torch.uint8,
                          device=dev)
        rep = lt.lt_pga_report()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        lt.lt_pga_complete(ctx, mask, obs, 0.5, 1.0, args.max_iters5, X, tol=args.tol5,
                           report=rep, ws=wsb)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out["to_residual"] = {
            "path": name, "tol": args.tol5, "max_iters": args.max_iters5,
            "continuation": {"mu0": mu0, "nu": 0.9} if mu0 > 0 else None,
            "iters_done": rep.iters_done, "rel_residual": rep.rel_residual,
            "reached": bool(rep.rel_residual <= args.tol5), "device_status": rep.device_status,
            "seconds": round(ms / 1e3, 3), "ms_per_iter": round(ms / max(rep.iters_done, 1), 2),
            "fp64_seconds_extrapolated": round(out["fp64"]["ms_per_iter"] * rep.iters_done / 1e3, 2),
            "fp64_note": "FP64 time per iteration measured over the first iterations above, "
                         "times the iterations this path needed (extrapolated)"}
    print(json.dumps(out))


def run_svt5(args):
    """--case svt5: lt_svt (tau 0.5) of a 540x960x3xI4 tensor with the large
    completion's slice shape (first-iterate kind: P_Omega(N(0,1)) with 20% observed;
    L_3 = DCT 3, L_4 = Q1 diag(d) Q2^T, cond 10), I4 = --i4 (40 by default: 120 slices,
    whose per-CTA working matrices, 1.17 MB each in FP32, exceed L2).  The slices do not
    fit shared memory: the Jacobi kernel keeps them in per-CTA workspace regions."""
    import torch
    from paper_2202_02870_gb300 import lt, synth
    prec = {"fp64": lt.LT_FP64, "fp32": lt.LT_FP32, "mixed": lt.LT_MIXED}[args.precision]
    dt = torch.float64 if prec == lt.LT_FP64 else torch.float32
    rng = synth.rng_for(5, 1)
    M4 = synth.conditioned_matrix(rng, args.i4, 10.0, two_sided=True)
    ctx = lt.Context([3, args.i4], [lt.lt_make_dct(3), M4], prec)
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev)
    g.manual_seed(20220705)
    shape = (args.i4, 3, 960, 540)
    G = torch.randn(shape, generator=g, device=dev, dtype=torch.float32)
    G = (G * (torch.rand(shape, generator=g, device=dev) < 0.2)).to(dt)
    D = torch.empty_like(G)
    wsb = torch.empty(lt.lt_workspace_size(ctx, lt.LT_OP_SVT, 540, 960), dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        lt.lt_svt(ctx, G, 0.5, D, ws=wsb)
    torch.cuda.synchronize()
    lt.lt_ctx_get_stats(ctx, reset=True)
    lt.lt_ctx_set_option(ctx, lt.LT_OPT_PROFILE, 1)
    for _ in range(args.steps):
        lt.lt_svt(ctx, G, 0.5, D, ws=wsb)
    st = lt.lt_ctx_get_stats(ctx, reset=True)
    j = st["jacobi"]
    jms = j["ms"] / max(j["launches"], 1)
    print(json.dumps({"case": "svt5", "precision": args.precision, "slices": 3 * args.i4,
                      "jacobi_ms_per_launch": round(jms, 3),
                      "slices_per_s": round(3 * args.i4 / (jms / 1e3), 2),
                      "jacobi_gflops_executed": round(j["flops"] / max(j["ms"], 1e-9) / 1e6, 1),
                      "algorithmic_bytes_per_launch": j["bytes"] / max(j["launches"], 1),
                      "phase_ms_per_slice": {k: round(v / (3 * args.i4 * args.steps) / 1.97e6, 3)
                                             for k, v in st["jacobi_phase_cycles"].items()}}))


def run_warmstart(args):
    """--case warmstart: what a warm start of the SVT's Jacobi iteration would save in the
    benchmark completion (Algorithm 5 on the 144x176x3x32 problem).  For iteration k,
    G^k = Y^k - step P_Omega(Y^k - M) is formed from the checkpoint of the run after k - 1
    iterations, and V^{k-1}, the right singular vectors of G^{k-1}, from lt_svd.  The
    slices are 144 x 176, so the SVT kernel orthogonalises the columns of the transposed
    slices, and the start a warm-started Jacobi would get is the left-rotated tensor
    C^k = U^{k-1,T} *_L G^k (lt_product), U^{k-1} the left singular vectors of G^{k-1}
    (lt_svd): transform-domain slices U_hat^{k-1,p,T} G_hat^{k,p}, the same singular
    values as G^k, with the previous iteration's singular vectors already applied.  The
    Jacobi launch of lt_svt on C^k against the one on G^k (CUDA events of the library,
    median of --steps calls) measures the saving; U^{k-1} *_L D_tau(C^k) must equal
    D_tau(G^k).  `ideal` applies G^k's own left singular vectors (the best any warm
    start could do)."""
    import torch
    from paper_2202_02870_gb300 import lt
    prec = {"fp64": lt.LT_FP64, "fp32": lt.LT_FP32, "mixed": lt.LT_MIXED}[args.precision]
    dt = torch.float64 if prec == lt.LT_FP64 else torch.float32
    c = problem_inputs(0)
    dev = torch.device("cuda", 0)
    shape = (144, 176, 3, 32)
    tsh = tuple(reversed(shape))
    to_dev = lambda a, t: torch.from_numpy(np.ascontiguousarray(a.ravel(order="F"))).to(t).reshape(
        tuple(reversed(a.shape))).to(dev)
    mats = [lt.lt_make_dct(3), lt.lt_make_dct(32)]
    ctx64 = lt.Context([3, 32], mats, lt.LT_FP64)
    Xt = torch.empty(tsh, dtype=torch.float64, device=dev)
    lt.lt_product(ctx64, to_dev(c["U"], torch.float64),
                  to_dev(np.asfortranarray(np.swapaxes(c["V"], 0, 1)), torch.float64), Xt)
    mask = torch.from_numpy(np.ascontiguousarray(c["mask"].ravel(order="F"))).reshape(tsh).to(dev)
    obs = (mask.double() * (Xt + to_dev(c["noise"], torch.float64))).to(dt)
    ctx = ctx64 if prec == lt.LT_FP64 else lt.Context([3, 32], mats, prec)
    tau, step = c["tau"], c["step"]

    def g_after(j):
        """G of iteration j + 1 from the state after j iterations of a cold run."""
        X = torch.zeros(tsh, dtype=dt, device=dev)
        prev = torch.zeros_like(X)
        st = lt.lt_pga_state(X_prev=prev.data_ptr(), t_prev=1.0, t=1.0, k=0)
        if j > 0:
            lt.lt_pga_complete(ctx, mask, obs, tau, step, j, X, state=st)
        torch.cuda.synchronize()
        beta = (st.t_prev - 1.0) / st.t if j > 0 else 0.0
        Y = X + beta * (X - prev)
        return Y - step * mask.to(dt) * (Y - obs)

    def jacobi_ms(G):
        D = torch.empty_like(G)
        for _ in range(2):
            lt.lt_svt(ctx, G, tau * step, D)
        torch.cuda.synchronize()
        lt.lt_ctx_get_stats(ctx, reset=True)
        lt.lt_ctx_set_option(ctx, lt.LT_OPT_PROFILE, 1)
        per = []
        for _ in range(args.steps):
            lt.lt_svt(ctx, G, tau * step, D)
            per.append(lt.lt_ctx_get_stats(ctx, reset=True)["jacobi"]["ms"])
        lt.lt_ctx_set_option(ctx, lt.LT_OPT_PROFILE, 0)
        return statistics.median(per), D

    def left_vectors(G):
        U = torch.empty((32, 3, 144, 144), dtype=dt, device=dev)
        S = torch.empty_like(G)
        V = torch.empty((32, 3, 176, 176), dtype=dt, device=dev)
        lt.lt_svd(ctx, G, U, S, V)
        return U

    def transpose(V):  # L-transpose: swap modes 1 and 2 (real transforms)
        return V.transpose(-1, -2).contiguous()

    out = {"case": "warmstart", "precision": args.precision, "iterations": {}}
    for k in args.warm_iters:
        Gp, Gk = g_after(k - 2), g_after(k - 1)
        Up, Uk = left_vectors(Gp), left_vectors(Gk)
        UpT, UkT = transpose(Up), transpose(Uk)
        Cw = torch.empty_like(Gk)
        Ci = torch.empty_like(Gk)
        lt.lt_product(ctx, UpT, Gk, Cw)
        lt.lt_product(ctx, UkT, Gk, Ci)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            lt.lt_product(ctx, UpT, Gk, Cw)
        e1.record()
        torch.cuda.synchronize()
        prod_ms = e0.elapsed_time(e1) / args.steps
        cold, Dc = jacobi_ms(Gk)
        warm, Dw = jacobi_ms(Cw)
        ideal, _ = jacobi_ms(Ci)
        back = torch.empty_like(Dw)
        lt.lt_product(ctx, Up, Dw, back)
        torch.cuda.synchronize()
        out["iterations"][k] = {
            "jacobi_ms_cold": round(cold, 3), "jacobi_ms_warm": round(warm, 3),
            "jacobi_ms_ideal": round(ideal, 3), "warm_over_cold": round(warm / cold, 3),
            "rotation_product_ms": round(prod_ms, 3),
            "svt_agreement": float(torch.linalg.norm(back - Dc) / torch.linalg.norm(Dc))}
    print(json.dumps(out))


def run_reference(args):
    """The FP64 oracle as it stands, on the host cores: each step is a bounded sample of
    the same workload (ORACLE_ITERS_PER_STEP PGA iterations)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import lt_oracle as O
    c = problem_inputs(0)
    Ms = [O.dct_matrix(3), O.dct_matrix(32)]
    X = O.product(c["U"], O.transpose(c["V"], Ms), Ms)
    obs = c["mask"] * (X + c["noise"])
    k = ORACLE_ITERS_PER_STEP
    for _ in range(args.warmup):
        O.pga(c["mask"], obs, c["tau"], c["step"], k, Ms)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.pga(c["mask"], obs, c["tau"], c["step"], k, Ms)
    dt = time.perf_counter() - t0
    value = args.steps * k / dt
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "iters/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "shape": [144, 176, 3, 32], "iters_per_step": k},
            "cpu_baseline": {"value": round(value, 4), "unit": "iters/s", "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"{k} PGA iterations per step of the 144x176x3x32 problem"},
            "e2e": {"value": round(value, 4), "unit": "iters/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--warm", type=int, default=8,
                    help="LT_OPT_WARM_START period of the FP64 completion context (0: off)")
    ap.add_argument("--warm32", type=int, default=4,
                    help="LT_OPT_WARM_START period of the FP32 / LT_MIXED completion contexts")
    ap.add_argument("--cpu-iters", type=int, default=15)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--batched-steps", type=int, default=2,
                    help="timed calls of the 64-problem batch (0 skips the batched leg)")
    ap.add_argument("--batched-iters", type=int, default=4,
                    help="PGA iterations per call of the 64-problem batch")
    ap.add_argument("--batched-iters-fp64", type=int, default=2,
                    help="PGA iterations of the FP64 call of the 64-problem batch")
    ap.add_argument("--fourier-steps", type=int, default=2,
                    help="timed steps of the Fourier-operator (TNN-PGA-F) leg; 0 skips it")
    ap.add_argument("--fourier-iters", type=int, default=10,
                    help="PGA iterations per step of the Fourier leg")
    ap.add_argument("--svt-steps", type=int, default=3,
                    help="timed calls per precision of the L-SVT legs (0 skips them)")
    ap.add_argument("--product-steps", type=int, default=5,
                    help="timed calls of the fifth-order product leg (0 skips it)")
    ap.add_argument("--warm-iters", type=int, nargs="+", default=[3, 10, 30, 60, 99],
                    help="--case warmstart: PGA iterations k at which G^k is measured")
    ap.add_argument("--i4", type=int, default=40,
                    help="mode-4 size of --case svt5 (slices = 3 * i4)")
    ap.add_argument("--iters5", type=int, default=3,
                    help="PGA iterations per path of --case pga5")
    ap.add_argument("--tol5", type=float, default=0.0,
                    help="--case pga5: also run --precision (fp32 or mixed) from a cold "
                         "start until the relative residual is <= this value")
    ap.add_argument("--mu0-frac", type=float, default=0.0,
                    help="--case pga5 --tol5: continuation with mu_0 = this x ||M||_F, nu = 0.9")
    ap.add_argument("--max-iters5", type=int, default=300,
                    help="--case pga5: iteration cap of the --tol5 run")
    ap.add_argument("--case", default="pga",
                    choices=["pga", "svt", "product", "product5", "transform5", "pga5",
                             "svt5", "warmstart"],
                    help="pga: the benchmark line; svt/product: single-operation runs "
                         "used for profiling")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "mixed"])
    ap.add_argument("--tc-tile-n", type=int, default=0, choices=[0, 32, 64, 128, 256],
                    help="LT_MIXED tensor-core tile width (0: the library's choice)")
    ap.add_argument("--jacobi-pairwise", type=int, default=0, choices=[0, 1, 2, 3],
                    help="1: rotate column pairs straight through shared memory (no "
                         "register blocks)")
    ap.add_argument("--jacobi-cluster", type=int, default=0, choices=[0, 1, 3, 4],
                    help="--case svt: SVT kernel form (LT_OPT_JACOBI_CLUSTER)")
    ap.add_argument("--jacobi-group", type=int, default=0, choices=[0, 8, 16, 32],
                    help="lanes per Jacobi column pair (0: the planner's choice)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    from paper_2202_02870_gb300 import build
    build.build()
    if args.case == "product5":
        run_product5(args)
        return
    if args.case == "transform5":
        run_transform5(args)
        return
    if args.case == "pga5":
        run_pga5(args)
        return
    if args.case == "svt5":
        run_svt5(args)
        return
    if args.case == "warmstart":
        run_warmstart(args)
        return
    if args.case != "pga":
        run_case(args)
        return
    run_ours(args)


if __name__ == "__main__":
    main()
