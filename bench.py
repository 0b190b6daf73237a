"""Benchmark: recursive FP32 TRSM + TRMM at m = n = 16384 on one GB300.

One step = TRSM (side L, lower, no transpose, non-unit, alpha = 1.5) followed
by TRMM with the same factor and alpha = 1/1.5 on the same right-hand side,
so B returns to itself (up to rounding) and the run can repeat without
re-staging. A step walks the whole hot path: the factor's operand planes
(made once per step from A and shared by both calls), leaf kernels,
tensor-core GEMM updates. Metric: TFLOP/s with the m^2 n convention per call
(2 * 16384^3 flop per step).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 launch under torch.distributed.run; every rank runs its own copy
of the workload (weak scaling), or with --shard its panel of the one
problem's right-hand sides (strong scaling: right-hand sides of TRSM/TRMM
are independent, so the work shards with no exchange); rank 0 prints one
JSON line.

--impl reference times the FP64 CPU oracle (plain substitution / triple
loop, OpenMP) on a bounded sample of the same workload's right-hand sides.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "TRSM/TRMM TFLOP/s (m^2n, % of peak) at n=16384; served solves/s, p50/p99 ms"
K_ORDER = 16384
NRHS = 16384
ALPHA = 1.5
SEED = 16384
CPU_SAMPLE_COLS = 32      # cpu_baseline sample (right-hand sides)
SPLIT_TERMS = 6           # tensor-core split in use (read back from the handle)
SWEEP_SIZES = "256,512,1024,2048,4096,8192,16384"
SPLIT_DESC = {6: "3 BF16 slices per operand, every slice product above 2^-24: FP32-grade",
              3: "2 BF16 slices per operand, about 2^-16 relative per product",
              1: "1 BF16 slice, about 2^-8 relative per product"}
REF_SAMPLE_COLS = 16      # per step of --impl reference


# DRAM traffic of gemm_tc_kernel per launch on this workload (m = n = 16384,
# 6-term split): dram__bytes_read.sum + dram__bytes_write.sum summed over the
# 132 GEMM launches of one step and divided by 132. The two counters take one
# ncu pass (checked on a small case first), so the capture is the full-size
# launch list with two metrics (its command and figures are kept with the
# ncu summaries). To be set back to None (null in the line) whenever
# gemm_tc.cu or this workload's plan changes, until captured again.
TRAFFIC_PER_LAUNCH = 316.27e6
# FP64 FMA rate measured by this build's own probe (bench.py --workload
# peaks; MEASURED_PEAKS.json holds no FP64 figure): the FP64 roofline
FP64_FMA_PROBE_TFLOPS = 1.057


def captured_traffic():
    # the capture is of the default workload (m = n = 16384, 6-term split,
    # automatic leaves); any other configuration reports null
    if (K_ORDER, NRHS, SPLIT_TERMS) != (16384, 16384, 6) or LEAF_USED is not None:
        return None
    return TRAFFIC_PER_LAUNCH


def triangle_upload_bytes(k, elem):
    """Bytes trx_copy_triangle_h2d moves for a lower k x k triangle: one
    rectangle of rows j0..k-1 per block of 256 columns."""
    return sum((k - j0) * (min(k, j0 + 256) - j0) for j0 in range(0, k, 256)) * elem


def flops_per_call(k, nrhs):
    return float(k) * k * nrhs


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0,
                "bf16_tflops_sustained": 1700.0}, "fallback"


# ---- clocks ---------------------------------------------------------------
class ClockSampler:
    """nvidia-smi sampling during the timed region (every 200 ms)."""
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and parts[0] != self.uuid:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "power_w_max": max(power), "samples": len(sm), "reasons": sorted(reasons)}


# ---- distributed helpers ----------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, world: int) -> float:
    """Max of a per-rank float over all ranks (identity for one rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) \
        if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---- CPU oracle timing --------------------------------------------------------
def oracle_sample(A, B, cols):
    """One TRSM + TRMM of the workload on `cols` right-hand sides (FP64
    oracle). Returns (seconds, flops)."""
    import oracle
    Bs = np.asfortranarray(B[:, :cols])
    t0 = time.perf_counter()
    X = oracle.trsm("L", "L", "N", "N", ALPHA, A, Bs)
    oracle.trmm("L", "L", "N", "N", 1.0 / ALPHA, A, X)
    dt = time.perf_counter() - t0
    return dt, 2.0 * flops_per_call(A.shape[0], cols)


DTYPE = np.float32


def host_inputs():
    from paper_2504_13821_gb300 import inputs
    return inputs.problem("L", "L", K_ORDER, NRHS, seed=SEED, dtype=DTYPE)


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    A, B = host_inputs()
    for _ in range(args.warmup):
        oracle_sample(A, B, REF_SAMPLE_COLS)
    total, flops = 0.0, 0.0
    for _ in range(args.steps):
        dt, fl = oracle_sample(A, B, REF_SAMPLE_COLS)
        total += dt
        flops += fl
    value = flops / total / 1e12
    cores = oracle.nthreads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(),
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": f"per step: TRSM + TRMM of the {K_ORDER}x{K_ORDER} factor "
                                   f"on {REF_SAMPLE_COLS} of the {NRHS} right-hand sides"},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# automatic cutoffs of the library for this workload (FP32, 16384 right-hand
# sides): TRSM 128-row leaves (wide leaf kernel), TRMM 1024-row diagonal blocks
# on the tensor cores; --leaf overrides both
# (FP64: 64-row leaves)
LEAF_USED = None


def auto_path_desc(k, n):
    """What the library's automatic choices (plan.cuh: use_thin_mode,
    thin_leaf_rows, the leaf kernel by right-hand-side count) run for FP32
    side-L TRSM and TRMM of order k with n right-hand sides."""
    thin_leaf = 0
    if k >= 4096 and 64 < n <= 1024 and not (n <= 128 and k < 8192):
        thin_leaf = 2048 if n <= 256 else 1024
    if thin_leaf and k > thin_leaf:
        trsm = f"TRSM leaves of {thin_leaf} rows as thin solves (64-row blocks, 16-column panels)"
    elif k > 256 and (n <= 64 or (n <= 256 and k * n <= 1 << 21)):
        trsm = "TRSM as one thin solve (64-row blocks, 16-column panels, one launch)"
    else:
        trsm = f"TRSM 128 ({'wide leaf' if n >= 1024 else 'lane-split leaf'})"
    if k > 256 and n <= 32:
        trmm = "TRMM as one thin product"
    else:
        trmm = "TRMM 1024-row diagonal blocks on the tensor cores" if k >= 1024 else "TRMM 64"
    return f"{trsm}, {trmm}"


def workload_config():
    prec = "FP32" if DTYPE == np.float32 else "FP64"
    return {"workload": f"{prec} TRSM(alpha=1.5) then TRMM(alpha=1/1.5), side L, lower, "
                        f"no transpose, non-unit, m={K_ORDER} n={NRHS}, column-major"
                        + ("; one prepared factor, its operand planes made once per step"
                           if DTYPE == np.float32 else ""),
            "m": K_ORDER, "n": NRHS,
            "leaf": LEAF_USED if LEAF_USED is not None else (
                auto_path_desc(K_ORDER, NRHS) if DTYPE == np.float32 else 64),
            "gemm": (f"tcgen05 kind::f16, {SPLIT_TERMS}-term split BF16 "
                     f"({SPLIT_DESC[SPLIT_TERMS]}), FP32 accumulation"
                     if DTYPE == np.float32 else "CUDA-core DFMA"),
            "graph": "cached CUDA graph per call",
            "l2": "inputs larger than L2 (A 1 GiB, B 1 GiB); no flush"}


# ---- GPU arm ----------------------------------------------------------------------
def run_gpu(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    import paper_2504_13821_gb300 as trx
    from paper_2504_13821_gb300 import _binding

    A_np, B_np = host_inputs()
    k, n = K_ORDER, NRHS
    if args.shard:
        # strong scaling: this rank's panel of the one problem's right-hand
        # sides (independent columns, no exchange); the whole job's work is
        # fixed as the rank count grows
        from paper_2504_13821_gb300.sharding import panel
        j0, j1 = panel(NRHS, world, rank)
        B_np = np.asfortranarray(B_np[:, j0:j1])
        n = j1 - j0
    colmajor = trx.to_colmajor
    A = colmajor(torch.from_numpy(A_np).to(dev))
    B = colmajor(torch.from_numpy(B_np).to(dev))
    h = trx.Handle(dev)
    if args.split:
        h.set_option(trx.OPT_SPLIT, args.split)
    if args.dag:
        h.set_option(trx.OPT_TRSM_DAG, args.dag)
    global SPLIT_TERMS
    SPLIT_TERMS = h.get_option(trx.OPT_SPLIT)
    if args.pdl:
        h.set_option(trx.OPT_PDL, 1)
    if args.panels:
        h.set_option(trx.OPT_PANELS, args.panels)
    if args.leaf:
        h.set_option(trx.OPT_LEAF, args.leaf)
        global LEAF_USED
        LEAF_USED = args.leaf
    if args.tc_leaf:
        h.set_option(trx.OPT_TRSM_TC_LEAF, 1)
        LEAF_USED = (f"TRSM {args.leaf or 128} as inverse GEMMs on the tensor cores, "
                     "TRMM 1024-row diagonal blocks on the tensor cores")
    stream = torch.cuda.current_stream(dev)
    # FP32: the factor's operand planes are made once per step (update), then
    # the TRSM and the TRMM both use them. FP64 has no planes: plain calls.
    f32 = DTYPE == np.float32
    factor = trx.Factor("L", "L", "N", "N", A, handle=h, stream=stream) if f32 else None

    def step(Bt):
        if f32:
            factor.update(stream=stream)
            factor.trsm(ALPHA, Bt, stream=stream)
            factor.trmm(1.0 / ALPHA, Bt, stream=stream)
        else:
            trx.trsm("L", "L", "N", "N", ALPHA, A, Bt, handle=h, stream=stream)
            trx.trmm("L", "L", "N", "N", 1.0 / ALPHA, A, Bt, handle=h, stream=stream)

    for _ in range(max(args.warmup, 0)):
        step(B)
    torch.cuda.synchronize()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step(B)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(world)
    ms_total = max_over_ranks(ev0.elapsed_time(ev1), world)
    ms_step = ms_total / args.steps
    flops_step = 2.0 * flops_per_call(k, n)
    # whole job: every rank's copy (weak scaling) or the one sharded problem
    job_flops_step = 2.0 * flops_per_call(k, NRHS) if args.shard else world * flops_step
    value = job_flops_step * args.steps / (ms_total * 1e-3) / 1e12

    # Per-kernel durations: one instrumented step (direct launches with a
    # CUDA event pair around every launch on the call's stream).
    h.set_option(trx.OPT_PROFILE, 1)
    h.profile(reset=True)
    step(B)
    prof = h.profile(reset=True)
    h.set_option(trx.OPT_PROFILE, 0)
    launches_step = sum(v["launches"] for v in prof.values())
    peaks, src = load_peaks()
    if DTYPE == np.float32:
        g = prof["gemm_tc"]
        kname = "gemm_tc_kernel (GEMM update, tcgen05)"
        peak_tc = peaks["bf16_tflops_sustained"] / SPLIT_TERMS
        peak_src = (f"{src} bf16 sustained {peaks['bf16_tflops_sustained']} TFLOP/s / "
                    f"{SPLIT_TERMS} split-product terms")
    else:
        g = prof["gemm_simt"]
        kname = "gemm_simt_kernel<double> (GEMM update, DFMA)"
        peak_tc = FP64_FMA_PROBE_TFLOPS
        peak_src = (f"this build's FP64 FMA probe (bench.py --workload peaks): "
                    f"{FP64_FMA_PROBE_TFLOPS} TFLOP/s")
    achieved = g["flops"] / (g["ms"] * 1e-3) / 1e12 if g["ms"] > 0 else 0.0
    kern_ms = sum(v["ms"] for v in prof.values())
    roofline = {
        "bound": "tensor" if DTYPE == np.float32 else "fp64",
        "kernel": kname,
        "achieved": achieved, "peak": peak_tc, "unit": "TFLOP/s",
        "frac": achieved / peak_tc if peak_tc else None,
        "traffic": captured_traffic() if DTYPE == np.float32 else None,
        "algorithmic_bytes_per_launch": g["bytes"] / g["launches"] if g["launches"] else None,
        "peak_source": peak_src,
        # the same kernel against the raw BF16 tensor peak: every algorithmic
        # flop is SPLIT_TERMS BF16 products on the pipe
        "tensor_pipe_tflops": SPLIT_TERMS * achieved if DTYPE == np.float32 else None,
        "frac_of_raw_bf16_burst": (SPLIT_TERMS * achieved / peaks["bf16_tflops"]
                                   if DTYPE == np.float32 else None),
        "launches_per_step": g["launches"],
        "share_of_kernel_time": g["ms"] / kern_ms if kern_ms else None,
        "per_class_ms": {kk: round(v["ms"], 4) for kk, v in prof.items() if v["launches"]},
        "whole_step_frac": (flops_step / (ms_step * 1e-3) / 1e12) / peak_tc,
    }
    # the leaves (the recursion's HBM/latency-bound part): their algorithmic
    # bytes (right-hand-side rows in and out, the triangle, the planes they
    # write) over their event-timed duration, against the HBM copy rate
    lf = prof.get("leaf_trsm", {"ms": 0, "bytes": 0, "launches": 0})
    leaf_roofline = None
    if lf["launches"] and lf["ms"] > 0:
        leaf_gbs = lf["bytes"] / (lf["ms"] * 1e-3) / 1e9
        leaf_roofline = {"bound": "hbm", "kernel": "TRSM leaves", "achieved": leaf_gbs,
                         "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": leaf_gbs / peaks["hbm_gbs"], "launches_per_step": lf["launches"],
                         "us_per_launch": 1e3 * lf["ms"] / lf["launches"]}

    # End to end through the public API: pinned host buffers, every step the
    # H2D copy of A's lower triangle (trx_copy_triangle_h2d: the part the
    # calls read) and of B, TRSM + TRMM, and the D2H copy of the result.
    # Pipelined over steps the way a stream of independent jobs would run:
    # two device slots, uploads on one copy stream, compute on the call's
    # stream, downloads on another copy stream, so step i+1's upload and step
    # i-1's download overlap step i's compute (the first upload and the last
    # download are in the timed region, unoverlapped). The same steps run
    # serially on one stream as well ("serial").
    e2e = None
    if not args.no_e2e:
        A_h = torch.from_numpy(A_np).pin_memory()
        B_h = torch.from_numpy(B_np).pin_memory()
        out_h = [torch.empty_like(B_h).pin_memory() for _ in range(2)]
        Ad = [torch.empty_like(A) for _ in range(2)]
        Bd = [torch.empty_like(B) for _ in range(2)]
        fac = [trx.Factor("L", "L", "N", "N", Ad[i], handle=h, stream=stream) if f32 else None
               for i in range(2)]

        def solve_slot(sl):
            if f32:
                fac[sl].update(stream=stream)
                fac[sl].trsm(ALPHA, Bd[sl], stream=stream)
                fac[sl].trmm(1.0 / ALPHA, Bd[sl], stream=stream)
            else:
                trx.trsm("L", "L", "N", "N", ALPHA, Ad[sl], Bd[sl], handle=h, stream=stream)
                trx.trmm("L", "L", "N", "N", 1.0 / ALPHA, Ad[sl], Bd[sl], handle=h, stream=stream)
        up, up_b, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        ev_up = [torch.cuda.Event() for _ in range(2)]
        ev_up_b = [torch.cuda.Event() for _ in range(2)]
        ev_done = [torch.cuda.Event() for _ in range(2)]
        ev_down = [torch.cuda.Event() for _ in range(2)]
        for i in range(2):
            ev_down[i].record(down)

        def e2e_step(i):
            sl = i % 2
            # A's triangle and B go up on two streams
            up.wait_event(ev_down[sl])                 # slot's last result read back
            up_b.wait_event(ev_down[sl])
            trx.copy_triangle_h2d("L", A_h, Ad[sl], stream=up)   # the triangle the calls read
            with torch.cuda.stream(up_b):
                Bd[sl].copy_(B_h, non_blocking=True)
            ev_up[sl].record(up)
            ev_up_b[sl].record(up_b)
            stream.wait_event(ev_up[sl])
            stream.wait_event(ev_up_b[sl])
            solve_slot(sl)
            ev_done[sl].record(stream)
            down.wait_event(ev_done[sl])
            with torch.cuda.stream(down):
                out_h[sl].copy_(Bd[sl], non_blocking=True)
            ev_down[sl].record(down)

        def e2e_serial_step():
            trx.copy_triangle_h2d("L", A_h, Ad[0], stream=stream)
            Bd[0].copy_(B_h, non_blocking=True)
            solve_slot(0)
            out_h[0].copy_(Bd[0], non_blocking=True)

        for i in range(2):
            e2e_step(i)
        e2e_serial_step()
        torch.cuda.synchronize()
        nbytes = B_h.numel() * B_h.element_size()
        a_bytes = triangle_upload_bytes(K_ORDER, A_h.element_size())
        e_steps = max(2, args.steps)
        barrier(world)
        t0 = time.perf_counter()
        for i in range(e_steps):
            e2e_step(i)
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, world)
        s_steps = max(1, min(args.steps, 3))
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(s_steps):
            e2e_serial_step()
        torch.cuda.synchronize()
        dts = max_over_ranks(time.perf_counter() - t0, world)
        ok = bool(torch.equal(out_h[0], out_h[1]))    # both slots returned the same result
        e2e = {"value": job_flops_step * e_steps / dt / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": a_bytes + nbytes, "d2h_bytes_per_step": nbytes,
               "ms_per_step": 1e3 * dt / e_steps, "steps": e_steps,
               "pipelined": "upload of step i+1 (A's lower triangle and B, two copy streams) "
                            "and download of step i-1 overlap step i",
               "slots_agree": ok,
               "serial": {"value": job_flops_step * s_steps / dts / 1e12,
                          "ms_per_step": 1e3 * dts / s_steps, "steps": s_steps}}
        for fc in fac:
            if fc is not None:
                fc.close()
        del Ad, Bd

    # Correctness of the timed data: after the round trips B is back to the
    # original up to rounding (TRMM undoes TRSM).
    drift = float((B.cpu() - torch.from_numpy(B_np)).abs().max() /
                  torch.from_numpy(B_np).abs().max())

    cpu = None
    if rank == 0 and not args.no_cpu:
        import oracle
        oracle.build()
        dt, fl = oracle_sample(A_np, B_np, CPU_SAMPLE_COLS)
        cpu = {"value": fl / dt / 1e12, "unit": "TFLOP/s", "cores": oracle.nthreads(),
               "kind": "oracle",
               "sample": f"TRSM + TRMM of the {K_ORDER}x{K_ORDER} factor on {CPU_SAMPLE_COLS} "
                         f"of the {NRHS} right-hand sides ({dt:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "strong" if args.shard else "weak",
            "vs_baseline": None,
            "dtype": "f32" if DTYPE == np.float32 else "f64", "data": "synthetic",
            "config": dict(workload_config(), parallelism=(
                f"right-hand-side panels over {world} ranks (one problem, no exchange)"
                if args.shard else f"{world} independent copies, one per rank")),
            "clocks": clk, "gpu_launches": launches_step * args.steps,
            "roofline": roofline, "leaf_roofline": leaf_roofline, "cpu_baseline": cpu,
            "e2e": e2e,
            "round_trip_drift": drift,
        }
        print(json.dumps(line), flush=True)
    if factor is not None:
        factor.close()
    h.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """Batched uneven workload: 4096 independent TRSM/TRMM problems, order
    log-uniform 16..512, 1..64 right-hand sides, random side and uplo, one
    persistent launch (cached graph), against a loop of single calls."""
    import torch
    import paper_2504_13821_gb300 as trx
    from paper_2504_13821_gb300 import inputs
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(4096)
    probs, flops, nbytes, fmas = [], 0.0, 0.0, 0.0
    w = np.dtype(DTYPE).itemsize
    for i in range(args.count):
        k = int(round(np.exp(rng.uniform(np.log(16), np.log(512)))))
        nrhs = int(rng.integers(1, 65))
        side, uplo = str(rng.choice(["L", "R"])), str(rng.choice(["L", "U"]))
        op = "S" if i % 2 == 0 else "M"
        m, n = (k, nrhs) if side == "L" else (nrhs, k)
        A, B = inputs.problem(side, uplo, m, n, seed=4096 * 1000 + i, dtype=DTYPE)
        At = trx.to_colmajor(torch.from_numpy(A).to(dev))
        Bt = trx.to_colmajor(torch.from_numpy(B).to(dev))
        probs.append((op, side, uplo, "N", "N", 1.5 if op == "S" else 1 / 1.5, At, Bt))
        flops += float(k) * k * nrhs
        # algorithmic work per problem: the referenced triangle read once, B
        # read and written once; k (k + 1) / 2 multiply-adds per right-hand side
        nbytes += w * (k * (k + 1) / 2.0 + 2.0 * k * nrhs)
        fmas += k * (k + 1) / 2.0 * nrhs
    h = trx.Handle(dev)
    table = None
    if not args.no_autotune:
        scratch = [(o, s_, u, t, d, a, A, B.clone()) for (o, s_, u, t, d, a, A, B) in probs]
        table = trx.batched_autotune(scratch, handle=h)
        del scratch
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps):
        for _ in range(max(args.warmup, 1)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    batch = trx.Batch(probs, handle=h)   # prepared once: descriptors kept on the device
    ms_batched = timed(lambda: batch.run(handle=h, stream=stream), args.steps)

    def loop():
        for (o, s_, u, t, d, a, A, B) in probs:
            (trx.trsm if o == "S" else trx.trmm)(s_, u, t, d, a, A, B, handle=h, stream=stream)
    ms_loop = None if args.no_loop else timed(loop, max(1, min(args.steps, 2)))
    # the kernel's two ceilings: HBM (measured copy peak) and the CUDA-core
    # FMA pipe of its element type (the library's own probe, measured here)
    peaks, src = load_peaks()
    kind = "ffma" if DTYPE == np.float32 else "dfma"
    probe_iters = 52905 if kind == "ffma" else 721
    fma_peak = max(trx.peak_probe(kind, probe_iters)[0] for _ in range(3))
    gbs = nbytes / (ms_batched * 1e-3) / 1e9
    tfl = 2.0 * fmas / (ms_batched * 1e-3) / 1e12
    hbm_frac, fma_frac = gbs / peaks["hbm_gbs"], tfl / fma_peak
    roofline = {"bound": "hbm" if hbm_frac >= fma_frac else "alu",
                "kernel": "batched_kernel (one persistent launch)",
                "achieved": gbs if hbm_frac >= fma_frac else tfl,
                "peak": peaks["hbm_gbs"] if hbm_frac >= fma_frac else fma_peak,
                "unit": "GB/s" if hbm_frac >= fma_frac else "TFLOP/s",
                "frac": max(hbm_frac, fma_frac), "traffic": None,
                "hbm": {"achieved_gbs": gbs, "peak_gbs": peaks["hbm_gbs"], "frac": hbm_frac,
                        "algorithmic_bytes": nbytes, "peak_source": src},
                "fma": {"achieved_tflops": tfl, "peak_tflops": fma_peak, "frac": fma_frac,
                        "peak_source": f"trx_peak_probe {kind}, measured in this run"}}
    line = {
        "metric": "batched uneven TRSM/TRMM problems/s", "value": args.count / (ms_batched * 1e-3),
        "unit": "problems/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_batched, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if DTYPE == np.float32 else "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.count} problems, order log-uniform 16..512, 1..64 "
                               "right-hand sides, random side/uplo, TRSM/TRMM alternating",
                   "tflops_m2n": flops / (ms_batched * 1e-3) / 1e12,
                   "autotune": table},
        "loop_of_single_calls": None if ms_loop is None else {
            "ms": ms_loop, "problems_per_s": args.count / (ms_loop * 1e-3)},
        "speedup_vs_loop": None if ms_loop is None else ms_loop / ms_batched,
        "roofline": roofline,
    }
    print(json.dumps(line), flush=True)
    h.close()
    return 0


def run_refined(args):
    """Refined FP32 TRSM (the precision form): the FP32 solve refined in FP64
    until the normwise backward error is at the FP64 level, side L, lower,
    on factors whose condition number is about 1e2, 1e4 and 1e6 (scales of
    the seeded generator stored in tests/golden/condition_scales.json),
    against the plain FP32 solve and the FP64 solve of the same data."""
    import torch
    import paper_2504_13821_gb300 as trx
    from paper_2504_13821_gb300 import inputs
    dev = torch.device("cuda", 0)
    with open(os.path.join(ROOT, "tests", "golden", "condition_scales.json")) as f:
        entries = [e for e in json.load(f)["entries"] if e["k"] == K_ORDER
                   and (args.kappa is None or e["target"] == args.kappa)]
    if not entries:
        print(json.dumps({"error": f"no stored condition scales for order {K_ORDER}"}))
        return 1
    k, n = K_ORDER, NRHS
    h = trx.Handle(dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps):
        for _ in range(max(args.warmup, 1)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    rows, total_ms = [], 0.0
    for e in entries:
        A, B = inputs.problem("L", "L", k, n, seed=e["seed"], dtype=np.float32, scale=e["scale"])
        At, Bt = trx.to_colmajor(torch.from_numpy(A).to(dev)), trx.to_colmajor(
            torch.from_numpy(B).to(dev))
        X = torch.empty((n, k), dtype=torch.float64, device=dev).t()
        info = {}

        def refined():
            info.update(trx.trsm_refined("L", "L", "N", "N", 1.5, At, Bt, out=X, handle=h)[1])
        ms_ref = timed(refined, args.steps)
        info_ff, X_ff = dict(info), X.clone()
        # the same refinement with the residual on the FP64 pipe
        h.set_option(trx.OPT_RESIDUAL, trx.RESIDUAL_FP64)
        ms_ref64 = timed(refined, max(1, min(args.steps, 3)))
        info_64 = dict(info)
        h.set_option(trx.OPT_RESIDUAL, trx.RESIDUAL_AUTO)
        X32 = Bt.clone()
        ms_32 = timed(lambda: trx.trsm("L", "L", "N", "N", 1.5, At, X32.copy_(Bt), handle=h),
                      args.steps)
        A64, B64 = At.double(), Bt.double()
        X64 = B64.clone()
        ms_64 = timed(lambda: trx.trsm("L", "L", "N", "N", 1.5, A64, X64.copy_(B64), handle=h),
                      max(1, min(args.steps, 3)))
        X32d = X32.double()

        def rel(a):
            return float((a - X64).abs().sum(dim=1).max() / X64.abs().sum(dim=1).max())
        rows.append({"kappa_target": e["target"], "kappa_estimate": e["kappa_estimate"],
                     "scale": e["scale"], "ms_refined": ms_ref, "ms_fp32": ms_32,
                     "ms_fp64": ms_64, "iterations": info_ff["iterations"],
                     "backward_error_updated_residual": info_ff["backward_error"],
                     "backward_error_fp32": info_ff["initial_backward_error"],
                     "fp64_residual": {"ms_refined": ms_ref64,
                                       "iterations": info_64["iterations"],
                                       "backward_error": info_64["backward_error"],
                                       "diff_vs_fp64_solve": rel(X)},
                     "diff_vs_fp64_solve": rel(X_ff), "diff_fp32_vs_fp64_solve": rel(X32d)})
        total_ms += ms_ref
        del At, Bt, X, X_ff, X32, A64, B64, X64, X32d
    line = {
        "metric": "refined FP32 TRSM solves/s", "value": len(rows) / (total_ms * 1e-3),
        "unit": "solves/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / len(rows), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"refined TRSM side L lower, k={k}, {n} right-hand sides, "
                               "alpha 1.5, kappa about 1e2/1e4/1e6, stop at backward error "
                               "sqrt(k) 2^-53 or when a correction stops lowering it; "
                               "float-float residual, updated by each correction "
                               "(its backward error excludes the first residual's own "
                               "rounding, about 2^-46 relative; the tests check the result's "
                               "backward error against the FP64 oracle); FP64-pipe residual "
                               "recomputed from X alongside",
                   "l2": "factor (k^2 FP32 = 256 MB at k = 8192) larger than L2, no flush"},
        "per_kappa": rows,
    }
    print(json.dumps(line), flush=True)
    h.close()
    return 0


def run_sweep(args):
    """The all-variant size sweep: TRSM and TRMM, all 16 side/uplo/trans/diag
    variants, FP32 and FP64, m = n in {256, 512, ..., 16384}, alpha = 1.5,
    the seeded generator with seed k + 1e6 * (variant index). One JSON line
    per point: device time of one call (CUDA events on the call's stream,
    B restored from a pristine copy before each call, outside the timed
    pair), TFLOP/s (m^2 n), and the errors against the FP64 oracle: for
    orders up to 4096 the whole result (TRSM backward error and forward
    error, TRMM normwise error) up to order 2048, above that a seeded sample of right-hand
    sides (columns for side L, rows for side R; each is an independent
    problem), with the oracle's time on the sample. A last line sums it up."""
    import torch
    import oracle
    import paper_2504_13821_gb300 as trx
    from paper_2504_13821_gb300 import inputs
    oracle.build()
    dev = torch.device("cuda", 0)
    h = trx.Handle(dev)
    if args.split:
        h.set_option(trx.OPT_SPLIT, args.split)
    terms = h.get_option(trx.OPT_SPLIT)
    stream = torch.cuda.current_stream(dev)
    sizes = [int(x) for x in args.sizes.split(",")]
    dtypes = args.dtypes.split(",")
    ops = args.ops.split(",")
    vsel = range(16) if args.variants == "all" else [int(x) for x in args.variants.split(",")]
    cores = oracle.nthreads()
    worst = {}
    npoints = 0
    for k in sizes:
        for vi in vsel:
            side, uplo, trans, diag = inputs.VARIANTS[vi]
            seed = inputs.variant_seed(k, vi)
            A64, B64 = inputs.problem(side, uplo, k, k, seed=seed, dtype=np.float64,
                                      poison_diag=(diag == "U"))
            full = k <= 2048
            rng = np.random.default_rng(seed + 17)
            nsamp = 16 if k >= 16384 else 32 if k >= 8192 else 64
            samp = None if full else np.sort(rng.choice(k, size=nsamp, replace=False))
            for dt in dtypes:
                npdt = np.float32 if dt == "f32" else np.float64
                A, B = A64.astype(npdt), B64.astype(npdt)
                Ad = trx.to_colmajor(torch.from_numpy(A).to(dev))
                B0 = trx.to_colmajor(torch.from_numpy(B).to(dev))
                Bd = B0.clone()
                fl = float(k) ** 3
                reps = 1 if (dt == "f64" and k >= 8192) else max(1, args.steps)
                for op in ops:
                    fn = trx.trsm if op == "trsm" else trx.trmm
                    times = []
                    for r in range(reps + 1):      # the first call warms up (graph capture)
                        Bd.copy_(B0)
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        fn(side, uplo, trans, diag, ALPHA, Ad, Bd, handle=h, stream=stream)
                        e1.record(stream)
                        torch.cuda.synchronize()
                        if r:
                            times.append(e0.elapsed_time(e1))
                    ms = statistics.median(times)
                    X = Bd.cpu().numpy().astype(np.float64)
                    A_o, B_o = A.astype(np.float64), B.astype(np.float64)
                    if samp is not None:
                        if side == "L":
                            X, B_o = X[:, samp], B_o[:, samp]
                        else:
                            X, B_o = X[samp, :], B_o[samp, :]
                        X, B_o = np.asfortranarray(X), np.asfortranarray(B_o)
                    t0 = time.perf_counter()
                    ref = (oracle.trsm if op == "trsm" else oracle.trmm)(
                        side, uplo, trans, diag, ALPHA, A_o, B_o)
                    t_or = time.perf_counter() - t0
                    fwd = oracle.forward_error(X, ref)
                    if op == "trsm":
                        err = oracle.trsm_backward_error(side, uplo, trans, diag, ALPHA, A_o, X,
                                                         B_o)["eta"]
                    else:
                        err = oracle.trmm_error(side, uplo, trans, diag, ALPHA, A_o, X, ref, B_o)
                    u = 2.0 ** -24 if dt == "f32" else 2.0 ** -53
                    bound = 8 * k * u
                    ok = bool(np.isfinite(err) and err <= bound)
                    nrhs_or = k if samp is None else len(samp)
                    line = {"workload": "sweep", "op": op, "dtype": dt,
                            "variant": side + uplo + trans + diag, "m": k, "n": k,
                            "ms": ms, "tflops": fl / (ms * 1e-3) / 1e12,
                            "error_metric": "backward" if op == "trsm" else "normwise",
                            "error": err, "bound": bound, "ok": ok, "forward_error": fwd,
                            "checked": "all" if samp is None else f"{len(samp)} sampled "
                                       + ("columns" if side == "L" else "rows"),
                            "oracle_s": t_or, "oracle_gflops": float(k) * k * nrhs_or / t_or / 1e9,
                            "oracle_cores": cores, "reps": reps,
                            "split_terms": terms if dt == "f32" else None}
                    print(json.dumps(line), flush=True)
                    npoints += 1
                    key = (op, dt)
                    w = worst.setdefault(key, {"max_err_over_bound": 0.0, "fails": 0})
                    w["max_err_over_bound"] = max(w["max_err_over_bound"], err / bound)
                    w["fails"] += 0 if ok else 1
                del Ad, B0, Bd
    print(json.dumps({"workload": "sweep", "summary": True, "points": npoints,
                      "per_op_dtype": {f"{a}/{b}": v for (a, b), v in worst.items()}}),
          flush=True)
    h.close()
    return 0


def run_precision(args):
    """The precision form against plain FP32 (config 3): FP32 TRSM side L,
    lower, no transpose, non-unit, alpha 1.5, m in {8192, 16384, 32768}, n in
    {256, m}, factors with kappa_1 about 1e2, 1e4, 1e6 (the stored scales of
    tests/golden/condition_scales.json). Per point and form: device time
    (CUDA events, median), and against the FP64 oracle on a seeded sample of
    16 right-hand sides (each column of a side-L solve is its own problem):
    the normwise backward error of the sample and its forward error. Forms:
      split6        the plain FP32 solve (6-term split: FP32-grade products)
      split3, split1 the same recursion with 3-term / 1-term BF16 products
      refine3_1e-6, refine1_1e-6  split-3 / split-1 solve + refinement with
                    the FP32-grade tensor-core residual, stopping at backward
                    error 1e-6 (the library's own estimate)
      refine6_fp64  split-6 solve + float-float residual refinement to an
                    FP64-level backward error
      fp64          the library's FP64 solve (CUDA-core DFMA), n = 256 and
                    m <= 8192 with n = m only (seconds per call beyond)
    One JSON line per point, then a summary line."""
    import torch
    import oracle
    import paper_2504_13821_gb300 as trx
    from paper_2504_13821_gb300 import inputs
    oracle.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    with open(os.path.join(ROOT, "tests", "golden", "condition_scales.json")) as f:
        entries = json.load(f)["entries"]
    sizes = [int(x) for x in args.sizes.split(",")]
    kappas = [1e2, 1e4, 1e6] if args.kappa is None else [args.kappa]
    nsel = args.nrhs_list.split(",")
    h = trx.Handle(dev)
    # the forms compare the recursion's update arithmetic: the thin CUDA-core
    # solve (no split), whole-call or as the leaves, is kept out of the table
    h.set_option(trx.OPT_THIN, -1)
    h.set_option(trx.OPT_THIN_LEAF, -1)
    alpha = 1.5

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    summary = []
    for k in sizes:
        for kap in kappas:
            e = next((x for x in entries if x["k"] == k and x["target"] == kap), None)
            if e is None:
                print(json.dumps({"workload": "precision", "k": k, "kappa": kap,
                                  "error": "no stored scale"}), flush=True)
                continue
            for ns in nsel:
                n = k if ns == "m" else int(ns)
                A, B = inputs.problem("L", "L", k, n, seed=e["seed"], dtype=np.float32,
                                      scale=e["scale"])
                cols = np.sort(np.random.default_rng(e["seed"] + n).choice(
                    n, size=min(16, n), replace=False))
                A64 = A.astype(np.float64)
                Bs = np.asfortranarray(B[:, cols].astype(np.float64))
                t0 = time.perf_counter()
                ref = oracle.trsm("L", "L", "N", "N", alpha, A64, Bs)
                t_or = time.perf_counter() - t0
                At = trx.to_colmajor(torch.from_numpy(A).to(dev))
                Bt = trx.to_colmajor(torch.from_numpy(B).to(dev))
                del A, B
                big = float(k) * k * n
                reps = 3 if big <= 2.0 ** 40 else 1
                rows = {}

                def check(Xs):
                    Xs = np.asfortranarray(Xs.astype(np.float64))
                    eta = oracle.trsm_backward_error("L", "L", "N", "N", alpha, A64, Xs,
                                                     Bs)["eta"]
                    return float(eta), float(oracle.forward_error(Xs, ref))

                X32 = torch.empty_like(Bt)
                for terms in (6, 3, 1):
                    h.set_option(trx.OPT_SPLIT, terms)
                    ms = timed(lambda: trx.trsm("L", "L", "N", "N", alpha, At, X32.copy_(Bt),
                                                handle=h, stream=stream), reps)
                    eta, fe = check(X32[:, cols].cpu().numpy())
                    rows[f"split{terms}"] = {"ms": ms, "backward_error": eta,
                                             "forward_error": fe}
                del X32
                X64 = torch.empty((n, k), dtype=torch.float64, device=dev).t()
                for terms in (3, 1):
                    h.set_option(trx.OPT_SPLIT, terms)
                    h.set_option(trx.OPT_RESIDUAL, trx.RESIDUAL_TC)
                    info = {}

                    def refined():
                        info.update(trx.trsm_refined("L", "L", "N", "N", alpha, At, Bt, out=X64,
                                                     handle=h, tol=1e-6, max_iter=10)[1])
                    ms = timed(refined, reps)
                    eta, fe = check(X64[:, cols].cpu().numpy())
                    rows[f"refine{terms}_1e-6"] = {"ms": ms, "backward_error": eta,
                                                   "forward_error": fe,
                                                   "corrections": info["iterations"],
                                                   "library_backward_error":
                                                       info["backward_error"]}
                h.set_option(trx.OPT_SPLIT, 6)
                h.set_option(trx.OPT_RESIDUAL, trx.RESIDUAL_AUTO)
                if not (k >= 32768 and n == k and not args.all_forms):
                    info = {}

                    def refined64():
                        info.update(trx.trsm_refined("L", "L", "N", "N", alpha, At, Bt, out=X64,
                                                     handle=h)[1])
                    ms = timed(refined64, 1 if big > 2.0 ** 40 else reps)
                    eta, fe = check(X64[:, cols].cpu().numpy())
                    rows["refine6_fp64"] = {"ms": ms, "backward_error": eta, "forward_error": fe,
                                            "corrections": info["iterations"]}
                del X64
                if n == 256 or k <= 8192:
                    A64d, B64d = At.double(), Bt.double()
                    Xd = B64d.clone()
                    ms = timed(lambda: trx.trsm("L", "L", "N", "N", alpha, A64d, Xd.copy_(B64d),
                                                handle=h, stream=stream), 1)
                    eta, fe = check(Xd[:, cols].cpu().numpy())
                    rows["fp64"] = {"ms": ms, "backward_error": eta, "forward_error": fe}
                    del A64d, B64d, Xd
                plain = rows["split6"]["ms"]
                best = min((v["ms"], name) for name, v in rows.items()
                           if v["backward_error"] <= 1e-6)
                line = {"workload": "precision", "k": k, "n": n, "kappa_target": kap,
                        "kappa_estimate": e["kappa_estimate"], "scale": e["scale"],
                        "seed": e["seed"], "checked_columns": len(cols),
                        "oracle_s": t_or, "forms": rows,
                        "fastest_at_1e-6": best[1], "fastest_ms": best[0],
                        "speedup_vs_split6_at_1e-6": plain / best[0]}
                print(json.dumps(line), flush=True)
                summary.append((k, n, kap, best[1], plain / best[0]))
                del At, Bt
                torch.cuda.empty_cache()
    print(json.dumps({"workload": "precision", "summary": [
        {"k": a, "n": b, "kappa": c, "fastest_at_1e-6": d, "speedup_vs_split6": s_}
        for a, b, c, d, s_ in summary]}), flush=True)
    h.close()
    return 0


def run_gemm(args):
    """The recursion's top-level GEMM update alone (trx_sgemm_update, tensor
    cores): C := C - A Y with M = K = k / 2 and N = nrhs (the largest update
    of an order-k TRSM), FP32 data, the handle's split. Times the call (its
    operand-plane conversions included) with CUDA events; the kernel alone
    is what a profiler capture of gemm_tc_kernel isolates."""
    import torch
    import paper_2504_13821_gb300 as trx
    dev = torch.device("cuda", 0)
    h = trx.Handle(dev)
    if args.split:
        h.set_option(trx.OPT_SPLIT, args.split)
    terms = h.get_option(trx.OPT_SPLIT)
    M = K = K_ORDER // 2
    N = NRHS
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    A = trx.to_colmajor(torch.rand(M, K, device=dev, generator=g) / K)
    Y = trx.to_colmajor(torch.randn(K, N, device=dev, generator=g))
    C = trx.to_colmajor(torch.randn(M, N, device=dev, generator=g))
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 1)):
        trx.gemm_update(1.0, -1.0, A, Y, C, handle=h, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        trx.gemm_update(1.0, -1.0, A, Y, C, handle=h, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    peaks, src = load_peaks()
    tflops = 2.0 * M * N * K / (ms * 1e-3) / 1e12
    print(json.dumps({"workload": "gemm", "M": M, "N": N, "K": K, "split_terms": terms,
                      "ms": ms, "tflops_with_conversion": tflops,
                      "peak": peaks["bf16_tflops_sustained"] / terms,
                      "peak_source": f"{src} bf16 sustained / {terms}"}), flush=True)
    h.close()
    return 0


def run_peaks(args):
    """Peak rates of the arithmetic units this library's kernels use, with
    its own probes (trx_peak_probe), under the protocol of the outside BF16
    and HBM measurements: the launch size calibrated to about 50 ms, best of
    10 launches ("burst") and launches back to back for about 4 s
    ("sustained"), SM clocks sampled during the sustained loop. One JSON
    line per kind."""
    import torch
    import paper_2504_13821_gb300 as trx
    dev = torch.device("cuda", 0)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    out = {}
    for kind in ("ffma", "dfma", "dmma", "tc_tf32", "tc_bf16"):
        iters = 64
        while True:                              # calibrate: ~50 ms per launch
            _, ms = trx.peak_probe(kind, iters)
            if ms >= 50.0 or iters > 1 << 40:
                break
            iters = int(iters * max(2.0, min(16.0, 55.0 / max(ms, 1e-3))))
        burst = max(trx.peak_probe(kind, iters)[0] for _ in range(10))
        clocks = ClockSampler(uuid)
        clocks.start()
        t0, rates = time.perf_counter(), []
        while time.perf_counter() - t0 < 4.0:
            rates.append(trx.peak_probe(kind, iters)[0])
        clk = clocks.stop()
        line = {"workload": "peaks", "kind": kind, "burst_tflops": burst,
                "sustained_tflops": float(np.mean(rates)), "launches": len(rates),
                "iters_per_launch": iters, "clocks": clk}
        out[kind] = line
        print(json.dumps(line), flush=True)
    return 0


def latency_stats(arrival: dict, done: dict) -> dict:
    """p50 / p99 latency (ms) and completions per second over a run."""
    if not done:
        return {"count": 0}
    lat = np.array([(done[r] - arrival[r]) * 1e3 for r in done])
    span = max(done.values()) - min(arrival[r] for r in done)
    # the largest latency among the requests arriving in each second
    t0 = min(arrival[r] for r in done)
    per_s = {}
    for r in done:
        b = int(arrival[r] - t0)
        per_s[b] = max(per_s.get(b, 0.0), (done[r] - arrival[r]) * 1e3)
    return {"count": len(done), "p50_ms": float(np.percentile(lat, 50)),
            "p90_ms": float(np.percentile(lat, 90)), "p99_ms": float(np.percentile(lat, 99)),
            "max_ms": float(lat.max()), "mean_ms": float(lat.mean()),
            "solves_per_s": len(done) / span if span > 0 else None,
            "max_ms_by_arrival_second": [round(per_s[b], 2) for b in sorted(per_s)]}


def run_serving(args):
    """Serving workload: open-loop Poisson arrivals (args.rate per second for
    args.duration seconds), 70% TRSM / 30% TRMM, order log-uniform 64..8192,
    right-hand sides log-uniform 1..1024, half FP32-refined and half FP64;
    each factor (same generator) is resident and reused by 1..50 requests;
    admission capped at 150 GB; a request takes one of 32 live factors of
    its precision at random, and a factor is replaced by a new one after its
    1..50 uses. FP32 TRSM requests are refined (the FP32
    solve plus args.refine_corrections float-float corrections, FP64 result)
    unless --no-refine; FP64 TRSM requests take the server's FP64 engine
    (args.fp64_corrections > 0: the FP32 solve plus that many float-float
    corrections; 0: the recursive DFMA solve); TRMM requests run in their
    factor's precision, FP64 TRMM as one float-float pass (--fp64-trmm 1)
    or the DFMA product. Large requests launch directly (--server-graphs:
    cached graphs, captured once per new buffer set). Requests go to the
    library's server (trx_server_*)
    at their arrival time; a request's latency runs from its scheduled
    arrival to the poll that reports it complete. Reports p50/p99 latency
    and solves/s, overall and per request kind."""
    import torch
    from paper_2504_13821_gb300 import serving
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(5)
    # per-stream workspace for the largest FP32 call of the mix (order 8192,
    # 1024 right-hand sides: BF16 operand planes of about 0.3 GB), made up
    # front so no request waits for a workspace to grow
    srv = serving.Server(0, streams=args.server_streams, budget_bytes=150 << 30,
                         max_inflight=4096,
                         workspace_bytes=args.server_workspace_mb << 20,
                         graphs=args.server_graphs,
                         refine_corrections=args.refine_corrections,
                         fp64_corrections=args.fp64_corrections,
                         fp64_trmm=args.fp64_trmm)
    refine = not args.no_refine
    arrival, done, failed, kind = {}, {}, [], {}

    def collect(items):
        now = time.perf_counter()
        for rid, st in items:
            done[rid] = now
            if st != 0:
                failed.append((rid, st))
    def make_factor(k, uplo, dtype):
        A = torch.empty(k, k, device=dev, dtype=dtype).uniform_(-1.0 / k, 1.0 / k)
        A = (torch.tril(A) if uplo == "L" else torch.triu(A))
        A.diagonal().copy_(1 + torch.randn(k, device=dev, dtype=dtype).abs())
        return A.t().contiguous().t()

    # warm-up before the arrivals start: one small and one large factor per
    # precision and triangle, TRSM and TRMM with few and many right-hand
    # sides, through the same generator calls as the run, so module loading
    # (the library's and torch's) and first-use setup are not charged to the
    # first requests
    warm = []
    for dtype in (torch.float32, torch.float64):
        for k, uplo in ((256, "L"), (8192, "U")):
            A = make_factor(k, uplo, dtype)
            fid = srv.register(A, uplo)
            for nrhs in (1, 1024):
                for op in ("S", "M"):
                    Bw = torch.randn(nrhs, k, device=dev, dtype=dtype).t()
                    if op == "S" and dtype == torch.float32 and refine:
                        Xw = torch.empty(nrhs, k, device=dev, dtype=torch.float64).t()
                        warm.append(srv.submit_refined(fid, "L", 1.0, Bw, Xw))
                    else:
                        warm.append(srv.submit(fid, op, "L", 1.0, Bw))
            if k == 8192:
                # the largest solves once per stream: refinement scratch made
                for _ in range(8):
                    Bw = torch.randn(1024, k, device=dev, dtype=dtype).t()
                    if dtype == torch.float32 and refine:
                        Xw = torch.empty(1024, k, device=dev, dtype=torch.float64).t()
                        warm.append(srv.submit_refined(fid, "L", 1.0, Bw, Xw))
                    else:
                        warm.append(srv.submit(fid, "S", "L", 1.0, Bw))
            srv.release(fid)
            del A
    warm_status = dict(srv.drain())
    if sorted(warm_status) != sorted(warm) or any(warm_status.values()):
        raise RuntimeError(f"serving warm-up failed: {warm_status}")
    t_start = time.perf_counter() + 0.5
    t_arr = t_start
    live = {}             # factor id -> [A, uses left, dtype, k, uplo]
    SERVING_POOL = 32
    submitted = 0
    rejected = 0
    flops = 0.0
    while True:
        t_arr += rng.exponential(1.0 / args.rate)
        if t_arr - t_start > args.duration:
            break
        dtype = torch.float64 if rng.random() < args.fp64_share else torch.float32
        # a pool of POOL live factors per precision: a request takes one at
        # random, and a factor leaves the pool after its 1..50 uses, replaced
        # by a new one (so factors are made at the rate their uses run out
        # and the resident set stays bounded)
        cands = [f for f, v in live.items() if v[2] == dtype]
        if len(cands) >= SERVING_POOL:
            fid = cands[int(rng.integers(len(cands)))]
        else:
            k = int(round(np.exp(rng.uniform(np.log(64), np.log(8192)))))
            uplo = str(rng.choice(["L", "U"]))
            A = make_factor(k, uplo, dtype)
            fid = srv.register(A, uplo)
            live[fid] = [A, int(rng.integers(1, 51)), dtype, k, uplo]
        live[fid][1] -= 1
        k = live[fid][3]
        last_use = live[fid][1] == 0
        if last_use:
            live.pop(fid)
        nrhs = int(round(np.exp(rng.uniform(0, np.log(1024)))))
        op = "S" if rng.random() < 0.7 else "M"
        if submitted - len(done) >= args.max_queue:
            # overload: the arrival is turned away (its buffers are never
            # made), so a server that falls behind ends the run with a count
            # of rejections instead of exhausting device memory
            rejected += 1
            if last_use:
                srv.release(fid)
            continue
        B = torch.randn(nrhs, k, device=dev, dtype=dtype).t()     # column-major k x nrhs
        refined = op == "S" and dtype == torch.float32 and refine
        X = torch.empty(nrhs, k, device=dev, dtype=torch.float64).t() if refined else None
        while time.perf_counter() < t_arr:
            collect(srv.poll())
        if refined:
            rid = srv.submit_refined(fid, "L", 1.5, B, X)
        else:
            rid = srv.submit(fid, op, "L", 1.5, B)
        arrival[rid] = t_arr
        kind[rid] = ("fp32-refined TRSM" if refined else
                     ("fp64 " if dtype == torch.float64 else "fp32 ") +
                     ("TRSM" if op == "S" else "TRMM"))
        del B, X                    # the server keeps them until the request completes
        if last_use:
            srv.release(fid)        # dropped once its submitted requests complete
        submitted += 1
        flops += float(k) * k * nrhs
    collect(srv.poll())
    while any(srv.pending()):
        srv.wait()
        collect(srv.poll())
    torch.cuda.synchronize()
    st = latency_stats(arrival, done)
    per_kind = {}
    for name in sorted(set(kind.values())):
        ids = [r for r in done if kind.get(r) == name]
        per_kind[name] = latency_stats({r: arrival[r] for r in ids}, {r: done[r] for r in ids})
    line = {"metric": "served solves/s, p50/p99 ms", "value": st.get("solves_per_s"),
            "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"Poisson {args.rate}/s for {args.duration} s, 70% TRSM, "
                                   "m log-uniform 64..8192, nrhs log-uniform 1..1024, "
                                   f"{args.fp64_share:.0%} FP64 (rest FP32), FP32 TRSM "
                                   + (f"refined ({args.refine_corrections} float-float "
                                      "corrections, FP64 result)" if refine else "plain")
                                   + ", FP64 TRSM "
                                   + (f"FP32 solve + {args.fp64_corrections} float-float "
                                      "corrections" if args.fp64_corrections else "DFMA")
                                   + ", FP64 TRMM "
                                   + ("one float-float pass" if args.fp64_trmm else "DFMA")
                                   + ", factors reused "
                                   f"1..50 times (pool of {SERVING_POOL} live factors per "
                                   "precision), 150 GB admission cap, native request server, "
                                   f"{args.server_streams} streams, "
                                   f"{args.server_workspace_mb} MB workspace per stream, "
                                   + ("cached graphs" if args.server_graphs else
                                      "direct launches"),
                       "requests": submitted, "offered_tflops": flops / args.duration / 1e12,
                       "failed": len(failed), "rejected_overload": rejected,
                       "max_queue": args.max_queue},
            "latency": st, "latency_per_kind": per_kind}
    print(json.dumps(line), flush=True)
    srv.close()
    return 0 if not failed else 1


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="trx", choices=["trx", "reference"])
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--leaf", type=int, default=0, help="recursion cutoff b (0: library default)")
    ap.add_argument("--pdl", action="store_true", help="launch with programmatic dependent launch")
    ap.add_argument("--tc-leaf", action="store_true",
                    help="FP32 TRSM leaves as inverse GEMMs on the tensor cores")
    ap.add_argument("--panels", type=int, default=0, help="TRSM column-panel branches (0: auto)")
    ap.add_argument("--k", type=int, default=None,
                    help="order of A (default 16384, refined workload 8192; smaller only for "
                         "profiling runs)")
    ap.add_argument("--nrhs", type=int, default=None,
                    help="right-hand sides (default 16384, refined workload 256)")
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--dag", type=int, default=0, choices=[-1, 0, 1],
                    help="FP32 TRSM: 1 device-scheduled solve, -1 recursive chain, 0 library default")
    ap.add_argument("--shard", action="store_true",
                    help="N > 1: split the one problem's right-hand sides over the ranks "
                         "(strong scaling) instead of one full copy per rank")
    ap.add_argument("--split", type=int, default=0, choices=[0, 1, 3, 6],
                    help="tensor-core split product terms (0: library default, 6)")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: arrivals per second")
    ap.add_argument("--duration", type=float, default=60.0, help="serving: seconds of arrivals")
    ap.add_argument("--fp64-share", type=float, default=0.5,
                    help="serving: fraction of FP64 requests (the rest FP32)")
    ap.add_argument("--sizes", default=SWEEP_SIZES,
                    help="sweep: orders m = n (precision: 8192,16384,32768)")
    ap.add_argument("--dtypes", default="f32,f64", help="sweep: element types")
    ap.add_argument("--ops", default="trsm,trmm", help="sweep: operations")
    ap.add_argument("--variants", default="all",
                    help="sweep: 'all' or comma-separated variant indices 0..15")
    ap.add_argument("--nrhs-list", default="256,m",
                    help="precision: right-hand sides per order ('m' = the order)")
    ap.add_argument("--all-forms", action="store_true",
                    help="precision: also the FP64-level refinement at m = n = 32768")
    ap.add_argument("--workload", default="square",
                    choices=["square", "batched", "serving", "refined", "sweep", "precision",
                             "peaks", "gemm"],
                    help="square: the n=16384 TRSM+TRMM step (default); batched: "
                         "4096 small uneven problems in one launch; serving: Poisson "
                         "arrivals; refined: FP32 TRSM refined in FP64 (k 8192, 256 "
                         "right-hand sides unless --k/--nrhs say otherwise)")
    ap.add_argument("--count", type=int, default=4096, help="problems (batched workload)")
    ap.add_argument("--server-streams", type=int, default=8,
                    help="serving: parallel streams (one handle each) for large requests")
    ap.add_argument("--server-graphs", action="store_true",
                    help="serving: large requests replay cached graphs (one capture per new "
                         "buffer set) instead of launching directly")
    ap.add_argument("--fp64-trmm", type=int, default=1, choices=[0, 1],
                    help="serving: FP64 TRMM as one float-float pass (1) or DFMA (0)")
    ap.add_argument("--refine-corrections", type=int, default=1,
                    help="serving: corrections of a refined FP32 TRSM request")
    ap.add_argument("--fp64-corrections", type=int, default=2,
                    help="serving: FP64 TRSM as FP32 solve + this many corrections (0: DFMA)")
    ap.add_argument("--max-queue", type=int, default=5000,
                    help="serving: requests submitted and not yet completed beyond which "
                         "arrivals are rejected")
    ap.add_argument("--no-refine", action="store_true",
                    help="serving: FP32 TRSM requests plain (no refinement)")
    ap.add_argument("--server-workspace-mb", type=int, default=512,
                    help="serving: per-stream workspace made when the server starts")
    ap.add_argument("--kappa", type=float, default=None,
                    help="refined workload: only the factor of this target condition number")
    ap.add_argument("--no-loop", action="store_true",
                    help="batched workload: skip the loop of single calls (profiling runs)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batched workload: keep the default block sizes (for profiling runs)")
    args = ap.parse_args(argv)
    global K_ORDER, NRHS, DTYPE
    refined = args.workload == "refined"
    K_ORDER = args.k if args.k is not None else (8192 if refined else 16384)
    NRHS = args.nrhs if args.nrhs is not None else (256 if refined else 16384)
    DTYPE = np.float32 if args.dtype == "f32" else np.float64
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "refined":
        return run_refined(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "peaks":
        return run_peaks(args)
    if args.workload == "gemm":
        return run_gemm(args)
    if args.workload == "precision":
        if args.sizes == SWEEP_SIZES:
            args.sizes = "8192,16384,32768"
        return run_precision(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
