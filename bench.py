"""Benchmark: amplitudes/s of random grid circuits by complex graphical-model
variable elimination on one GB300 (and N replicas under torchrun).

Default workload: 5x5 grid, depth 20, seed 0, a batch of 1024 uniformly random
output bitstrings, complex64 elimination with an FP64 slice sum.  One step =
one full pass of the path (leaf factors for the batch, every elimination step,
FP64 accumulation) over one batch.  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference   # the FP64 CPU oracle on a bounded sample
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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import qgm_inputs as qi  # noqa: E402

METRIC = "amplitudes/sec on 1 GB300 at stated rel. error vs FP64; % of tensor/HBM roofline"
UNIT = "amplitudes/s"
L2_BYTES = 129 * 2 ** 20

# DRAM traffic per launch of the dominant kernel from one ncu capture, keyed by
# the sha1 of the kernel source it was taken on (null once the source changed):
# for the compiled resident executor, the CUDA source generated for the plan.
NCU_TRAFFIC = {"e03135235b82": 141824.0}   # qgm_resident_plan, profiles/qgm_resident_plan_grid5x5_d20_b1024.md


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="grid5x5_d20_b1024", choices=sorted(qi.WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--executor", type=int, default=0, help="0 auto, 1 stepwise, 2 resident, 3 compiled resident")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_hash(plan=None, chunk=1):
    """sha1 (12 hex digits) of the dominant kernel's source: the CUDA source
    generated for the plan when the compiled resident executor runs it, else
    exec.cu (the other executors' kernels)."""
    h = hashlib.sha1()
    if plan is not None:
        h.update(plan.kernel_source(chunk, 0).encode())
    else:
        with open(os.path.join(ROOT, "paper_1712_05384_gb300", "csrc", "exec.cu"), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""
        else:
            self.out = ""

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_rate(c, bits, seconds):
    """FP64 oracle (bucket elimination, vertical order) on a time-bounded sample."""
    from oracle import ugm, ve
    m = ugm.build(c)
    order = ve.vertical_order(m, c)
    t0 = time.perf_counter()
    done = 0
    for x in bits:
        ve.amplitude(c, x, m, order)
        done += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return done / dt, done, dt


def run_reference(args, rank, world):
    if rank != 0:
        return
    rows, cols, depth, B, param = qi.WORKLOADS[args.workload]
    c = qi.grid_circuit(rows, cols, depth, 0, param=param)
    bits = qi.bitstrings(c.n, max(B, 1), 0)
    per_step = max(1, min(len(bits), 8))
    from oracle import ugm, ve
    m = ugm.build(c)
    order = ve.vertical_order(m, c)
    for w in range(args.warmup):
        for x in bits[:per_step]:
            ve.amplitude(c, x, m, order)
    t0 = time.perf_counter()
    for s in range(args.steps):
        sel = bits[(s * per_step) % len(bits):][:per_step]
        for x in sel:
            ve.amplitude(c, x, m, order)
    dt = time.perf_counter() - t0
    n_amp = per_step * args.steps
    v = n_amp / dt
    sample = (f"{per_step} bitstrings per step of the {args.workload} workload, "
              f"FP64 bucket elimination in the vertical order (oracle/ve.py)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "grid": f"{rows}x{cols}", "depth": depth,
                   "batch_per_gpu": B, "seed": 0, "parallelism": "replicas1",
                   "sample_per_step": per_step},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    import torch.distributed as dist
    import paper_1712_05384_gb300 as q
    from paper_1712_05384_gb300 import build

    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    q.lib()

    rows, cols, depth, B, param = qi.WORKLOADS[args.workload]
    if B == 0:
        raise SystemExit("the benchmark runs batch workloads")
    c_py = qi.grid_circuit(rows, cols, depth, 0, param=param)
    # weak scaling: each rank takes its own batch of B bitstrings (a
    # contiguous block of the job's B * world; no data-path collective)
    from paper_1712_05384_gb300 import shard
    all_bits = qi.bitstrings(c_py.n, B * world, 0)
    bits = shard.shard(all_bits, rank, world)
    plan = q.Plan(q.Model(q.Circuit.grid(rows, cols, depth, 0, param)), batch=B,
                  executor=args.executor).bind()
    info = plan.info
    stream = torch.cuda.current_stream(dev)
    d_bits = torch.from_numpy(bits.astype(np.int64)).to(dev)
    d_out = torch.empty(2 * B, dtype=torch.float64, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        plan.amplitudes(d_bits, d_out, B=B, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if plan.status(stream) != 0:
        raise RuntimeError("device status not OK after warm-up")

    # device-timed region: K steps, L2 flushed (untimed) between them
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            step()
            evs[i][1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_ms = sum(a.elapsed_time(b) for a, b in evs)
    if world > 1:
        t = torch.tensor([t_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_ms = float(t.item())
    value = world * B * args.steps / (t_ms / 1e3)

    # end to end through the public host API: host bitstrings in, host
    # amplitudes out, copies inside the timed region
    hb = torch.from_numpy(bits.view(np.int64).copy()).pin_memory()
    hout = torch.empty(2 * B, dtype=torch.float64).pin_memory()
    for _ in range(3):
        q._lib.check(q.lib().qgm_amplitudes_host(plan._h, hb.data_ptr(), B, hout.data_ptr(),
                                                 stream.cuda_stream))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        q._lib.check(q.lib().qgm_amplitudes_host(plan._h, hb.data_ptr(), B, hout.data_ptr(),
                                                 stream.cuda_stream))
    e2e_s = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = world * B * args.steps / e2e_s

    # roofline of the dominant kernel, per-launch times from a pass with CUDA
    # events on the launching stream
    step_bytes, step_flops = plan.step_costs()
    ex_kind, ex_chunk, ex_smem = plan.executor()
    reps = 5
    ms = np.zeros(info.n_steps + 2)
    for _ in range(reps):
        flush.fill_(1.0)
        ms += plan.profile(d_bits, d_out, B=B, stream=stream)
    ms /= reps
    traffic = NCU_TRAFFIC.get(kernel_hash(plan if ex_kind == q.EXEC_COMPILED else None, ex_chunk))
    if ex_kind in (q.EXEC_RESIDENT, q.EXEC_COMPILED):
        # all intermediates live in shared memory: bound by the SM's FP32/ALU
        # issue, peak = 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz
        k_ms = float(ms[0])
        peak = 152 * 128 * 2 * 2.070e9 / 1e12
        achieved = float(step_flops.sum()) / (k_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": f"{'qgm_resident_plan (compiled for this plan)' if ex_kind == q.EXEC_COMPILED else 'k_resident'}"
                          f" (whole pass, {ex_chunk} bitstring(s) per CTA, {ex_smem} B shared memory)",
                "algorithmic_flops_per_pass": float(step_flops.sum()),
                "algorithmic_bytes_per_pass": float(step_bytes.sum()),
                "kernel_ms_per_pass": k_ms,
                "peak_source": "derived: FP32 lanes x SMs x max SM clock"}
        launches = args.steps
    else:
        k_ms = float(ms[1:-1].sum())
        achieved = float(step_bytes.sum()) / (k_ms / 1e3) / 1e9
        peak, peak_kind = peaks()
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "k_step_batched (all elimination steps)",
                "algorithmic_bytes_per_pass": float(step_bytes.sum()),
                "kernel_ms_per_pass": k_ms, "peak_source": peak_kind}
        launches = args.steps * int(info.n_slices * (info.n_steps + 2) + 1)

    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": t_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64",
        "data": "synthetic",
        "config": {"workload": args.workload, "grid": f"{rows}x{cols}", "depth": depth,
                   "batch_per_gpu": B, "seed": 0, "order": info.order_kind,
                   "max_clique": info.max_clique, "steps_per_pass": info.n_steps,
                   "slices": info.n_slices, "parallelism": f"replicas{world}",
                   "executor": {1: "stepwise", 2: "resident", 3: "compiled resident"}.get(ex_kind), "chunk": ex_chunk,
                   "gemm_steps": info.n_gemm_steps, "gemm_steps_split_bf16": info.n_gemm_tc_steps,
                   "l2": "flushed between timed steps (264 MB write, untimed)"},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 8 * B,
                "d2h_bytes_per_step": 16 * B},
        "roofline": roof,
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, done, dt = cpu_oracle_rate(c_py, bits, args.cpu_seconds)
        res["cpu_baseline"] = {
            "value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {done} of the {B} bitstrings, {dt:.1f} s, FP64 bucket elimination "
                      f"(oracle/ve.py, vertical order, numpy single thread)"}
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
