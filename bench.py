#!/usr/bin/env python
"""Benchmark of the GB300 inverse-factorization path.

One step = one complete factorization of the workload's synthetic overlap
matrix S (resident in HBM) through the C ABI: truncation of S, Gershgorin
bound, every refinement sweep (block-sparse products with truncation, sums,
norms, stop tests) until the stop rule, returning Z.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload NAME]

Prints one JSON line.  `value` is factorizations per second over all ranks
(each rank factorizes its own copy: weak scaling, no collective on the data
path).  `e2e` repeats the measurement with S in pinned host memory and Z read
back to pinned host memory inside the timed region.  `roofline` rates the
FP64 block-product kernel by its algorithmic flops (2 bs^3 per multiplied
block pair) over its CUDA-event time.  `--impl reference` times the CPU
oracle on the same workload.
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
sys.path.insert(0, ROOT)

WORKLOADS = {
    # 1D chain of 4096 normalized s-Gaussians, spacing 1.4 bohr +-0.1, exponents
    # (0.17, 0.62, 3.4); BSR 32x32; tau = 1e-10; FP64 refinement from I/sqrt(beta)
    "irsi-chain-n4096-bs32": dict(geom="chain", n=4096, bs=32, tau=1e-10, target=1e-10, method="refine", m=2,
                                  seed=0, leaf=512),
    # the same chain through localized inverse factorization (512-row leaves)
    "lif-chain-n4096-bs32": dict(geom="chain", n=4096, bs=32, tau=1e-10, target=1e-10, method="localized", m=2,
                                 seed=0, leaf=512),
}
DEFAULT_WORKLOAD = "irsi-chain-n4096-bs32"
METRIC = "Inverse-factor time & block-GEMM TFLOP/s: mixed vs FP64 at ||I-Z*SZ||_F<=1e-10"
UNIT = "factorizations/s"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["bf16_tflops"]), float(m["hbm_gbs"]), "measured"
    except Exception:
        return 1900.0, 6800.0, "fallback"


def fp64_peak_tflops():
    """FP64 peak: the measured dense-bf16 peak times the nominal FP64/BF16
    ratio of GB300 (1.25 / 2250 TFLOP/s)."""
    bf16, _, src = _peaks()
    return bf16 * 1.25 / 2250.0, src


def make_input(w):
    from paper_1901_07993_gb300 import synth
    if w["geom"] == "chain":
        return synth.chain_overlap(w["n"], w["bs"], seed=w["seed"])
    return synth.cluster_overlap(w["n"], w["bs"], seed=w["seed"])


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
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
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        except OSError:
            return None
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(want_nccl: bool):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if want_nccl else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(world, x: float) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_factorize(S, w):
    import oracle
    if w["method"] == "refine":
        return oracle.irsi(S, m=w["m"], tau=w["tau"], target=w["target"])
    return oracle.lif(S, m=w["m"], tau=w["tau"], target=w["target"], leaf_size=w["leaf"])


def cpu_baseline(S, w, budget_s: float = 10.0):
    """The oracle, as it stands, on the same workload for about budget_s."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    count = 0
    while True:
        oracle_factorize(S, w)
        count += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": count / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{count} complete factorization(s) of the same workload, single-threaded FP64 C, {dt:.1f} s"}


def run_reference(args, w, world, rank):
    """CPU oracle arm (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    S = make_input(w)
    for _ in range(args.warmup):
        oracle_factorize(S, w)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_factorize(S, w)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    v = args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, **{k: w[k] for k in ("n", "bs", "tau", "target", "m")}},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} complete factorizations (plus {args.warmup} warm-up)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    w = WORKLOADS[args.workload]

    if args.impl == "reference":
        world, rank, _ = dist_setup(want_nccl=False)
        run_reference(args, w, world, rank)
        return

    import numpy as np
    import torch
    world, rank, local = dist_setup(want_nccl=True)
    torch.cuda.set_device(local)
    from paper_1901_07993_gb300 import build as libbuild
    from paper_1901_07993_gb300 import ifac
    libbuild.build()
    ctx = ifac.Context()
    S_h = make_input(w)
    S = ifac.upload(ctx, S_h)
    o = ifac.opts(m=w["m"], leaf_size=w["leaf"], profile=True)
    factor = ifac.inv_factor_refine if w["method"] == "refine" else ifac.inv_factor_localized
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):
        Z, rep = factor(ctx, S, w["tau"], w["target"], o)
        del Z
    torch.cuda.synchronize()

    # ---- device-resident timed region ----
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    reps = []
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()  # L2 flush between timed steps, outside the events
            starts[k].record()
            Z, rep = factor(ctx, S, w["tau"], w["target"], o)
            ends[k].record()
            reps.append(rep)
            if k < args.steps - 1:
                del Z
        torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = allmax(world, sum(step_ms))
    value = world * args.steps / (total_ms / 1e3)

    # roofline of the FP64 block-product kernel (events around each launch)
    gemm_ms = sum(r.gemm_ms for r in reps)
    gemm_flops = sum(r.flops for r in reps)
    launches = sum(r.gemm_launches for r in reps)
    achieved = gemm_flops / (gemm_ms / 1e3) / 1e12 if gemm_ms > 0 else 0.0
    peak, peak_src = fp64_peak_tflops()
    roofline = {"bound": "alu", "kernel": "k_gemm_fp64<%d>" % w["bs"], "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_source": f"{peak_src} bf16 x nominal FP64/BF16 ratio 1.25/2250",
                "launches_per_step": launches / args.steps,
                "flops_per_launch": gemm_flops / max(launches, 1),
                "avg_launch_us": 1e3 * gemm_ms / max(launches, 1),
                "gemm_share_of_step": gemm_ms / sum(step_ms)}

    # ---- end to end through the C ABI with pinned host buffers ----
    def pinned(a):
        t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()

    S_pin = type(S_h)(S_h.n, S_h.bs, pinned(S_h.row_ptr), pinned(S_h.col_idx), pinned(S_h.val))
    nnzb_Z = reps[-1].nnzb_Z
    z_rp = pinned(np.zeros(S_h.nb + 1, np.int32))
    z_ci = pinned(np.zeros(nnzb_Z, np.int32))
    z_val = pinned(np.zeros((nnzb_Z, w["bs"], w["bs"])))
    o_e2e = ifac.opts(m=w["m"], leaf_size=w["leaf"])
    e2e_ms = []
    barrier(world)
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Sd = ifac.upload(ctx, S_pin)
        Zd, rep_e = factor(ctx, Sd, w["tau"], w["target"], o_e2e)
        assert rep_e.nnzb_Z == nnzb_Z
        ctx.check(ctx.lib.ifac_bsr_download(ctx.h, Zd.ptr(), z_rp.ctypes.data, z_ci.ctypes.data,
                                            z_val.ctypes.data))
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        del Zd, Sd
    barrier(world)
    e2e_total = allmax(world, sum(e2e_ms))
    h2d = S_h.row_ptr.nbytes + S_h.col_idx.nbytes + S_h.val.nbytes
    d2h = z_rp.nbytes + z_ci.nbytes + z_val.nbytes

    resid = ifac.inv_factor_resid(ctx, S, Z)
    clocks = clk.summary()
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(S_h, w)
    r0 = reps[-1]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "geometry": w["geom"], "n": w["n"], "bs": w["bs"], "tau": w["tau"],
                   "target": w["target"], "m": w["m"], "method": w["method"], "parallelism": f"replicas{world}",
                   "l2": "flushed between timed steps (512 MB write)"},
        "block_gemm_tflops": gemm_flops / (sum(step_ms) / 1e3) / 1e12,
        "s_per_factorization": total_ms / args.steps / 1e3,
        "resid_fro": resid, "resid_target_met": resid <= w["target"],
        "sweeps": r0.sweeps, "delta_fro": r0.delta_fro, "nnzb_Z": r0.nnzb_Z, "block_pairs": r0.block_pairs,
        "gpu_launches": int(sum(r.launches for r in reps)),
        "roofline": roofline,
        "e2e": {"value": world * args.steps / (e2e_total / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
