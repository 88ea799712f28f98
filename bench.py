#!/usr/bin/env python
"""Benchmark of the GB300 inverse-factorization path.

One step = one complete factorization of the workload's synthetic overlap
matrix S (resident in HBM) through the C ABI: truncation of S, Gershgorin
bound, every refinement sweep (block-sparse products with truncation, sums,
norms, stop tests) until the stop rule, returning Z.  The default workload
factorizes a 262,144-row 1D-chain overlap matrix (BSR 64 x 64, tau = 1e-12)
to ||I - Z^T S Z||_F <= 1e-10 with TF32 tensor-core products and FP64 final
delta evaluations; the same factorization with FP64 products and with BF16
products is timed beside it ("compare").

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload NAME]

Prints one JSON line.  `value` is factorizations per second over all ranks
(each rank factorizes its own copy: weak scaling, no collective on the data
path).  `e2e` repeats the measurement with S in pinned host memory and Z read
back to pinned host memory inside the timed region.  `roofline` rates the
block-product kernel with the most device time by its algorithmic flops
(2 bs^3 per multiplied stored block pair; per slice pair for split products)
over its CUDA-event time; `kernels` lists every block-product kernel of the
run.  `--impl reference` times the CPU oracle on the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # 1D chain of 4096 normalized s-Gaussians, spacing 1.4 bohr +-0.1, exponents
    # (0.17, 0.62, 3.4); BSR 32x32; tau = 1e-10; FP64 refinement from I/sqrt(beta)
    "irsi-chain-n4096-bs32": dict(geom="chain", n=4096, bs=32, tau=1e-10, target=1e-10, method="refine", m=2,
                                  seed=0, leaf=512, prec="fp64", compare=(), sample_n=None),
    # the same construction at n = 262,144 in BSR 64x64, tau = 1e-12 (the 1e-10
    # target is reachable): TF32 products, FP64 delta at the end; FP64 and BF16 beside
    "irsi-mixed-chain-n262144-bs64": dict(geom="chain", n=262144, bs=64, tau=1e-12, target=1e-10, method="refine",
                                          m=2, seed=0, leaf=512, prec="tf32", compare=("fp64", "bf16"),
                                          sample_n=4096),
    # one block-sparse product on a fully dense 256 x 256 pattern of 64 x 64
    # blocks (n = 16384), BF16 inputs, FP32 accumulation: the tensor-core kernel alone
    "product-dense-bf16-n16384": dict(geom="dense", n=16384, bs=64, tau=0.0, target=0.0, method="product", m=2,
                                      seed=1, leaf=512, prec="bf16", compare=(), sample_n=None),
    # the same at n = 8192 (operands of about L2 size): the profiling case
    "product-dense-bf16-n8192": dict(geom="dense", n=8192, bs=64, tau=0.0, target=0.0, method="product", m=2,
                                     seed=1, leaf=512, prec="bf16", compare=(), sample_n=None),
    # the split FP64-accurate product (7 BF16 slices, 28 slice pairs) on the
    # same dense pattern at n = 8192: the profiling case of the split kernel
    "product-dense-split-n8192": dict(geom="dense", n=8192, bs=64, tau=0.0, target=0.0, method="product", m=2,
                                      seed=1, leaf=512, prec="split", compare=(), sample_n=None),
    # config 3's recipe on its 3D geometry (random sequential addition at 0.1
    # points per bohr^3, RCB order) at the largest size that fits in HBM with
    # every intermediate in FP64: n = 32,768, bs 64, block-dense factor.  TF32
    # sweeps, then delta with split FP64-accurate products of 8 slices (dense
    # operands need the 8th: 7 slices err by about 2e-10 in ||delta||_F at
    # n = 3072), tau = 1e-14 (at 1e-12 the truncated products of delta miss
    # about sqrt(blocks) x tau of the residual)
    "irsi-mixed-cluster-n32768-bs64": dict(geom="cluster", n=32768, bs=64, tau=1e-14, target=1e-10,
                                           method="refine", m=2, seed=0, leaf=512, prec="tf32", compare=(),
                                           sample_n=2048, cost_exp=3, split_slices=8),
    # the same at n = 16,384 beside the FP64 schedule with every product on the
    # split kernel (FP64-accurate throughout): the mixed-vs-FP64 comparison
    # on the 3D geometry
    "irsi-mixed-cluster-n16384-bs64": dict(geom="cluster", n=16384, bs=64, tau=1e-14, target=1e-10,
                                           method="refine", m=2, seed=0, leaf=512, prec="tf32", compare=("split",),
                                           sample_n=2048, cost_exp=3, split_slices=8),
    # the mixed-precision refinement at n = 65,536: the profiling case of the
    # kernels of the default workload (a quarter of its rows)
    "irsi-mixed-chain-n65536-bs64": dict(geom="chain", n=65536, bs=64, tau=1e-12, target=1e-10, method="refine",
                                         m=2, seed=0, leaf=512, prec="tf32", compare=(), sample_n=4096),
    # 64 independent matrices refined together: 32 chains and 32 3D clusters,
    # sizes log-uniform in [512, 8192] (seed 3, member j generated with seed
    # 3000 + j), BSR 64x64, tau = 1e-12 (the 1e-10 target is reachable), the
    # mixed schedule per member (TF32 sweeps, then delta with split FP64-accurate
    # products of 8 slices: the 3D members' floors need the extra 7 bits),
    # FP64-accurate final residual of every member
    "batch64-tf32-n512-8192": dict(geom="batch", n=0, bs=64, tau=1e-12, target=1e-10, method="batched", m=2,
                                   seed=3, leaf=512, prec="tf32", compare=(), sample_n=None,
                                   count=64, nmin=512, nmax=8192, split_slices=8),
    # config 4 over [2048, 16384] (the upper half of [16384, 32768] does not
    # fit the device with FP64 intermediates of the dense 3D members), block
    # size and bs-64 tile schedule picked by the library's autotuner from
    # timed probes of the generated members (generated at bs 64, re-blocked);
    # tau = 1e-14: the 3D members hold up to 60,000 blocks, and delta
    # evaluated from products truncated at 1e-12 misses about
    # sqrt(blocks) x 1e-12 > 1e-10 of the true residual
    "batch64-tf32-n2048-16384": dict(geom="batch", n=0, bs=64, tau=1e-14, target=1e-10, method="batched", m=2,
                                     seed=3, leaf=512, prec="tf32", compare=(), sample_n=None,
                                     count=64, nmin=2048, nmax=16384, split_slices=8, autotune=True),
    # the adjoint: L = tr(Z_6^T F Z_6) after 6 frozen-pattern sweeps on the
    # 16,384-row chain (bs 32), F = N(0,1) * S_ij symmetric (seed 5); one step =
    # recording run + reverse pass (dL/dS), FP64
    "adjoint-chain-n16384-bs32": dict(geom="chain", n=16384, bs=32, tau=1e-10, target=0.0, method="adjoint", m=2,
                                      seed=0, leaf=512, prec="fp64", compare=(), sample_n=None, K=6, fseed=5),
    # the 16,384-row chain through recursive inverse Cholesky (Algorithm 1;
    # 128-row leaves, 7 levels: the fastest of 64/128/256/512 on the box), FP64
    "rinch-chain-n16384-bs32": dict(geom="chain", n=16384, bs=32, tau=1e-10, target=1e-8, method="rinch", m=2,
                                    seed=0, leaf=128, prec="fp64", compare=(), sample_n=None),
    # the 4096-row 3D cluster through localized inverse factorization that
    # switches to recursive inverse Cholesky at 2048 rows (the paper switches
    # below 16384), 128-row leaves, FP64
    "lif-rinch-cluster-n4096-bs32": dict(geom="cluster", n=4096, bs=32, tau=1e-10, target=1e-10,
                                         method="localized", m=2, seed=0, leaf=128, prec="fp64", compare=(),
                                         sample_n=None, rinch_rows=2048),
    # the paper's settings (Section 5: m = 4, tau = 1e-5 after every product,
    # on S and on leaves, local delta for the refinements, bs 32) for the three
    # methods on a 65,536-row chain and a 16,384-row 3D cluster; LIF switches
    # to RINCH at 4096 / 2048 rows (the paper: 16384 rows of 5.4M / 2.0M).
    # Reports ||I - Z^T S Z||_F per method (the quantities of Table 1)
    "table1-paper-settings": dict(geom="pair", n=0, bs=32, tau=1e-5, target=0.0, method="table1", m=4,
                                  seed=0, leaf=512, prec="fp64", compare=(), sample_n=None,
                                  cases=(("chain", 65536, 4096), ("cluster", 16384, 2048))),
    # the config-2 recipe (3D cluster, LIF, 512-row leaves, tau 1e-10) at
    # n = 8192 in BSR 64x64 with every product on the split FP64-accurate
    # tensor-core kernel (the FP64 pipe needs seconds at n = 4096 already)
    "lif-split-cluster-n8192-bs64": dict(geom="cluster", n=8192, bs=64, tau=1e-10, target=1e-10,
                                         method="localized", m=2, seed=0, leaf=512, prec="split", compare=(),
                                         sample_n=1024, cost_exp=3),
    # the same recipe at n = 16,384: the size scaling of LIF on the 3D geometry
    "lif-split-cluster-n16384-bs64": dict(geom="cluster", n=16384, bs=64, tau=1e-10, target=1e-10,
                                          method="localized", m=2, seed=0, leaf=512, prec="split", compare=(),
                                          sample_n=1024, cost_exp=3),
    # the 4096-row chain through localized inverse factorization (512-row leaves)
    "lif-chain-n4096-bs32": dict(geom="chain", n=4096, bs=32, tau=1e-10, target=1e-10, method="localized", m=2,
                                 seed=0, leaf=512, prec="fp64", compare=(), sample_n=None),
}
DEFAULT_WORKLOAD = "irsi-mixed-chain-n262144-bs64"
PREC = {"fp64": 0, "tf32": 1, "bf16": 2, "split": 3}
METRIC = "Inverse-factor time & block-GEMM TFLOP/s: mixed vs FP64 at ||I-Z*SZ||_F<=1e-10"
UNIT = "factorizations/s"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# block-product kernels, averaged over the launches of the first
# factorization of the workload, from an ncu capture of that workload
# (--clock-control none, one pass; profiles/ holds the summaries and the
# commands).  A kernel changed since its capture has no entry.  Keyed by
# workload, then by kernel_rooflines' kernel key.
DRAM_TRAFFIC = {
    "irsi-mixed-chain-n262144-bs64": {
        "tc": (562179475.7, "ncu capture of this workload's first factorization: k_gemm_band_lp<4>, 26 launches"),
        "split": (2087311104.0, "ncu capture of this workload's first factorization: k_gemm_split_band, 8 launches"),
    },
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["bf16_tflops"]), float(m["hbm_gbs"]), "measured"
    except Exception:
        return 1900.0, 6800.0, "fallback"


def hbm_peak_gbs():
    """Measured copy bandwidth (MEASURED_PEAKS.json), else the fallback."""
    _, hbm, src = _peaks()
    return hbm, src


def fp64_peak_tflops():
    """FP64 peak: the measured dense-bf16 peak times the nominal FP64/BF16
    ratio of GB300 (1.25 / 2250 TFLOP/s)."""
    bf16, _, src = _peaks()
    return bf16 * 1.25 / 2250.0, src


def tensor_peak_tflops(prec: str):
    """Dense tensor peak for the product's input format: measured bf16, or
    measured bf16 times the nominal TF32/BF16 ratio (1.1 / 2.25 PFLOP/s)."""
    bf16, _, src = _peaks()
    return (bf16 if prec == "bf16" else bf16 * 1.1 / 2.25), src


def make_input(w, n=None):
    from paper_1901_07993_gb300 import synth
    n = n or w["n"]
    if w["geom"] == "chain":
        return synth.chain_overlap(n, w["bs"], seed=w["seed"])
    return synth.cluster_overlap(n, w["bs"], seed=w["seed"])


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        # raw samples beside the run's other outputs (BENCH_CLOCKS_DIR), else the temp directory
        self.path = os.path.join(os.environ.get("BENCH_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"clocks_{os.getpid()}.csv")

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
    if w["method"] == "rinch":
        return oracle.rinch(S, tau=w["tau"], leaf_size=w["leaf"])
    return oracle.lif(S, m=w["m"], tau=w["tau"], target=w["target"], leaf_size=w["leaf"],
                      rinch_rows=w.get("rinch_rows", 0))


def nproc() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_sizes(w):
    """Two sizes of the workload's construction at which the oracle is timed
    to measure how its cost grows with n: n/16 and n/4 for the chain (at
    least 16,384 rows for the 262,144-row workload), the sample size and half
    of it for the 3D clusters (block-dense factors, cubic cost)."""
    if w["geom"] == "chain" and w["n"] >= 65536:
        return w["n"] // 16, w["n"] // 4
    s = w.get("sample_n") or w["n"]
    return max(s // 2, w["bs"] * 4), s


def _oracle_seconds(S, w, threads, runs=1):
    import oracle
    oracle.set_threads(threads)
    best = float("inf")
    for _ in range(runs):
        t0 = time.perf_counter()
        oracle_factorize(S, w)
        best = min(best, time.perf_counter() - t0)
    return best


def cpu_baseline(w, full_budget_s: float = 20.0):
    """The oracle, as it stands, on the machine's host cores: single-threaded and
    with all cores (OpenMP over output block rows), each timed at two sizes
    of the workload's construction to measure the cost exponent p of
    t ~ n^p.  The all-core oracle also factorizes the full workload when its
    predicted time is within full_budget_s (then `value` is measured, not
    scaled); the single-threaded figure is scaled from the larger size with
    the measured exponent."""
    import math

    import oracle
    oracle.build()
    cores = nproc()
    n1, n2 = cpu_sizes(w)
    S1, S2 = make_input(w, n1), make_input(w, n2)
    t = {}
    for th in (1, cores):
        _oracle_seconds(S1, w, th)  # warm-up (page-in, first touch)
        t[(th, n1)] = _oracle_seconds(S1, w, th, runs=2)
        t[(th, n2)] = _oracle_seconds(S2, w, th, runs=1 if th == 1 else 2)
    exps = {th: math.log(t[(th, n2)] / t[(th, n1)]) / math.log(n2 / n1) for th in (1, cores)}
    n = w["n"]
    pred_all = t[(cores, n2)] * (n / n2) ** exps[cores]
    if n == n2:
        t_all, how = t[(cores, n2)], "measured on the workload itself"
    elif pred_all <= full_budget_s:
        t_all, how = _oracle_seconds(make_input(w), w, cores, runs=1), "measured on the workload itself"
    else:
        t_all, how = pred_all, f"scaled from n = {n2} with the measured exponent"
    t_one = t[(1, n2)] * (n / n2) ** exps[1]
    oracle.set_threads(cores)
    return {"value": 1.0 / t_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"complete FP64 factorizations by the C oracle with OpenMP over output block rows on "
                       f"{cores} cores ({how}); timed at n = {n1} and {n2}: "
                       f"{t[(cores, n1)]:.3g} s and {t[(cores, n2)]:.3g} s, cost exponent {exps[cores]:.2f}"),
            "single_thread": {"value": 1.0 / t_one, "unit": UNIT, "cores": 1,
                              "seconds_at": {str(n1): t[(1, n1)], str(n2): t[(1, n2)]},
                              "cost_exponent": exps[1],
                              "sample": f"scaled from n = {n2} to n = {n} by (n/{n2})^{exps[1]:.2f}"},
            "all_core_cost_exponent": exps[cores], "parallel_speedup_at_n2": t[(1, n2)] / t[(cores, n2)]}


def run_reference(args, w, world, rank):
    """CPU oracle arm (rank 0 only): every step is one factorization of the
    workload by the oracle with all host cores, when that fits the time
    budget; otherwise of the larger sample size, scaled by the measured cost
    exponent."""
    if rank != 0:
        return
    if w["method"] not in ("refine", "rinch", "localized"):
        print(json.dumps({"impl": "reference", "unavailable": f"the oracle arm times factorizations; "
                          f"workload {args.workload} ({w['method']}) has no single-factorization reference"}),
              flush=True)
        return
    import math

    import oracle
    oracle.build()
    cores = nproc()
    oracle.set_threads(cores)
    S = make_input(w)
    t_first = _oracle_seconds(S, w, cores)
    scale, what = 1.0, "complete FP64 factorizations of the workload itself"
    if t_first * (args.steps + args.warmup) > 300.0:
        n1, n2 = cpu_sizes(w)
        S1, S = make_input(w, n1), make_input(w, n2)
        t1, t2 = _oracle_seconds(S1, w, cores), _oracle_seconds(S, w, cores)
        p = math.log(t2 / t1) / math.log(n2 / n1)
        scale = (n2 / w["n"]) ** p
        what = (f"complete FP64 factorizations of the same construction at n = {n2}, rate scaled by "
                f"({n2}/{w['n']})^{p:.2f} (exponent measured at n = {n1} and {n2})")
    for _ in range(max(args.warmup - 1, 0)):
        oracle_factorize(S, w)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_factorize(S, w)
        times.append(time.perf_counter() - t0)
    tot = sum(times) / scale
    v = args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64",  # the oracle computes every step in FP64
            "data": "synthetic", "config": config_of(w, args.workload, world),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} {what} (plus {args.warmup} warm-up), OpenMP over output "
                                       f"block rows on {cores} cores"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(w, name, world):
    return {"workload": name, "geometry": w["geom"], "n": w["n"], "bs": w["bs"], "tau": w["tau"],
            "target": w["target"], "m": w["m"], "method": w["method"], "precision": w["prec"],
            "parallelism": f"replicas{world}", "l2": "flushed between timed steps (512 MB write)"}


DTYPE = {"fp64": "f64", "tf32": "tf32/f32acc+f64", "bf16": "bf16/f32acc+f64", "split": "f64 (bf16 slices, exact f32acc)"}


def timed_factorizations(ctx, ifac, factor, S, w, o, steps, flush):
    """steps factorizations, each bracketed by CUDA events on the library's
    stream (torch's current stream), with an L2 flush before each outside the
    events.  Returns (per-step ms, reports, last Z)."""
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    reps, Z = [], None
    for k in range(steps):
        flush.zero_()
        starts[k].record()
        Z, rep = factor(ctx, S, w["tau"], w["target"], o)
        ends[k].record()
        reps.append(rep)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(starts, ends)], reps, Z


SPLIT_PAIRS = 28  # slice pairs (s, t) with s + t <= 8 of the default 7-slice split product


def kernel_rooflines(reps, bs, prec, traffic=None):
    """Live CUDA-event rooflines of the block-product kernels.

    Work per kernel is the method's (2 bs^3 flops per multiplied stored block
    pair; zero blocks inside tiles are not counted; for the split kernel the
    tensor work is its BF16 slice products, s (s + 1) / 2 per block pair at
    s slices, and the FP64-equivalent rate is given beside it) and its
    algorithmic bytes as the library reports them (every operand block read
    once at the width the kernel reads it, every result block written once).
    The bound is the roofline that binds at that arithmetic intensity: HBM
    (measured copy bandwidth) below the ridge point, the tensor (TF32/BF16,
    split: BF16) or FP64 peak above it; both fractions are given.  `traffic` maps a kernel key to (DRAM bytes per launch, source)
    from an ncu capture of the same kernel and workload; kernels without one
    report null."""
    out = {}
    traffic = traffic or {}
    fl = 2.0 * bs ** 3
    hbm, hbm_src = hbm_peak_gbs()
    kinds = (("fp64", "gemm_ms", "fp64_pairs", "gemm_launches", "fp64_bytes", f"k_gemm_fp64<{bs}>"),
             ("tc", "tc_ms", "tc_pairs", "tc_launches", "tc_bytes", f"k_gemm_tc/k_gemm_band_lp<{'2' if prec == 'bf16' else '4'}>"),
             ("split", "split_ms", "split_pairs", "split_launches", "split_bytes", "k_gemm_split_band / k_gemm_tc<2> (split FP64)"))
    for key, ms_f, pairs_f, launch_f, bytes_f, kname in kinds:
        ms = sum(getattr(r, ms_f) for r in reps)
        if ms <= 0:
            continue
        launches = sum(getattr(r, launch_f) for r in reps)
        flops = sum(getattr(r, pairs_f) for r in reps) * fl
        fp64_equiv = flops / (ms / 1e3) / 1e12
        if key == "split":
            flops = sum(r.split_slice_pairs for r in reps) * fl
        nbytes = sum(getattr(r, bytes_f) for r in reps)
        tflops = flops / (ms / 1e3) / 1e12
        gbs = nbytes / (ms / 1e3) / 1e9
        if key == "fp64":
            cpk, csrc = fp64_peak_tflops()
            cbound, csrc = "alu", f"{csrc} bf16 x nominal FP64/BF16 ratio 1.25/2250"
        else:
            cp = "bf16" if key == "split" else prec
            cpk, csrc = tensor_peak_tflops(cp)
            cbound = "tensor"
            csrc = f"{csrc} bf16" + ("" if cp == "bf16" else " x nominal TF32/BF16 ratio 1.1/2.25")
        intensity = flops / max(nbytes, 1.0)
        ridge = cpk * 1e12 / (hbm * 1e9)
        mem_bound = intensity < ridge
        e = {"bound": "hbm" if mem_bound else cbound, "kernel": kname,
             "achieved": gbs if mem_bound else tflops, "peak": hbm if mem_bound else cpk,
             "unit": "GB/s" if mem_bound else "TFLOP/s",
             "frac": (gbs / hbm) if mem_bound else (tflops / cpk),
             "traffic": traffic[key][0] if key in traffic else None,
             "peak_source": hbm_src + " copy bandwidth" if mem_bound else csrc,
             "algorithmic_bytes_per_launch": nbytes / max(launches, 1),
             "flops_per_launch": flops / max(launches, 1),
             "intensity_flop_per_byte": intensity, "ridge_flop_per_byte": ridge,
             "hbm_gbs": gbs, "hbm_frac": gbs / hbm,
             "tflops": tflops, "compute_peak_tflops": cpk, "compute_frac": tflops / cpk,
             "launches_per_step": launches / len(reps), "avg_launch_us": 1e3 * ms / max(launches, 1),
             "ms_per_step": ms / len(reps)}
        if key == "split":
            e["slice_pairs_per_block_pair"] = sum(r.split_slice_pairs for r in reps) / max(
                sum(r.split_pairs for r in reps), 1)
            e["bf16_slice_tflops"] = tflops
            e["fp64_equivalent_tflops"] = fp64_equiv
            e["note"] = ("flops are the BF16 slice products (2 bs^3 per slice pair); fp64_equivalent_tflops "
                         "counts the FP64 product's 2 bs^3 per stored block pair")
        if e["traffic"] is not None:
            e["traffic_unit"] = "bytes per launch"
            e["traffic_source"] = traffic[key][1]
            e["traffic_over_algorithmic"] = e["traffic"] / max(e["algorithmic_bytes_per_launch"], 1.0)
        out[key] = e
    return out


def tc_dense_probe(ctx, ifac, nb=256):
    """Tensor-core kernel on a dense 16384 x 16384 BSR (64 x 64 blocks)
    product: events around the kernel (profiled refinement-free call)."""
    import torch
    from paper_1901_07993_gb300 import synth
    A = synth.random_bsr(nb, 64, 1.0, seed=1)
    dA = ifac.upload(ctx, A)
    res = {}
    for name, prec in (("bf16", 2), ("tf32", 1)):
        C = ifac.bsr_gemm_trunc(ctx, dA, False, dA, False, 1.0, 0.0, prec)
        del C
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
        e0.record()
        C = ifac.bsr_gemm_trunc(ctx, dA, False, dA, False, 1.0, 0.0, prec)
        e1.record()
        torch.cuda.synchronize()
        del C
        ms = e0.elapsed_time(e1)
        fl = 2.0 * (nb * 64) ** 3
        peak, _ = tensor_peak_tflops(name)
        res[name] = {"n": nb * 64, "ms_per_call": ms, "tflops_call": fl / ms / 1e9, "frac_of_peak": fl / ms / 1e9 / peak}
    return res


def batch_inputs(w):
    """Members of the batch workload: sizes log-uniform in [nmin, nmax] drawn
    with numpy PCG64 (seed), alternating chain and 3D cluster."""
    import numpy as np
    from paper_1901_07993_gb300 import synth
    rng = np.random.default_rng(w["seed"])
    sizes = np.exp(rng.uniform(np.log(w["nmin"]), np.log(w["nmax"]), size=w["count"])).astype(int)
    out = []
    for j, n in enumerate(sizes):
        if j % 2 == 0:
            out.append(synth.chain_overlap(int(n), w["bs"], seed=1000 * w["seed"] + j))
        else:
            out.append(synth.cluster_overlap(int(n), w["bs"], seed=1000 * w["seed"] + j))
    return out


def run_batched(args, w, world, rank, local, ctx, ifac):
    """One batched refinement of all members per step (inputs resident)."""
    import numpy as np
    import torch
    members = batch_inputs(w)
    dS = [ifac.upload(ctx, S) for S in members]
    ctx.set_split_slices(w.get("split_slices", 7))
    o = ifac.opts(m=w["m"], prec=PREC[w["prec"]], profile=True, max_iter=100)
    tune = None
    if w.get("autotune"):
        # block size and tile schedule from the library's timed probes (not
        # part of the timed steps); the members are re-blocked on the device
        t0 = time.perf_counter()
        tune = ifac.autotune_batched(ctx, dS, w["tau"], o)
        if tune["bs"] != w["bs"]:
            dS = [ifac.bsr_reblock(ctx, S, tune["bs"]) for S in dS]
        tune["seconds"] = time.perf_counter() - t0
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        Zs, reps, rc = ifac.inv_factor_refine_batched(ctx, dS, w["tau"], w["target"], o)
        del Zs
    torch.cuda.synchronize()
    ms, last = [], None
    barrier(world)
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(True), torch.cuda.Event(True)
            a.record()
            Zs, reps, rc = ifac.inv_factor_refine_batched(ctx, dS, w["tau"], w["target"], o)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
            last = reps
            del Zs
    barrier(world)
    total = allmax(world, sum(ms))
    r0 = last[0]
    kern = kernel_rooflines([last[0]], w["bs"], w["prec"])
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": world * args.steps / (total / 1e3), "unit": "batches/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[w["prec"]], "data": "synthetic",
            "config": {**config_of(w, args.workload, world), "count": w["count"],
                       "split_slices": w.get("split_slices", 7),
                       "sizes": [int(S.n) for S in members],
                       "bs_run": tune["bs"] if tune else w["bs"], "autotune": tune},
            "members": [{"n": int(S.n), "kind": "chain" if j % 2 == 0 else "cluster", "sweeps": r.sweeps,
                         "low_sweeps": r.low_sweeps, "fp64_delta_evals": r.fp64_delta_evals,
                         "resid_fro_fp64": r.resid_fro, "stop": r.stop_reason}
                        for j, (S, r) in enumerate(zip(members, last))],
            "resid_max": max(r.resid_fro for r in last),
            "resid_target_met": all(r.resid_fro <= w["target"] for r in last),
            "block_pairs": r0.block_pairs, "block_gemm_tflops": r0.flops / (total / args.steps / 1e3) / 1e12,
            "kernels": kern, "roofline": max(kern.values(), key=lambda v: v["ms_per_step"]) if kern else None,
            "gpu_launches": int(r0.launches * args.steps), "clocks": clk.summary()}), flush=True)


def run_table1(args, w, world, rank, local, ctx, ifac):
    """RINCH, LIF and IRSI with the paper's settings; one step = the three
    factorizations of both inputs.  Residuals ||I - Z^T S Z||_F (FP64)."""
    import torch
    from paper_1901_07993_gb300 import synth
    rows = []
    total_ms = 0.0
    for geom, n, switch in w["cases"]:
        S_h = synth.chain_overlap(n, w["bs"], seed=w["seed"]) if geom == "chain" else \
            synth.cluster_overlap(n, w["bs"], seed=w["seed"])
        S = ifac.upload(ctx, S_h)
        methods = {
            "RINCH": lambda: ifac.inv_factor_rinch(ctx, S, w["tau"], ifac.opts(leaf_size=128)),
            "LIF": lambda: ifac.inv_factor_localized(ctx, S, w["tau"], 0.0,
                                                     ifac.opts(m=w["m"], leaf_size=128, rinch_rows=switch)),
            "IRSI": lambda: ifac.inv_factor_refine(ctx, S, w["tau"], 0.0,
                                                   ifac.opts(m=w["m"], local_delta=True, max_iter=100)),
        }
        for name, f in methods.items():
            Z, rep = f()  # warm-up
            del Z
            ms = []
            for _ in range(max(1, args.steps)):
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
                e0.record()
                Z, rep = f()
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            r = ifac.inv_factor_resid(ctx, S, Z)
            total_ms += min(ms)
            rows.append({"input": f"{geom} n={n}", "method": name, "resid_fro": r, "ms": min(ms),
                         "sweeps": rep.sweeps, "levels": rep.levels, "nnzb_Z": rep.nnzb_Z})
            del Z
    if rank == 0:
        order = {}
        for inp in {r["input"] for r in rows}:
            rs = sorted((r for r in rows if r["input"] == inp), key=lambda r: r["resid_fro"])
            order[inp] = " < ".join(r["method"] for r in rs)
        print(json.dumps({
            "metric": "||I - Z^T S Z||_F of RINCH, LIF and IRSI at the paper's settings (Table 1)",
            "value": total_ms, "unit": "ms (sum of the six factorizations)", "n_gpus": world,
            "steps": args.steps, "warmup": 1, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "tau": w["tau"], "m": w["m"], "bs": w["bs"],
                       "cases": [list(c) for c in w["cases"]]},
            "results": rows, "error_order": order,
            "paper_order": "RINCH < LIF < IRSI (Glu-Ala and water clusters)"}), flush=True)


def run_adjoint(args, w, world, rank, local, ctx, ifac):
    """One adjoint evaluation (forward recording run + reverse pass) per step."""
    import torch
    from paper_1901_07993_gb300 import synth
    S_h = make_input(w)
    F_h = synth.fock_like(S_h, seed=w["fseed"])
    S, F = ifac.upload(ctx, S_h), ifac.upload(ctx, F_h)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        L, G = ifac.inv_factor_refine_adjoint(ctx, S, F, w["K"], w["tau"])
        del G
    torch.cuda.synchronize()
    ms = []
    barrier(world)
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(True), torch.cuda.Event(True)
            a.record()
            L, G = ifac.inv_factor_refine_adjoint(ctx, S, F, w["K"], w["tau"])
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
            del G
    barrier(world)
    total = allmax(world, sum(ms))
    if rank == 0:
        print(json.dumps({
            "metric": "adjoint dL/dS of 6 refinement sweeps (forward + reverse)", "value": world * args.steps / (total / 1e3),
            "unit": "gradients/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": {**config_of(w, args.workload, world), "K": w["K"]},
            "loss": L, "clocks": clk.summary()}), flush=True)


def run_product(args, w, world, rank, local, ctx, ifac):
    """One block-sparse product per step (dense pattern), CUDA events around the call."""
    import torch
    from paper_1901_07993_gb300 import synth
    nb = w["n"] // w["bs"]
    A = synth.random_bsr(nb, w["bs"], 1.0, seed=w["seed"])
    dA = ifac.upload(ctx, A)
    prec = PREC[w["prec"]]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        C = ifac.bsr_gemm_trunc(ctx, dA, False, dA, False, 1.0, 0.0, prec)
        del C
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier(world)
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            starts[k].record()
            C = ifac.bsr_gemm_trunc(ctx, dA, False, dA, False, 1.0, 0.0, prec)
            ends[k].record()
            del C
        torch.cuda.synchronize()
    barrier(world)
    ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    total = allmax(world, sum(ms))
    fl = 2.0 * w["n"] ** 3
    split = w["prec"] == "split"
    peak, src = tensor_peak_tflops("bf16" if split else w["prec"])
    ach = (SPLIT_PAIRS if split else 1) * fl / (sum(ms) / args.steps / 1e3) / 1e12
    extra = {"fp64_equivalent_tflops": ach / SPLIT_PAIRS,
             "note": f"achieved = {SPLIT_PAIRS} BF16 slice-pair products per block pair"} if split else {}
    if rank == 0:
        print(json.dumps({
            "metric": "block-sparse product TFLOP/s (dense pattern, tensor cores)", "value": world * args.steps / (total / 1e3),
            "unit": "products/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[w["prec"]], "data": "synthetic", "config": config_of(w, args.workload, world),
            "roofline": {"bound": "tensor", "kernel": "k_gemm_tc (whole bsr_gemm_trunc call)", "achieved": ach,
                         "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                         "peak_source": src, **extra}, "clocks": clk.summary()}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the comparison precisions, the end-to-end leg and the dense probe (profiling runs)")
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
    if w["method"] == "product":
        run_product(args, w, world, rank, local, ctx, ifac)
        return
    if w["method"] == "batched":
        run_batched(args, w, world, rank, local, ctx, ifac)
        return
    if w["method"] == "adjoint":
        run_adjoint(args, w, world, rank, local, ctx, ifac)
        return
    if w["method"] == "table1":
        run_table1(args, w, world, rank, local, ctx, ifac)
        return
    S_h = make_input(w)
    S = ifac.upload(ctx, S_h)
    if w.get("split_slices"):
        ctx.set_split_slices(w["split_slices"])
    if w["method"] == "rinch":
        def factor(ctx_, S_, tau, target, o_):
            return ifac.inv_factor_rinch(ctx_, S_, tau, o_)
    else:
        factor = ifac.inv_factor_refine if w["method"] == "refine" else ifac.inv_factor_localized
    o = ifac.opts(m=w["m"], leaf_size=w["leaf"], prec=PREC[w["prec"]], profile=True, max_iter=100,
                  rinch_rows=w.get("rinch_rows", 0))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):
        Z, rep = factor(ctx, S, w["tau"], w["target"], o)
        del Z
    torch.cuda.synchronize()

    # ---- device-resident timed region ----
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        step_ms, reps, Z = timed_factorizations(ctx, ifac, factor, S, w, o, args.steps, flush)
    barrier(world)
    torch.cuda.synchronize()
    total_ms = allmax(world, sum(step_ms))
    value = world * args.steps / (total_ms / 1e3)
    kernels = kernel_rooflines(reps, w["bs"], w["prec"], DRAM_TRAFFIC.get(args.workload))
    dominant = max(kernels, key=lambda k: kernels[k]["ms_per_step"]) if kernels else None
    roofline = dict(kernels[dominant]) if dominant else None
    resid = ifac.inv_factor_resid(ctx, S, Z)

    # ---- the same factorization in the comparison precisions ----
    compare = {}
    for cp in (() if args.no_compare else w["compare"]):
        oc = ifac.opts(m=w["m"], leaf_size=w["leaf"], prec=PREC[cp], profile=True, max_iter=100)
        Zc, _ = factor(ctx, S, w["tau"], w["target"], oc)  # warm-up
        del Zc
        ksteps = max(2, args.steps // 3)
        ms_c, reps_c, Zc = timed_factorizations(ctx, ifac, factor, S, w, oc, ksteps, flush)
        r = reps_c[-1]
        compare[cp] = {"value": world * ksteps / (allmax(world, sum(ms_c)) / 1e3), "unit": UNIT, "steps": ksteps,
                       "ms_per_step": sum(ms_c) / ksteps, "resid_fro": ifac.inv_factor_resid(ctx, S, Zc),
                       "sweeps": r.sweeps, "fp64_delta_evals": r.fp64_delta_evals, "low_sweeps": r.low_sweeps,
                       "delta_fro": r.delta_fro, "kernels": kernel_rooflines(reps_c, w["bs"], cp)}
        del Zc

    # ---- end to end through the C ABI with pinned host buffers ----
    def pinned(a):
        t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()

    S_pin = type(S_h)(S_h.n, S_h.bs, pinned(S_h.row_ptr), pinned(S_h.col_idx), pinned(S_h.val))
    o_e2e = ifac.opts(m=w["m"], leaf_size=w["leaf"], prec=PREC[w["prec"]], max_iter=100,
                      rinch_rows=w.get("rinch_rows", 0))
    z_bufs = None
    e2e_ms = []
    barrier(world)
    torch.cuda.synchronize()
    for k in range(0 if args.no_compare else args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Sd = ifac.upload(ctx, S_pin)
        Zd, rep_e = factor(ctx, Sd, w["tau"], w["target"], o_e2e)
        if z_bufs is None or z_bufs[1].shape[0] != rep_e.nnzb_Z:
            t_alloc = time.perf_counter()
            z_bufs = (pinned(np.zeros(S_h.nb + 1, np.int32)), pinned(np.zeros(rep_e.nnzb_Z, np.int32)),
                      pinned(np.zeros((rep_e.nnzb_Z, w["bs"], w["bs"]))))
            t0 += time.perf_counter() - t_alloc  # pinned-buffer allocation is not part of the step
        ctx.check(ctx.lib.ifac_bsr_download(ctx.h, Zd.ptr(), z_bufs[0].ctypes.data, z_bufs[1].ctypes.data,
                                            z_bufs[2].ctypes.data))
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        del Zd, Sd
    barrier(world)
    e2e_total = allmax(world, sum(e2e_ms))
    h2d = S_h.row_ptr.nbytes + S_h.col_idx.nbytes + S_h.val.nbytes
    d2h = sum(b.nbytes for b in z_bufs) if z_bufs else 0

    probe = tc_dense_probe(ctx, ifac) if w["prec"] != "fp64" and not args.no_compare else None
    clocks = clk.summary()
    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)
    r0 = reps[-1]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[w["prec"]],
        "data": "synthetic",
        "config": config_of(w, args.workload, world),
        "s_per_factorization": total_ms / args.steps / 1e3,
        "block_gemm_tflops": r0.flops / (total_ms / args.steps / 1e3) / 1e12,
        "resid_fro": resid, "resid_target_met": resid <= w["target"],
        "sweeps": r0.sweeps, "low_sweeps": r0.low_sweeps, "fp64_delta_evals": r0.fp64_delta_evals,
        "delta_fro": r0.delta_fro, "nnzb_Z": r0.nnzb_Z, "block_pairs": r0.block_pairs,
        "gpu_launches": int(sum(r.launches for r in reps)),
        "roofline": roofline, "kernels": kernels, "compare": compare, "tc_dense_probe": probe,
        "e2e": {"value": world * args.steps / (e2e_total / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h} if e2e_ms else None,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
