#!/usr/bin/env python3
"""Kernel K-means throughput on GB300: iterations/s of whole fits, plus K-build TFLOP/s.

One step = one complete ``popcorn_fit`` through the C ABI on the images workload
(n = 70,000 points, d = 784: integers 0..255 / 255 with 80% of each row zeroed,
an MNIST-shaped stand-in; k = 10, Gaussian kernel sigma = 28, random initial
labels, 50 fixed passes; K stored in FP32 as the block-packed upper triangle,
9.9 GB, far larger than L2, so every pass streams it from HBM).  A step runs
every row of the hot path: the K build (norms, Gram tiles, kernel epilogue),
then per pass the K-streaming segmented reduction (the symmetric pass: blocks on
and above the diagonal, row and column sums), the self-similarity sums, and the
distance/argmin/histogram pass.

``value`` is the plain FP32 form (CUDA-core K build).  The same line carries the
BF16X3 and BF16 forms (tensor-core K builds) and BF16X3 with K stored in FP16 (the
tensor-core symmetric pass) with their objective errors against the FP64 oracle, the
rooflines of the dominant kernels, and extra legs for the other workloads: rings
(n = 20,000, d = 8, to convergence), blobs (n = 2,000, 30 passes, L2-resident), the
256-instance batch (one CUDA graph; FP32 K, and BF16 K on the tensor cores) and the
n = 200,000 mixture on the recompute path (FP8 and BF16).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload images|rings|blobs|mixture|batched] [--precision P]
                    [--k-storage fp32|fp16|bf16] [--k-pass auto|full|symmetric] [--no-extras]

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same
workload (rank 0 only).  Under torchrun each rank runs an independent replica
(the workload is one problem; there is no data-path collective) and the
timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Kernel K-means iters/s + K-build TFLOP/s, FP32 vs BF16/batched at ≤1e-3 obj err"
WORKLOAD = "images"
WORKLOAD_DESC = ("images n=70000 d=784 k=10 (integers 0..255/255, 80% of each row zeroed), Gaussian sigma=28, "
                 "random init, 50 fixed passes, K stored FP32 (block-packed upper triangle)")
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
GB300_SMS = 152
FP32_LANES_PER_CLK_SM = 128          # FP32 FMA/ADD lanes per clock per SM
XU_EX2_PER_CLK_SM = 32               # ex2.approx per clock per SM (microbenchmark)
L2_INGEST_B_PER_CLK_SM = 36          # bytes per clock an SM takes in from L2 (microbenchmark)


def aggregate_over_ranks(times, counts, dist, device):
    """Whole-job figures of replicas run by every rank: the max of each time over
    ranks (the job ends with its slowest rank) and the sum of each count."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return [float(x) for x in times], [float(x) for x in counts]
    import torch

    t = torch.tensor([float(x) for x in times], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(x) for x in counts], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return t.tolist(), c.tolist()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing leg")
    ap.add_argument("--no-extras", action="store_true", help="skip the other workloads' legs")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink n (profiling captures only; the reported workload is scale 1)")
    ap.add_argument("--workload", default=WORKLOAD, choices=["images", "rings", "blobs", "mixture", "batched"],
                    help="images (default, the reported line), rings, blobs, mixture (recompute path), "
                         "batched (256 instances in one graph)")
    ap.add_argument("--autotune", default="on", choices=["on", "off"],
                    help="time candidate schedules in the warm-up (batched and recompute paths)")
    ap.add_argument("--precision", default=None, choices=["fp32", "bf16", "bf16x3", "fp8"],
                    help="K-build precision (default: the workload's)")
    ap.add_argument("--k-pass", default="auto", choices=["auto", "full", "symmetric"],
                    help="how a pass reads a stored FP32 K: the library's choice, the full square, or the blocks "
                         "on and above the diagonal (row and column sums, then a fold)")
    ap.add_argument("--k-storage", default="fp32", choices=["fp32", "fp16", "bf16"],
                    help="element type of the stored K (the build is FP32 or tensor-core; K is rounded once)")
    ap.add_argument("--sym-tile", type=int, default=0, choices=list(range(9)),
                    help="super-tile edge of the symmetric pass (0: the library's choice)")
    ap.add_argument("--sweep", default=None, choices=["kbuild"],
                    help="kbuild: the K build's GEMM-versus-SYRK sweep (n in {1e4, 5e4} x d in {1e2 .. 1e5}): the "
                         "symmetric and the full tile schedule of each precision, cuBLAS SGEMM / SSYRK run as "
                         "comparators, and the tuned choice")
    ap.add_argument("--compare", default=None, choices=["paper"],
                    help="paper: also time the paper's formulation through library calls (cuBLAS GEMM + "
                         "elementwise kernel function, cuSPARSE SpMM/SpMV per pass) on the same inputs")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    """The roofline denominators: measured HBM copy bandwidth and BF16 GEMM rate, else the fallbacks."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            m = json.load(f)
        return {"hbm": float(m["hbm_gbs"]), "bf16": float(m["bf16_tflops"]),
                "bf16_sustained": float(m.get("bf16_tflops_sustained", m["bf16_tflops"])),
                "sm_mhz": float(m.get("sm_max_mhz", 2070.0)), "source": "measured (MEASURED_PEAKS.json)"}
    except Exception:
        return {"hbm": FALLBACK_HBM_GBS, "bf16": FALLBACK_BF16_TFLOPS, "bf16_sustained": 1700.0, "sm_mhz": 2070.0,
                "source": "fallback (6.8 TB/s, 1.9 PFLOP/s bf16: an earlier GB300 measurement)"}


def recorded_traffic(kernel: str, src_file: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is unchanged."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)[kernel]
        if t.get("workload") != workload:
            return None
        with open(os.path.join(ROOT, "paper_2501_05587_gb300", "csrc", src_file), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
        if t.get("source_sha256") != sha:
            return None
        return float(t["dram_bytes_per_launch"])
    except Exception:
        return None


def sym_bytes(n: int, k: int, nslots: int, sorted_form: bool = True, ebytes: int = 4):
    """Bytes of one symmetric stream launch: the scope table's algorithmic figure for triangular
    storage (ebytes n (n + 1) / 2 + n: the unique entries of K once, 4 bytes an entry in FP32
    and 2 in FP16 / BF16, plus the labels), and what the kernel moves besides: the 128-blocks
    of the packed triangle, the slot stores, and per block its labels (branch form) or its
    column and row lists (sorted form: a 128-byte header and 4 bytes an entry, 128 + 3k
    padded to 4, plus 4; both from L2)."""
    T = (n + 127) // 128
    blocks = T * (T + 1) / 2
    lists = 2.0 * (128 + 4 * (((128 + 3 * k + 3) // 4) * 4 + 4))
    return {"algorithmic": ebytes * n * (n + 1) / 2.0 + n,
            "packed_tiles": 16384.0 * ebytes * blocks,
            "slot_stores": 4.0 * nslots * k * n,
            "labels": (lists if sorted_form else 256.0) * blocks}


def pass_roofline(wl, prof, pk, k_storage="fp32"):
    """HBM roofline of the dominant kernel of a pass (stored K): the symmetric stream or the
    full-square reduction.  Its launch time comes from the library's CUDA events on the
    launching stream (reduce minus fold), averaged over the profiled fits' passes."""
    n, k = wl.n, wl.k
    eb = 4 if k_storage == "fp32" else 2
    info = prof[-1]["info"]
    passes = sum(r["iterations"] for r in prof)
    red = sum(r["info"]["reduce_ms"] for r in prof)
    fold = sum(r["info"]["fold_ms"] for r in prof)
    if info["k_pass_used"] == 1:
        b = sym_bytes(n, k, info["schedule"][2], info["sym_form"] == 2, eb)
        if info["sym_form"] == 3:
            # one-hot operands of the block column and the block row with every block (L2)
            T = (n + 127) // 128
            b["labels"] = 2.0 * 256 * info["schedule"][3] * T * (T + 1) / 2
        ms = (red - fold) / max(passes, 1)
        ach = b["algorithmic"] / (ms / 1e3) / 1e9 if ms > 0 else 0.0
        # sym_form: 1 branch, 2 sorted, 3 tensor-core (the stream launch time of the last two
        # includes their per-pass label kernel: the sort, or the one-hot operand)
        kern = {1: "reduce_sym_kernel", 2: "reduce_sym_sorted_kernel", 3: "reduce_sym_mma_kernel"}[info["sym_form"]]
        return {"kernel": kern, "bound": "hbm", "achieved": ach, "peak": pk["hbm"], "unit": "GB/s",
                "frac": ach / pk["hbm"],
                "traffic": recorded_traffic(kern, "reduce_sym_mma.cu" if info["sym_form"] == 3 else "reduce_sym.cu",
                                            wl.name),
                "peak_source": pk["source"] + " HBM copy", "algorithmic_bytes_per_launch": b["algorithmic"],
                "moved_bytes_per_launch": {x: b[x] for x in ("packed_tiles", "slot_stores", "labels")},
                "k_storage": k_storage, "avg_launch_ms": ms, "fold_avg_launch_ms": fold / max(passes, 1),
                "pass_avg_ms": (red + sum(r["info"]["assign_ms"] for r in prof)) / max(passes, 1),
                "schedule": {"super_tile": info["schedule"][0], "ring": info["schedule"][1],
                             "slots": info["schedule"][2], "accumulators": info["schedule"][3]}}
    if info["k_pass_used"] == 3:
        # the whole fit in one launch (K in L2): a pass reads the full square from L2; the
        # ceiling is what the SMs can take in from L2, 36 bytes per clock per SM (measured
        # by stand-alone probes), and at this size the pass is mostly grid-barrier latency
        ms = sum(r["info"]["loop_ms"] for r in prof) / max(passes, 1)
        alg = 4.0 * n * n + n
        ach = alg / (ms / 1e3) / 1e9 if ms > 0 else 0.0
        peak = L2_INGEST_B_PER_CLK_SM * GB300_SMS * pk["sm_mhz"] * 1e6 / 1e9
        return {"kernel": "fit_fused_kernel", "bound": "l2", "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "traffic": None,
                "peak_source": f"{L2_INGEST_B_PER_CLK_SM} B/clk/SM L2 ingest (probe) x {GB300_SMS} SMs x "
                               f"{pk['sm_mhz']:.0f} MHz",
                "algorithmic_bytes_per_pass": alg, "pass_avg_ms": ms}
    ms = red / max(passes, 1)
    alg = float(eb) * n * n + n
    ach = alg / (ms / 1e3) / 1e9 if ms > 0 else 0.0
    # a half K read as the full square runs on the tensor cores (schedule[3]: its TMEM
    # columns); the launch time here also holds the one-hot operands and the z reduction
    kern = "batched_mma_kernel" if eb == 2 and info["schedule"][3] > 0 else "reduce_kernel"
    return {"kernel": kern, "bound": "hbm", "k_storage": k_storage, "achieved": ach, "peak": pk["hbm"], "unit": "GB/s",
            "frac": ach / pk["hbm"],
            "traffic": recorded_traffic("reduce_kernel", "iterate.cu", wl.name) if kern == "reduce_kernel" else None,
            "peak_source": pk["source"] + " HBM copy", "algorithmic_bytes_per_launch": alg, "avg_launch_ms": ms}


def kbuild_roofline(wl, precision, kb_ms, pk, k_storage="fp32"):
    """Roofline of the K build.  FP32 (CUDA cores): bound by the FP32 lanes -- a Gaussian entry
    takes a subtract and a multiply-add per coordinate, a polynomial / linear one a multiply-add,
    over the n (n + 1) / 2 unique pairs; peak = 128 lanes x 152 SMs x the maximum SM clock.
    BF16 / BF16X3 (tcgen05): the executed MMA flops of the row-pair tiles (BF16X3: three
    products per k-step) against the measured BF16 peak."""
    n, d = float(wl.n), float(wl.d)
    sec = kb_ms / 1e3
    if precision == "fp32":
        # the Gaussian's distance form, decided as the library decides it: the norm expansion
        # (one multiply-add a coordinate) when 4 sqrt(d) u max_i r_i gamma / sigma^2 <= 1e-6,
        # else coordinate differences (a subtract and a multiply-add)
        form = None
        per = 1.0
        if wl.kernel["kind"] == "gaussian":
            maxr = float((wl.P.astype(np.float64) ** 2).sum(axis=1).max())
            c = float(wl.kernel.get("gamma", 1.0)) / float(wl.kernel["sigma"]) ** 2
            expand = 4.0 * np.sqrt(d) * 2.0 ** -24 * maxr * c <= 1e-6
            form = "norm expansion (Eq. 12)" if expand else "coordinate differences"
            per = 1.0 if expand else 2.0
        ops = per * n * (n + 1) / 2 * d
        peak = FP32_LANES_PER_CLK_SM * GB300_SMS * pk["sm_mhz"] * 1e6 / 1e12
        ach = ops / sec / 1e12
        # d > 16 with a dot-product form (linear, polynomial, Gaussian by the norm expansion)
        # runs the 16 x 8 f32x2 tile; coordinate differences and d <= 16 the other kernels
        kern = "kbuild_dot_kernel" if wl.d > 16 and per == 1.0 else "kbuild_simt_kernel"
        return {"kernel": kern, "bound": "alu", "achieved": ach, "peak": peak, "unit": "Tlane-ops/s",
                "frac": ach / peak, "traffic": recorded_traffic(kern, "kbuild_simt.cu", wl.name),
                "peak_source": f"{FP32_LANES_PER_CLK_SM} FP32 lanes/clk/SM x {GB300_SMS} SMs x "
                               f"{pk['sm_mhz']:.0f} MHz (unit counts and clock)",
                "algorithmic_lane_ops_per_launch": ops, "avg_launch_ms": kb_ms, "distance_form": form}
    T = (wl.n + 127) // 128
    T2 = (T + 1) // 2
    tiles = T2 * T - T2 * (T2 - 1)
    dpad = (wl.d + 63) // 64 * 64
    depth = dpad * (3 if precision == "bf16x3" else 1)
    flops = tiles * 2.0 * 128 * 128 * 2.0 * depth
    ach = flops / sec / 1e12
    return {"kernel": "kbuild_tc_kernel", "bound": "tensor", "achieved": ach, "peak": pk["bf16"], "unit": "TFLOP/s",
            "frac": ach / pk["bf16"],
            "traffic": (recorded_traffic("kbuild_tc_kernel" + ("" if k_storage == "fp32" else f"[{k_storage} K]"),
                                         "kbuild_tc.cu", wl.name) if precision == "bf16x3" else None),
            "k_storage": k_storage,
            "peak_source": pk["source"] + " bf16 burst",
            "executed_mma_flops_per_launch": flops, "avg_launch_ms": kb_ms}


def recompute_rooflines(wl, avg_ms: float, pk):
    """Rooflines of one recompute pass (sort + tiles + reduction), the binding one first.

    tensor: 2 n^2 d algorithmic MMA flops against the measured BF16 burst peak (FP8:
    twice that, the nominal FP8/BF16 ratio); alu: n^2 exp2 evaluations (Gaussian)
    against 32 per clock per SM at the maximum SM clock."""
    peak_t = pk["bf16"] * (2.0 if wl.precision == "fp8" else 1.0)
    n, d = float(wl.n), float(wl.d)
    sec = avg_ms / 1e3 if avg_ms > 0 else float("inf")
    t_ach = 2.0 * n * n * d / sec / 1e12
    tensor = {"kernel": "recompute_kernel", "bound": "tensor", "achieved": t_ach, "peak": peak_t,
              "unit": "TFLOP/s", "frac": t_ach / peak_t, "traffic": None,
              "peak_source": pk["source"] + " bf16 burst" + (" x2 for FP8 (nominal ratio)" if wl.precision == "fp8"
                                                             else ""),
              "algorithmic_flops_per_launch": 2.0 * n * n * d, "avg_launch_ms": avg_ms}
    peak_x = XU_EX2_PER_CLK_SM * GB300_SMS * pk["sm_mhz"] * 1e6 / 1e12
    x_ach = n * n / sec / 1e12
    alu = {"kernel": "recompute_kernel", "bound": "alu", "achieved": x_ach, "peak": peak_x,
           "unit": "Texp2/s", "frac": x_ach / peak_x, "traffic": None,
           "peak_source": f"{XU_EX2_PER_CLK_SM} ex2/clk/SM x {GB300_SMS} SMs x {pk['sm_mhz']:.0f} MHz (ex2 microbenchmark)",
           "algorithmic_exp2_per_launch": n * n, "avg_launch_ms": avg_ms}
    if wl.kernel["kind"] != "gaussian":
        return tensor, None
    return (tensor, alu) if tensor["frac"] >= alu["frac"] else (alu, tensor)


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 100 ms during the timed region."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, f".clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.gpu)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return None
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
            os.remove(self.path)
        except Exception:
            return None
        sm, smax, reasons = [], 0.0, set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax = max(smax, float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], r[5:9]):
                if v.lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_cores():
    try:
        from threadpoolctl import threadpool_info
        n = max((int(i.get("num_threads", 1)) for i in threadpool_info()), default=1)
        return n
    except Exception:
        return os.cpu_count() or 1


def oracle_fit_sample(wl, n_sample: int):
    """The FP64 oracle as it stands on the first n_sample points of the workload: K build,
    then the workload's passes from its initial labels.  Returns (K, fit, build s, loop s)."""
    import oracle

    P = wl.P[:n_sample]
    lab = wl.init_labels[:n_sample].copy()
    t0 = time.perf_counter()
    K = oracle.kernel_matrix(P, wl.kernel)
    t_build = time.perf_counter() - t0
    t1 = time.perf_counter()
    fit = oracle.fit(K, wl.k, lab, wl.max_iter, check_convergence=wl.check_convergence)
    t_loop = time.perf_counter() - t1
    return K, fit, t_build, t_loop


def cpu_baseline(wl, n_sample: int):
    """Oracle K build + passes on a bounded sample, its whole-fit rate scaled to the full
    workload by (n_sample / n)^2 (both the build and each pass scale with n^2)."""
    K, fit, t_build, t_loop = oracle_fit_sample(wl, n_sample)
    scale = (n_sample / wl.n) ** 2
    it_s = fit["iterations"] / (t_build + t_loop) * scale
    base = {"value": it_s, "unit": "iters/s", "cores": oracle_cores(), "kind": "oracle",
            "sample": (f"first {n_sample} of {wl.n} points: FP64 oracle K build ({t_build:.2f} s) + "
                       f"{fit['iterations']} passes ({t_loop:.2f} s); whole-fit rate scaled by (n_sample/n)^2 = "
                       f"{scale:.3g} to the full workload")}
    return base, K, fit


SAMPLE = {"images": 2500, "rings": 12000, "blobs": 2000, "mixture": 6000}
REF_SAMPLE = {"images": 1200, "rings": 8000, "blobs": 2000, "mixture": 3000}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import synth

    wl = synth.workload(args.workload if args.workload != "batched" else WORKLOAD)
    n_s = REF_SAMPLE.get(wl.name.split("_")[0], 1500)
    for _ in range(args.warmup):
        oracle_fit_sample(wl, max(n_s // 2, 16))
    t_all = 0.0
    passes_all = 0
    for _ in range(args.steps):
        _, fit, tb, tl = oracle_fit_sample(wl, n_s)
        t_all += tb + tl
        passes_all += fit["iterations"]
    scale = (n_s / wl.n) ** 2
    value = passes_all / t_all * scale
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC if wl.name.startswith("images") else wl.name,
                       "n": wl.n, "d": wl.d, "k": wl.k},
            "cpu_baseline": {"value": value, "unit": "iters/s", "cores": oracle_cores(), "kind": "oracle",
                             "sample": (f"each step: FP64 oracle K build + {wl.max_iter} passes on the first "
                                        f"{n_s} points; whole-fit rate scaled by (n_sample/n)^2 = {scale:.3g}")},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def timed(torch, stream, fn, steps, warmup):
    """warmup untimed calls, then `steps` calls between CUDA events on `stream` (synchronized
    on both sides); returns (ms, results)."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = [fn() for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), res


def fit_form(pc, torch, stream, wl, P, lab, out, precision, steps, warmup, **kw):
    """One precision form of the workload: timed fits (no library events), then the same fits
    with the library's per-kernel events (the breakdown and the kernels' launch times)."""
    def step(timing=False):
        return pc.popcorn_fit(P, wl.k, wl.kernel, lab, max_iter=wl.max_iter, check_convergence=wl.check_convergence,
                              precision=precision, timing=timing, labels_out=out, store_k=wl.store_k, **kw)

    ms, res = timed(torch, stream, step, steps, warmup)
    prof = [step(True) for _ in range(steps)]
    torch.cuda.synchronize()
    iters = sum(r["iterations"] for r in res)
    kb_ms = sum(r["info"]["kbuild_ms"] for r in prof) / len(prof)
    red = sum(r["info"]["reduce_ms"] for r in prof) / len(prof)
    asg = sum(r["info"]["assign_ms"] for r in prof) / len(prof)
    n, d = wl.n, wl.d
    return {"ms": ms, "res": res, "prof": prof, "iters": iters,
            "summary": {"value": iters / (ms / 1e3), "unit": "iters/s", "ms_per_fit": ms / steps,
                        "passes_per_fit": iters / steps, "objective": res[-1]["objective"],
                        "kbuild_ms": kb_ms,
                        "kbuild_tflops": float(n) * (n + 1) * d / (kb_ms / 1e3) / 1e12 if kb_ms > 0 else None,
                        "kbuild_tflops_gemm_equivalent": 2.0 * n * n * d / (kb_ms / 1e3) / 1e12 if kb_ms > 0 else None,
                        "breakdown_ms_per_fit": {"kbuild": kb_ms, "reduce": red, "assign": asg},
                        "k_pass": {0: "recompute", 1: "symmetric", 2: "full", 3: "fused fit (full square, one launch)"}[
                            prof[-1]["info"]["k_pass_used"]],
                        "gpu_launches_per_fit": res[-1]["info"]["kernel_launches"]}}


def graph_us_per_pass(pc, torch, wl, P, lab, out, precision, steps, **kw):
    """Fixed-iteration fits with phase events only: the passes run as one CUDA graph, and
    loop_ms is that graph's time (every pass plus the objective pass)."""
    res = [pc.popcorn_fit(P, wl.k, wl.kernel, lab, max_iter=wl.max_iter, check_convergence=False,
                          precision=precision, timing="phases", labels_out=out, store_k=wl.store_k, **kw)
           for _ in range(steps)]
    torch.cuda.synchronize()
    return 1e3 * sum(r["info"]["loop_ms"] for r in res) / sum(r["iterations"] for r in res)


def leg_workload(pc, torch, stream, name, steps, warmup, pk, **kw):
    """An extra workload leg: its default form, timed like the headline."""
    import synth

    wl = synth.workload(name)
    P = torch.from_numpy(wl.P).cuda()
    lab = torch.from_numpy(wl.init_labels).cuda()
    out = torch.empty_like(lab)
    f = fit_form(pc, torch, stream, wl, P, lab, out, wl.precision, steps, warmup, **kw)
    s = f["summary"]
    s["workload"] = wl.name
    if wl.store_k:
        s["roofline_pass"] = pass_roofline(wl, f["prof"], pk)
        loop = sum(r["info"]["loop_ms"] for r in f["prof"]) / len(f["prof"])
        s["loop_us_per_pass_plain_launches"] = 1e3 * loop / max(s["passes_per_fit"], 1)
        if not wl.check_convergence:
            s["loop_us_per_pass_graph"] = graph_us_per_pass(pc, torch, wl, P, lab, out, wl.precision, steps, **kw)
    else:
        avg = sum(r["info"]["reduce_ms"] for r in f["prof"]) / max(1, sum(r["iterations"] for r in f["prof"]))
        s["pass_ms"] = avg
        s["roofline_pass"], s["roofline_pass_secondary"] = recompute_rooflines(wl, avg, pk)
        s["schedule"] = f["prof"][-1]["info"]["schedule"]
    return s, wl, f


def leg_batched(pc, torch, stream, steps, warmup, precision, autotune, scale=1.0, k_storage="fp32"):
    """256 independent instances (n in [500, 8000], d in {8, 32, 64}, k in [4, 64], polynomial and
    Gaussian kernels), 30 passes each, one popcorn_fit_batched call (one CUDA graph) per step."""
    import synth

    wls = synth.batched_instances(int(256 * scale) or 1, seed=0)
    insts = [{"P": torch.from_numpy(w.P).cuda(), "k": w.k, "kernel": w.kernel,
              "init_labels": torch.from_numpy(w.init_labels).cuda()} for w in wls]

    def step():
        return pc.popcorn_fit_batched(insts, max_iter=30, precision=precision, check_convergence=False, timing=True,
                                      autotune=autotune, k_storage=k_storage)

    ms, res = timed(torch, stream, step, steps, warmup)
    passes = sum(sum(r["iterations"]) for r in res)
    kbytes = sum((4.0 if k_storage == "fp32" else 2.0) * w.n * w.n for w in wls)
    graph_ms = sum(r["info"]["loop_ms"] for r in res) / len(res)
    # the same instances as separate fits (a half K from a tensor-core build exists only for the
    # symmetric pass's k <= 32, so that pairing has no separate-fit counterpart for every instance)
    seq_ms = None
    if k_storage == "fp32" or precision == "fp32":
        e2 = torch.cuda.Event(enable_timing=True)
        e3 = torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        for x in insts:
            pc.popcorn_fit(x["P"], x["k"], x["kernel"], x["init_labels"], max_iter=30, precision=precision,
                           check_convergence=False, k_storage=k_storage)
        e3.record(stream)
        torch.cuda.synchronize()
        seq_ms = e2.elapsed_time(e3)
    return {"value": passes / (ms / 1e3), "unit": "instance-passes/s", "ms_per_step": ms / steps,
            "precision": precision, "k_storage": k_storage, "instances": len(wls), "K_GB": kbytes / 1e9,
            "_objectives": res[-1]["objectives"],
            "_labels": [x.cpu().numpy() for x in res[-1]["labels"]],
            "graph_ms": graph_ms, "effective_GBps_of_K_reads": kbytes * 30 / (graph_ms / 1e3) / 1e9,
            "separate_fits_ms": seq_ms,
            "batched_speedup_vs_separate_fits": seq_ms / (ms / steps) if seq_ms else None,
            "gpu_launches_per_step": res[-1]["info"]["kernel_launches"],
            "schedule": {"autotune": autotune, "columns_per_unit": res[-1]["info"]["schedule"][0],
                         "warps_per_block": res[-1]["info"]["schedule"][1],
                         "blocks_per_sm": res[-1]["info"]["schedule"][2]}}


def run_batched(args):
    import torch

    import paper_2501_05587_gb300 as pc

    prec = args.precision or "fp32"
    stream = torch.cuda.current_stream()
    s = leg_batched(pc, torch, stream, args.steps, args.warmup, prec, args.autotune == "on", args.scale,
                    k_storage=args.k_storage)
    s.pop("_objectives", None)
    s.pop("_labels", None)
    line = {"metric": METRIC, "value": s["value"], "unit": s["unit"], "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": s["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": {"workload": f"batched: {s['instances']} instances, 30 passes each, K stored "
                                   f"{args.k_storage.upper()} ({s['K_GB']:.1f} GB)", "precision": prec},
            "gpu_launches": s["gpu_launches_per_step"] * args.steps, "batched": s}
    print(json.dumps(line), flush=True)
    return 0


def sample_objective_errors(pc, torch, wl, Ko, ofit, n_sample, forms):
    """GPU fits of each precision form on the oracle's sample (same points, same initial labels,
    same passes): the FP64 objective of their labels against the objective the oracle's fit
    reaches, and the reported objective against the FP64 objective of the same labels."""
    import oracle

    P = torch.from_numpy(np.ascontiguousarray(wl.P[:n_sample])).cuda()
    lab = torch.from_numpy(np.ascontiguousarray(wl.init_labels[:n_sample])).cuda()
    out = {}
    for form in forms:
        key, prec, kst = form if isinstance(form, tuple) else (form, form, "fp32")
        r = pc.popcorn_fit(P, wl.k, wl.kernel, lab, max_iter=wl.max_iter, check_convergence=wl.check_convergence,
                           precision=prec, store_k=wl.store_k, k_storage=kst)
        labels = r["labels"].cpu().numpy()
        J = oracle.objective(Ko, labels, wl.k)
        out[key] = {"objective_rel_err_vs_oracle_fit": abs(J - ofit["objective"]) / abs(ofit["objective"]),
                     "reported_vs_fp64_of_labels": abs(r["objective"] - J) / abs(J),
                     "labels_equal_to_oracle_fit": float(np.mean(labels == ofit["labels"]))}
    return out


def run_paper_pipeline(args):
    """The paper's formulation on the same GPU, through library calls only (a comparator:
    none of this is on the library's path).

    K build (Sec. 3.2, Alg. 2 lines 1-2): B = P P^T by a cuBLAS GEMM (torch.matmul; FP32 with
    TF32 off, or BF16 operands for --precision bf16), then the kernel function as elementwise
    passes.  Each pass (Alg. 2 lines 7-14): V (k x n, CSR, V_cj = 1/|L_c|) times K by a
    cuSPARSE SpMM, the gather e_i = (V K)_{cl(i), i}, z = V e by a cuSPARSE SpMV (Eq. 14),
    D = diag(K) - 2 (V K)^T + z, the row argmin and the new counts.  Same inputs and number of
    passes as one popcorn_fit of the same workload; one JSON line with both."""
    import torch

    import synth
    import paper_2501_05587_gb300 as pc

    torch.backends.cuda.matmul.allow_tf32 = False
    wl = synth.workload(args.workload, scale=args.scale)
    prec = args.precision or wl.precision
    if prec not in ("fp32", "bf16") or not wl.store_k:
        print(json.dumps({"compare": "paper", "unavailable": "the comparator covers stored-K FP32/BF16 fits"}))
        return 0
    P = torch.from_numpy(wl.P).cuda()
    lab0 = torch.from_numpy(wl.init_labels).cuda()
    n, k = wl.n, wl.k
    kern = wl.kernel
    # ours first: the pass count the paper pipeline then runs
    ours = pc.popcorn_fit(P, k, kern, lab0, max_iter=wl.max_iter, check_convergence=wl.check_convergence,
                          precision=prec, timing=True)
    passes = int(ours["iterations"])
    for _ in range(max(args.warmup - 1, 0)):
        pc.popcorn_fit(P, k, kern, lab0, max_iter=passes, check_convergence=False, precision=prec, timing=True)
    torch.cuda.synchronize()
    o0, o1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    o0.record()
    ours = pc.popcorn_fit(P, k, kern, lab0, max_iter=passes, check_convergence=False, precision=prec, timing=True)
    o1.record()
    torch.cuda.synchronize()
    ours_ms = o0.elapsed_time(o1)

    def kbuild():
        if prec == "bf16":
            Pb = P.to(torch.bfloat16)
            K = (Pb @ Pb.T).float()
            r = (Pb.float() * Pb.float()).sum(1)
        else:
            K = P @ P.T
            r = (P * P).sum(1)
        if kern["kind"] == "gaussian":
            K.mul_(-2.0).add_(r[:, None]).add_(r[None, :]).clamp_min_(0.0)
            K.mul_(-kern["gamma"] / (kern["sigma"] ** 2)).exp_()
            K.fill_diagonal_(1.0)
        elif kern["kind"] == "polynomial":
            K.mul_(kern["gamma"]).add_(kern["coef0"]).pow_(kern["degree"])
        return K

    ar = torch.arange(n, device="cuda")

    def one_pass(K, kd, labels):
        counts = torch.bincount(labels, minlength=k)
        inv = torch.where(counts > 0, 1.0 / counts.clamp_min(1).float(), torch.zeros_like(counts, dtype=torch.float32))
        order = torch.argsort(labels, stable=True)
        crow = torch.zeros(k + 1, dtype=torch.int64, device="cuda")
        crow[1:] = torch.cumsum(counts, 0)
        V = torch.sparse_csr_tensor(crow, order, inv[labels[order]], size=(k, n))
        VK = torch.sparse.mm(V, K)                             # SpMM: (K V^T)^T
        e = VK[labels, ar]                                      # gather
        z = torch.sparse.mm(V, e[:, None]).squeeze(1)           # SpMV: z_c = ||c_c||^2
        D = kd[:, None] - 2.0 * VK.T + z[None, :]
        D[:, counts == 0] = float("inf")
        return D.argmin(1), D

    def fit():
        K = kbuild()
        kd = torch.diagonal(K).clone()
        labels = lab0.long()
        for _ in range(passes):
            labels, D = one_pass(K, kd, labels)
        return K, kd, labels

    for _ in range(args.warmup):
        fit()
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record()
    K = kbuild()
    e1.record()
    kd = torch.diagonal(K).clone()
    labels = lab0.long()
    for _ in range(passes):
        labels, D = one_pass(K, kd, labels)
    e2.record()
    torch.cuda.synchronize()
    kb_ms, loop_ms = e0.elapsed_time(e1), e1.elapsed_time(e2)
    # objective of the final labels, as Alg. 2 defines it: sum_i D_{i, cl(i)} with the last centroids
    _, D = one_pass(K, kd, labels)
    J_paper = float(D[ar, labels].double().sum())
    same = float((labels.int() == ours["labels"]).float().mean())
    line = {"compare": "paper", "workload": wl.name, "precision": prec, "n": n, "d": wl.d, "k": k,
            "passes": passes,
            "paper_pipeline": {"kbuild_ms": kb_ms, "loop_ms": loop_ms, "iters_per_s": passes / ((kb_ms + loop_ms) / 1e3),
                               "per_pass_ms": loop_ms / passes,
                               "kbuild_tflops_gemm": 2.0 * n * n * wl.d / (kb_ms / 1e3) / 1e12,
                               "libraries": "cuBLAS GEMM (torch.matmul), cuSPARSE SpMM/SpMV (torch.sparse CSR)"},
            "ours": {"kbuild_ms": ours["info"]["kbuild_ms"], "loop_ms": ours["info"]["loop_ms"],
                     "iters_per_s": passes / (ours_ms / 1e3),
                     "per_pass_ms": ours["info"]["loop_ms"] / passes},
            "speedup_whole_fit": ((kb_ms + loop_ms) / ours_ms),
            "speedup_per_pass": (loop_ms / passes) / (ours["info"]["loop_ms"] / passes),
            "labels_equal_fraction": same,
            "objective_ours": ours["objective"], "objective_paper_pipeline": J_paper}
    print(json.dumps(line), flush=True)
    return 0


def _cublas():
    """ctypes handle on the cuBLAS library torch has loaded (found through the process's maps)."""
    import ctypes

    try:
        with open("/proc/self/maps") as f:
            paths = {line.split()[-1] for line in f if "libcublas.so" in line and "Lt" not in line}
        for path in sorted(paths):
            lib = ctypes.CDLL(path)
            if hasattr(lib, "cublasSsyrk_v2"):
                return lib
    except Exception:
        pass
    return None


def run_sweep_kbuild(args):
    """The paper's GEMM-versus-SYRK experiment (Sec. 5.2: n in {1e4, 5e4}, d in {1e2, 1e3, 1e4,
    1e5}; Sec. 4.2's rule: GEMM when n / d > 100) re-run on this GPU.  B = P P^T (linear kernel,
    P uniform in [0, 1), seeded on the device).  Ours: popcorn_kernel_matrix_ex in each precision
    with the symmetric schedule (tiles on and above the diagonal, stored with their transposes:
    the SYRK form) and the full schedule (every tile: the GEMM form), then the tuned choice
    (schedule "tune": both timed, the faster cached).  Comparators, library calls only: cuBLAS
    SGEMM (torch.mm, TF32 off) and cuBLAS SSYRK (ctypes), FP32 as in the paper."""
    import ctypes

    import torch

    import paper_2501_05587_gb300 as pc

    torch.backends.cuda.matmul.allow_tf32 = False
    stream = torch.cuda.current_stream()
    lin = {"kind": "linear", "gamma": 1.0, "coef0": 0.0, "degree": 1, "sigma": 1.0}
    ns = [int(x) for x in os.environ.get("SWEEP_N", "10000,50000").split(",")]
    ds = [int(x) for x in os.environ.get("SWEEP_D", "100,1000,10000,100000").split(",")]

    def clock(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if ms < 1000.0:   # short: best of three more
            for _ in range(3):
                e0.record(stream)
                fn()
                e1.record(stream)
                torch.cuda.synchronize()
                ms = min(ms, e0.elapsed_time(e1))
        return ms

    torch.mm(torch.ones(8, 8, device="cuda"), torch.ones(8, 8, device="cuda"))
    torch.cuda.synchronize()
    cublas = _cublas()
    rows = []
    for n in ns:
        for d in ds:
            g = torch.Generator(device="cuda")
            g.manual_seed(1000003 * n + d)
            P = torch.rand((n, d), generator=g, device="cuda", dtype=torch.float32)
            ldk = (n + 3) // 4 * 4
            Kb = torch.empty((n, ldk), dtype=torch.float32, device="cuda")
            K = Kb[:, :n]
            kd = torch.empty(n, dtype=torch.float32, device="cuda")
            gemm_flops, alg_flops = 2.0 * n * n * d, float(n) * (n + 1) * d
            row = {"n": n, "d": d, "n_over_d": n / d,
                   "paper_rule": "gemm" if n / d > 100 else "syrk", "ms": {}}
            for prec in ("fp32", "bf16x3", "bf16"):
                for sched in ("symmetric", "full"):
                    row["ms"][f"ours_{prec}_{sched}"] = clock(
                        lambda: pc.popcorn_kernel_matrix(P, lin, prec, K, kd, schedule=sched))
                pc.popcorn_kernel_matrix(P, lin, prec, K, kd, schedule="tune")
                row.setdefault("tuned", {})[prec] = ("full" if row["ms"][f"ours_{prec}_full"] <
                                                     row["ms"][f"ours_{prec}_symmetric"] else "symmetric")
            del Kb, K
            C = torch.empty((n, n), dtype=torch.float32, device="cuda")
            row["ms"]["cublas_sgemm"] = clock(lambda: torch.mm(P, P.T, out=C))
            if cublas is not None:
                handle = ctypes.c_void_p(torch.cuda.current_blas_handle())
                cublas.cublasSetStream_v2(handle, ctypes.c_void_p(stream.cuda_stream))
                alpha, beta = ctypes.c_float(1.0), ctypes.c_float(0.0)

                def syrk():
                    # row-major P (n x d) is the column-major d x n matrix A: C = A^T A (upper)
                    st = cublas.cublasSsyrk_v2(handle, 1, 1, n, d, ctypes.byref(alpha), ctypes.c_void_p(P.data_ptr()),
                                               d, ctypes.byref(beta), ctypes.c_void_p(C.data_ptr()), n)
                    if st != 0:
                        raise RuntimeError(f"cublasSsyrk_v2 returned {st}")
                row["ms"]["cublas_ssyrk"] = clock(syrk)
            del C, P
            torch.cuda.empty_cache()
            row["gemm_equivalent_tflops"] = {k: gemm_flops / (v / 1e3) / 1e12 for k, v in row["ms"].items()}
            row["algorithmic_tflops"] = {k: alg_flops / (v / 1e3) / 1e12 for k, v in row["ms"].items()}
            row["full_over_symmetric"] = {p_: row["ms"][f"ours_{p_}_full"] / row["ms"][f"ours_{p_}_symmetric"]
                                          for p_ in ("fp32", "bf16x3", "bf16")}
            if "cublas_ssyrk" in row["ms"]:
                row["cublas_sgemm_over_ssyrk"] = row["ms"]["cublas_sgemm"] / row["ms"]["cublas_ssyrk"]
            rows.append(row)
            print(json.dumps({"sweep": "kbuild", **row}), flush=True)
    print(json.dumps({"sweep": "kbuild", "points": len(rows), "cublas_ssyrk": cublas is not None}), flush=True)
    return 0


def main():
    args = parse()
    if args.compare == "paper":
        return run_paper_pipeline(args)
    if args.sweep == "kbuild":
        return run_sweep_kbuild(args)
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batched":
        return run_batched(args)

    import torch

    import synth
    import paper_2501_05587_gb300 as pc

    assert args.warmup >= 3, "at least 3 warm-up steps"
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    pk = peaks()
    wl = synth.workload(args.workload, scale=args.scale)
    if args.precision:
        wl.precision = args.precision
    headline = args.workload == WORKLOAD and args.scale == 1.0 and not args.precision and args.k_storage == "fp32"
    P = torch.from_numpy(wl.P).cuda()
    lab = torch.from_numpy(wl.init_labels).cuda()
    out = torch.empty_like(lab)
    # the recompute path's schedule (row blocks per tile, units per SM) is autotuned in the warm-up
    kw = {"autotune": args.autotune == "on" and not wl.store_k, "k_pass": args.k_pass, "sym_tile": args.sym_tile,
          "k_storage": args.k_storage}

    stream = torch.cuda.current_stream()
    with ClockSampler(local) as clocks:
        barrier()
        torch.cuda.synchronize()
        main_form = fit_form(pc, torch, stream, wl, P, lab, out, wl.precision, args.steps, args.warmup, **kw)
        torch.cuda.synchronize()
        barrier()
    clk = clocks.summary()
    ms, iters = main_form["ms"], main_form["iters"]
    launches = sum(r["info"]["kernel_launches"] for r in main_form["res"])

    # end to end through the same call with pinned host buffers (copies inside the timed region)
    Ph = torch.from_numpy(wl.P).pin_memory()
    Lh = torch.from_numpy(wl.init_labels).pin_memory()
    Oh = torch.empty(wl.n, dtype=torch.int32).pin_memory()

    def host_step():
        return pc.popcorn_fit(Ph, wl.k, wl.kernel, Lh, max_iter=wl.max_iter, check_convergence=wl.check_convergence,
                              precision=wl.precision, labels_out=Oh, store_k=wl.store_k, **kw)

    for _ in range(args.warmup):
        host_step()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_res = [host_step() for _ in range(args.steps)]
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    barrier()

    (ms, t_e2e), (iters_all, e2e_iters_all, launches_all) = aggregate_over_ranks(
        [ms, t_e2e], [iters, sum(r["iterations"] for r in e2e_res), launches], dist, "cuda")
    launches_all = int(launches_all)

    if rank == 0:
        n, k = wl.n, wl.k
        value = iters_all / (ms / 1e3)
        s = main_form["summary"]
        prof = main_form["prof"]
        kb_ms = s["kbuild_ms"]
        rooflines = []
        if wl.store_k:
            rp = pass_roofline(wl, prof, pk, args.k_storage)
            rk = kbuild_roofline(wl, wl.precision, kb_ms, pk, args.k_storage)
            pass_total = s["breakdown_ms_per_fit"]["reduce"] - sum(r["info"]["fold_ms"] for r in prof) / len(prof)
            # the dominant kernel of a fit: the K build or the stream kernel summed over the passes
            rooflines = [rk, rp] if kb_ms >= pass_total else [rp, rk]
            rooflines[0]["share_of_fit"] = (kb_ms if rooflines[0] is rk else pass_total) / s["ms_per_fit"]
        else:
            avg = s["breakdown_ms_per_fit"]["reduce"] / max(s["passes_per_fit"], 1)
            rooflines = [x for x in recompute_rooflines(wl, avg, pk) if x is not None]
        line = {
            "metric": METRIC,
            "value": value,
            "unit": "iters/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32" if wl.precision == "fp32" else f"{wl.precision} operands, f32 accumulate/K",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC if headline else f"{wl.name} scaled x{args.scale}",
                       "precision": wl.precision, "n": n, "d": wl.d, "k": k,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": (f"inputs larger than L2 (K = {4 * n * n / 1e9:.2f} GB as the full square; "
                              + ("its block-packed upper triangle" if s["k_pass"] == "symmetric" else
                                 "all of it" if s["k_pass"] == "full" else "recomputed, never stored")
                              + " read every pass)"),
                       "k_pass": s["k_pass"], "passes_per_fit": iters / args.steps},
            "kbuild_tflops": s["kbuild_tflops"],
            "kbuild_tflops_gemm_equivalent": s["kbuild_tflops_gemm_equivalent"],
            "kbuild_ms": kb_ms,
            "breakdown_ms_per_step": s["breakdown_ms_per_fit"],
            "pass_ms_graph": (graph_us_per_pass(pc, torch, wl, P, lab, out, wl.precision, args.steps, **kw) / 1e3
                              if wl.store_k and not wl.check_convergence else None),
            "objective": s["objective"],
            "roofline": rooflines[0],
            "e2e": {"value": e2e_iters_all / t_e2e, "unit": "iters/s",
                    "h2d_bytes_per_step": int(e2e_res[0]["info"]["h2d_bytes"]),
                    "d2h_bytes_per_step": int(e2e_res[0]["info"]["d2h_bytes"])},
            "gpu_launches": launches_all,
            "clocks": clk,
        }
        if len(rooflines) > 1:
            line["roofline_secondary"] = rooflines[1]
        forms = {}
        if headline and world == 1:
            # the tensor-core forms of the same fit: BF16X3 (split-BF16 cross term) and BF16,
            # and BF16X3 with K stored in FP16 (Gaussian K <= 1: 11 significant bits)
            for key, prec, kst in (("bf16x3", "bf16x3", "fp32"), ("bf16", "bf16", "fp32"),
                                   ("bf16x3_k_fp16", "bf16x3", "fp16")):
                try:   # a supplementary form never hides the headline
                    f = fit_form(pc, torch, stream, wl, P, lab, out, prec, args.steps, args.warmup,
                                 **{**kw, "k_storage": kst})
                    fs = f["summary"]
                    fs["k_storage"] = kst
                    fs["objective_rel_diff_vs_fp32_fit"] = abs(fs["objective"] - s["objective"]) / abs(s["objective"])
                    fs["speedup_vs_fp32_fit"] = fs["value"] / value
                    fs["roofline_kbuild"] = kbuild_roofline(wl, prec, fs["kbuild_ms"], pk, kst)
                    fs["roofline_pass"] = pass_roofline(wl, f["prof"], pk, kst)
                except Exception as ex:
                    fs = {"error": f"{type(ex).__name__}: {ex}"}
                forms[key] = fs
                line[key] = fs
        if headline and world == 1 and not args.no_extras:
            extras = {}
            for name in ("rings", "blobs", "mixture"):
                try:
                    kwx = {"autotune": args.autotune == "on"} if name == "mixture" else {}
                    es, ewl, _ = leg_workload(pc, torch, stream, name, args.steps, args.warmup, pk, **kwx)
                    if name == "mixture":
                        ewl.precision = "bf16"
                        Pm = torch.from_numpy(ewl.P).cuda()
                        Lm = torch.from_numpy(ewl.init_labels).cuda()
                        fb = fit_form(pc, torch, stream, ewl, Pm, Lm, torch.empty_like(Lm), "bf16", args.steps,
                                      args.warmup, **kwx)
                        avg = fb["summary"]["breakdown_ms_per_fit"]["reduce"] / max(fb["summary"]["passes_per_fit"], 1)
                        fb["summary"]["pass_ms"] = avg
                        fb["summary"]["roofline_pass"], _ = recompute_rooflines(ewl, avg, pk)
                        es = {"fp8": es, "bf16": fb["summary"]}
                    extras[name] = es
                except Exception as ex:   # an extra leg never hides the headline
                    extras[name] = {"error": f"{type(ex).__name__}: {ex}"}
            # batched forms: FP32 and BF16 builds with an FP32 K, and the FP32 build with a BF16 K
            # (every square rounded once, read by the tensor-core stream); objectives against the
            # FP32 form's, instance by instance
            for key, prec, kst in (("batched_fp32", "fp32", "fp32"), ("batched_bf16", "bf16", "fp32"),
                                   ("batched_fp32_k_bf16", "fp32", "bf16")):
                try:
                    extras[key] = leg_batched(pc, torch, stream, max(3, args.steps // 4), args.warmup, prec,
                                              args.autotune == "on", k_storage=kst)
                except Exception as ex:
                    extras[key] = {"error": f"{type(ex).__name__}: {ex}"}
            # each form's reported objectives against the FP64 objective of its own labels on the
            # exact K, on the 8 smallest instances (the oracle's K of each, FP64 on the host)
            batch_sample = None
            if not args.no_cpu_baseline:
                import oracle

                bw = synth.batched_instances(256, seed=0)
                batch_sample = sorted(range(len(bw)), key=lambda t: bw[t].n)[:8]
                bK = {t: oracle.kernel_matrix(bw[t].P, bw[t].kernel) for t in batch_sample}
            for key in ("batched_fp32", "batched_bf16", "batched_fp32_k_bf16"):
                x = extras.get(key, {})
                o, lab = x.pop("_objectives", None), x.pop("_labels", None)
                if o is None:
                    continue
                if batch_sample is not None:
                    x["objective_vs_fp64_of_labels_on_sample"] = {
                        "instances": [int(bw[t].n) for t in batch_sample],
                        "max_rel_err": max(abs(o[t] - oracle.objective(bK[t], lab[t], bw[t].k))
                                           / abs(oracle.objective(bK[t], lab[t], bw[t].k)) for t in batch_sample)}
                if key != "batched_fp32" and "value" in extras.get("batched_fp32", {}):
                    x["speedup_vs_fp32_batched"] = x["value"] / extras["batched_fp32"]["value"]
            line["extras"] = extras
        if world == 1 and not args.no_cpu_baseline:
            n_s = min(SAMPLE.get(wl.name.split("_")[0], 2000), wl.n)
            base, Ko, ofit = cpu_baseline(wl, n_s)
            line["cpu_baseline"] = base
            if wl.store_k:
                try:
                    errs = sample_objective_errors(pc, torch, wl, Ko, ofit, n_s,
                                                   ["fp32", "bf16x3", "bf16", ("bf16x3_k_fp16", "bf16x3", "fp16")]
                                                   if headline else [(wl.precision, wl.precision, args.k_storage)])
                except Exception as ex:
                    errs = {"error": f"{type(ex).__name__}: {ex}"}
                line["objective_vs_oracle_on_sample"] = {"sample": f"first {n_s} points, same initial labels and "
                                                                   f"passes as the oracle's fit", **errs}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
