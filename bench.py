#!/usr/bin/env python3
"""Kernel K-means throughput on GB300: iterations/s of whole fits, plus K-build TFLOP/s.

One step = one complete ``popcorn_fit`` through the C ABI on the rings workload
(n = 20,000 points in the plane zero-padded to d = 8, k = 4, Gaussian kernel
sigma = 0.5, random initial labels, passes until no label changes, at most
100; K materialized in FP32 = 1.6 GB, larger than L2, so every pass streams it
from HBM).  A step runs every row of the hot path: the K build (norms, Gram
tiles, kernel epilogue), then per pass the K-streaming segmented reduction,
the self-similarity sums, and the distance/argmin/histogram pass.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

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
WORKLOAD = "rings"
WORKLOAD_DESC = ("rings n=20000 d=8 (2 + 6 zero pad) k=4, Gaussian sigma=0.5, random init, "
                 "passes to convergence (max 100), K materialized FP32 (1.6 GB)")
FALLBACK_HBM_GBS = 6800.0
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


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
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink n (profiling captures only; the reported workload is scale 1)")
    ap.add_argument("--workload", default=WORKLOAD, choices=["rings", "blobs", "images", "mixture", "batched"],
                    help="rings (default, the reported line), blobs, images, mixture (recompute path), "
                         "batched (256 instances in one graph)")
    ap.add_argument("--autotune", default="on", choices=["on", "off"],
                    help="time candidate schedules in the warm-up (batched and recompute paths)")
    ap.add_argument("--precision", default=None, choices=["fp32", "bf16", "bf16x3", "fp8"],
                    help="K-build precision (default: the workload's)")
    ap.add_argument("--k-pass", default="auto", choices=["auto", "full", "symmetric"],
                    help="how a pass reads a stored FP32 K: the library's choice, the full square, or the blocks "
                         "on and above the diagonal (row and column sums, then a fold)")
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
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured (MEASURED_PEAKS.json: STREAM-style copy)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback (6.8 TB/s, earlier GB300 copy measurement)"


# exp2 unit (MUFU) rate measured on GB300: 32 ex2.approx per clock per SM (152 SMs)
XU_EX2_PER_CLK_SM = 32
GB300_SMS = 152


def recompute_rooflines(wl, avg_ms: float, clk: dict):
    """Rooflines of one recompute pass (sort + tiles + reduction), the binding one first.

    tensor: 2 n^2 d algorithmic MMA flops against the measured BF16 burst peak (FP8:
    twice that, the nominal FP8/BF16 ratio); alu: n^2 exp2 evaluations (Gaussian)
    against 32 per clock per SM at the maximum SM clock."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        bf16, src = float(m["bf16_tflops"]), "measured bf16 burst (MEASURED_PEAKS.json)"
        sm_mhz = float(m.get("sm_max_mhz", 2070.0))
    except Exception:
        bf16, src, sm_mhz = 1900.0, "fallback 1.9 PFLOP/s bf16", 2070.0
    peak_t = bf16 * (2.0 if wl.precision == "fp8" else 1.0)
    n, d = float(wl.n), float(wl.d)
    sec = avg_ms / 1e3 if avg_ms > 0 else float("inf")
    t_ach = 2.0 * n * n * d / sec / 1e12
    tensor = {"kernel": "recompute_kernel", "bound": "tensor", "achieved": t_ach, "peak": peak_t,
              "unit": "TFLOP/s", "frac": t_ach / peak_t, "traffic": None,
              "peak_source": src + (" x2 for FP8 (nominal ratio)" if wl.precision == "fp8" else ""),
              "algorithmic_flops_per_launch": 2.0 * n * n * d, "avg_launch_ms": avg_ms}
    peak_x = XU_EX2_PER_CLK_SM * GB300_SMS * sm_mhz * 1e6 / 1e12
    x_ach = n * n / sec / 1e12
    alu = {"kernel": "recompute_kernel", "bound": "alu", "achieved": x_ach, "peak": peak_x,
           "unit": "Texp2/s", "frac": x_ach / peak_x, "traffic": None,
           "peak_source": f"{XU_EX2_PER_CLK_SM} ex2/clk/SM x {GB300_SMS} SMs x {sm_mhz:.0f} MHz (ex2 microbenchmark)",
           "algorithmic_exp2_per_launch": n * n, "avg_launch_ms": avg_ms}
    if wl.kernel["kind"] != "gaussian":
        return tensor, None
    return (tensor, alu) if tensor["frac"] >= alu["frac"] else (alu, tensor)


def recorded_traffic(kernel: str, src_file: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is unchanged."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)[kernel]
        with open(os.path.join(ROOT, "paper_2501_05587_gb300", "csrc", src_file), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
        if t.get("source_sha256") != sha:
            return None
        return float(t["dram_bytes_per_launch"])
    except Exception:
        return None


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


def oracle_sample_rate(wl, n_sample: int, budget_s: float):
    """The FP64 oracle as it stands, on the first n_sample points of the workload.

    Returns (passes per second on the sample, sample description, passes, seconds).
    """
    import oracle

    P = wl.P[:n_sample]
    lab = wl.init_labels[:n_sample].copy()
    t0 = time.perf_counter()
    K = oracle.kernel_matrix(P, wl.kernel)
    t_build = time.perf_counter() - t0
    passes = 0
    t1 = time.perf_counter()
    while passes < wl.max_iter and time.perf_counter() - t1 < budget_s:
        st = oracle.step(K, lab, wl.k)
        passes += 1
        lab = st["labels"]
        if st["changed"] == 0:
            break
    t_loop = time.perf_counter() - t1
    return passes, t_build, t_loop


def oracle_cores():
    try:
        from threadpoolctl import threadpool_info
        n = max((int(i.get("num_threads", 1)) for i in threadpool_info()), default=1)
        return n
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(wl, n_sample=16000, budget_s=25.0):
    passes, t_build, t_loop = oracle_sample_rate(wl, n_sample, budget_s)
    # per-pass and K-build work scale with n^2; convert to full-workload iters/s
    scale = (n_sample / wl.n) ** 2
    it_s = passes / t_loop * scale if t_loop > 0 else 0.0
    return {"value": it_s, "unit": "iters/s", "cores": oracle_cores(), "kind": "oracle",
            "sample": (f"first {n_sample} of {wl.n} points, {passes} FP64 passes in {t_loop:.2f} s "
                       f"(K build {t_build:.2f} s); rate scaled by (n_sample/n)^2 = {scale:.4f} "
                       f"to the full workload")}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import synth

    wl = synth.workload(WORKLOAD)
    n_sample = 12000
    for _ in range(args.warmup):
        oracle_sample_rate(wl, 2000, 2.0)
    t_all = 0.0
    passes_all = 0
    for _ in range(args.steps):
        passes, t_build, t_loop = oracle_sample_rate(wl, n_sample, 15.0)
        t_all += t_build + t_loop
        passes_all += passes
    scale = (n_sample / wl.n) ** 2
    value = passes_all / t_all * scale
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "n": wl.n, "d": wl.d, "k": wl.k},
            "cpu_baseline": {"value": value, "unit": "iters/s", "cores": oracle_cores(), "kind": "oracle",
                             "sample": (f"each step: FP64 oracle K build + passes on the first {n_sample} "
                                        f"points; whole-fit rate scaled by (n_sample/n)^2 = {scale:.4f}")},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batched(args):
    """256 independent instances (n in [500, 8000], d in {8, 32, 64}, k in [4, 64], polynomial and
    Gaussian kernels), 30 passes each, one popcorn_fit_batched call per step."""
    import torch

    import synth
    import paper_2501_05587_gb300 as pc

    prec = args.precision or "fp32"
    wls = synth.batched_instances(int(256 * args.scale) or 1, seed=0)
    insts = [{"P": torch.from_numpy(w.P).cuda(), "k": w.k, "kernel": w.kernel,
              "init_labels": torch.from_numpy(w.init_labels).cuda()} for w in wls]

    def step():
        return pc.popcorn_fit_batched(insts, max_iter=30, precision=prec, check_convergence=False, timing=True,
                                      autotune=args.autotune == "on")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    res = [step() for _ in range(args.steps)]
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    passes = sum(sum(r["iterations"]) for r in res)
    kbytes = sum(4.0 * w.n * w.n for w in wls)
    graph_ms = sum(r["info"]["loop_ms"] for r in res) / len(res)
    # the same instances as separate popcorn_fit calls (the unbatched form), one sweep
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record()
    for x in insts:
        pc.popcorn_fit(x["P"], x["k"], x["kernel"], x["init_labels"], max_iter=30, precision=prec,
                       check_convergence=False)
    e3.record()
    torch.cuda.synchronize()
    seq_ms = e2.elapsed_time(e3)
    line = {"metric": METRIC, "value": passes / (ms / 1e3), "unit": "instance-passes/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": {"workload": f"batched: {len(wls)} instances, 30 passes each, K stored FP32 "
                                   f"({kbytes / 1e9:.1f} GB)", "precision": prec},
            "graph_ms": graph_ms, "effective_GBps_of_K_reads": kbytes * 30 / (graph_ms / 1e3) / 1e9,
            "separate_fits_ms": seq_ms, "batched_speedup_vs_separate_fits": seq_ms / (ms / args.steps),
            "gpu_launches": sum(r["info"]["kernel_launches"] for r in res),
            "schedule": {"autotune": args.autotune, "columns_per_unit": res[-1]["info"]["schedule"][0],
                         "warps_per_block": res[-1]["info"]["schedule"][1],
                         "blocks_per_sm": res[-1]["info"]["schedule"][2]}}
    print(json.dumps(line), flush=True)
    return 0


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


def main():
    args = parse()
    if args.compare == "paper":
        return run_paper_pipeline(args)
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

    wl = synth.workload(args.workload, scale=args.scale)
    if args.precision:
        wl.precision = args.precision
    P = torch.from_numpy(wl.P).cuda()
    lab = torch.from_numpy(wl.init_labels).cuda()
    out = torch.empty_like(lab)

    # the recompute path's schedule (row blocks per tile, units per SM) is autotuned in the warm-up
    tune = args.autotune == "on" and not wl.store_k

    def step(timing=True):
        return pc.popcorn_fit(P, wl.k, wl.kernel, lab, max_iter=wl.max_iter, check_convergence=wl.check_convergence,
                              precision=wl.precision, timing=timing, labels_out=out, store_k=wl.store_k,
                              autotune=tune, k_pass=args.k_pass)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    results, prof = [], []
    with ClockSampler(local) as clocks:
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            results.append(step(timing=False))
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        # The same fits again with the library's per-kernel CUDA events (on the launch stream):
        # the phase breakdown and the roofline kernel's launch time come from these.  The events
        # cost a few percent of a fit, so they stay out of the timed region above.
        for _ in range(args.steps):
            prof.append(step(timing=True))
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.summary()

    iters = sum(r["iterations"] for r in results)
    red_ms = sum(r["info"]["reduce_ms"] for r in prof)
    red_n = sum(r["info"]["reduce_launches"] for r in prof)
    asg_ms = sum(r["info"]["assign_ms"] for r in prof)
    kb_ms = sum(r["info"]["kbuild_ms"] for r in prof)
    launches = sum(r["info"]["kernel_launches"] for r in results)

    # end to end through the same call with pinned host buffers (copies inside the timed region)
    Ph = torch.from_numpy(wl.P).pin_memory()
    Lh = torch.from_numpy(wl.init_labels).pin_memory()
    Oh = torch.empty(wl.n, dtype=torch.int32).pin_memory()
    def host_step():
        return pc.popcorn_fit(Ph, wl.k, wl.kernel, Lh, max_iter=wl.max_iter, check_convergence=wl.check_convergence,
                              precision=wl.precision, labels_out=Oh, store_k=wl.store_k, autotune=tune,
                              k_pass=args.k_pass)

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
        kb_flops = float(n) * (n + 1) * wl.d           # algorithmic: n(n+1)/2 unique dot products, 2d flops each
        alg_bytes = 4.0 * n * n + n                      # K read once + label bytes, per reduction launch
        avg_red_ms = red_ms / max(red_n, 1)
        peak, peak_src = peaks()
        achieved = alg_bytes / (avg_red_ms / 1e3) / 1e9 if avg_red_ms > 0 else 0.0
        traffic = recorded_traffic("reduce_kernel", "iterate.cu")
        roof = {"kernel": "reduce_kernel", "bound": "hbm", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                "peak_source": peak_src,
                "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_red_ms}
        roof2 = None
        if results[-1]["info"]["k_pass_used"] == 1:
            # symmetric pass: the stream kernel alone (its CUDA-event time is the pass's
            # reduction minus the fold, both recorded by the library on the launch stream)
            T = (n + 127) // 128
            tri = sum(min(128, n - 128 * I) * (n - 128 * I) for I in range(T))   # elements of blocks (I, J >= I)
            fold_ms = sum(r["info"]["fold_ms"] for r in prof)
            passes = sum(r["iterations"] for r in prof)
            avg_stream_ms = (red_ms - fold_ms) / max(passes, 1)
            alg_bytes = 4.0 * tri + 4.0 * T * k * n + 256.0 * T * (T + 1) / 2   # K blocks, slots, labels
            achieved = alg_bytes / (avg_stream_ms / 1e3) / 1e9 if avg_stream_ms > 0 else 0.0
            roof = {"kernel": "reduce_sym_kernel", "bound": "hbm", "achieved": achieved, "peak": peak,
                    "unit": "GB/s", "frac": achieved / peak, "traffic": recorded_traffic("reduce_sym_kernel",
                                                                                         "reduce_sym.cu"),
                    "peak_source": peak_src, "algorithmic_bytes_per_launch": alg_bytes,
                    "avg_launch_ms": avg_stream_ms,
                    "pass": "symmetric: blocks on and above the diagonal, then sym_fold_kernel",
                    "fold_avg_launch_ms": fold_ms / max(passes, 1)}
        if not wl.store_k:
            # recompute pass: tensor cores (2 n^2 d flops) and the exp2 unit (n^2 kernel values)
            roof, roof2 = recompute_rooflines(wl, avg_red_ms, clk)
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
            "config": {"workload": (WORKLOAD_DESC if args.workload == WORKLOAD and args.scale == 1.0
                                    else f"{wl.name} scaled x{args.scale}"),
                       "precision": wl.precision,
                       "n": n, "d": wl.d, "k": k,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": (f"inputs larger than L2 (K = {4 * wl.n * wl.n / 1e9:.2f} GB; "
                              + ("its upper triangle of 128-blocks" if results[-1]["info"]["k_pass_used"] == 1
                                 else "all of it") + " streamed every pass)"),
                       "k_pass": {0: "recompute", 1: "symmetric", 2: "full"}[results[-1]["info"]["k_pass_used"]],
                       "passes_per_fit": iters / args.steps},
            "kbuild_tflops": kb_flops / (kb_ms / args.steps / 1e3) / 1e12 if kb_ms > 0 else None,
            "kbuild_tflops_gemm_equivalent": (2.0 * n * n * wl.d / (kb_ms / args.steps / 1e3) / 1e12
                                              if kb_ms > 0 else None),
            "kbuild_ms": kb_ms / args.steps,
            "loop_iters_per_s": iters / ((red_ms + asg_ms) / 1e3) if red_ms > 0 else None,
            "breakdown_ms_per_step": {"kbuild": kb_ms / args.steps, "reduce": red_ms / args.steps,
                                      "assign": asg_ms / args.steps},
            "roofline": roof,
            "e2e": {"value": e2e_iters_all / t_e2e, "unit": "iters/s",
                    "h2d_bytes_per_step": int(e2e_res[0]["info"]["h2d_bytes"]),
                    "d2h_bytes_per_step": int(e2e_res[0]["info"]["d2h_bytes"])},
            "gpu_launches": launches_all,
            "clocks": clk,
        }
        if roof2 is not None:
            line["roofline_secondary"] = roof2
            line["schedule"] = {"autotune": args.autotune, "row_blocks_per_tile": results[-1]["info"]["schedule"][0],
                                "column_segments": results[-1]["info"]["schedule"][1],
                                "units_per_sm_target": results[-1]["info"]["schedule"][2]}
        if args.workload == WORKLOAD and args.scale == 1.0:
            # the same fits with K stored in FP16: half the bytes per pass (an extra, not the headline)
            def step16():
                return pc.popcorn_fit(P, wl.k, wl.kernel, lab, max_iter=wl.max_iter, check_convergence=True,
                                      timing=True, labels_out=out, k_storage="fp16")
            for _ in range(args.warmup):
                step16()
            torch.cuda.synchronize()
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            r16 = [step16() for _ in range(args.steps)]
            f1.record(stream)
            torch.cuda.synchronize()
            ms16 = f0.elapsed_time(f1)
            it16 = sum(r["iterations"] for r in r16)
            red16 = sum(r["info"]["reduce_ms"] for r in r16) / max(1, sum(r["info"]["reduce_launches"] for r in r16))
            line["k_fp16"] = {"value": it16 / (ms16 / 1e3), "unit": "iters/s", "passes_per_fit": it16 / args.steps,
                              "objective_rel_diff_vs_fp32_k": abs(r16[0]["objective"] - results[0]["objective"])
                              / abs(results[0]["objective"]),
                              "reduce_avg_launch_ms": red16,
                              "reduce_GBps": (2.0 * n * n + n) / (red16 / 1e3) / 1e9 if red16 > 0 else None}
        if world == 1 and not args.no_cpu_baseline and args.workload == WORKLOAD:
            line["cpu_baseline"] = cpu_baseline(wl)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
