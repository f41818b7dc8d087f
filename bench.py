"""Benchmark: repeated-pattern multivector FETI solves on one GB300.

Workload (default): 3D elasticity, three 16^3-element Q1 cube patterns (E = 1, nu = 0.3), 4 x 6 x 8 = 192
occurrences with seeded rotations of the cube, clamped face x = 0, body force N(0,1) per dof (n_lambda =
427,392, 1152 rigid modes).  A step is one pass of the whole method on that structure: FP64 factorisation of the
three patterns (zero-pivot detection, kernel, S^+), coarse problem and d, block ORTHODIR with k = 32 to
||r|| / ||r0|| <= 1e-8 (local products on the tensor cores in bf16 pairs inside FP64 outer refinement), and the
recovery of lambda and u.  Inputs (pattern stiffness, links, loads) are resident on the device when the timed
region starts; the operands of every step are larger than L2 (the S^dag operators alone are 0.25 GB in bf16
pairs), and L2 is flushed between steps as well.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision fp64|fp32|tf32x3|bf16x3|auto] [--k K] [--workload c3|c2|c1|c4|c5]

Under torchrun (N > 1) every rank solves its own independently seeded structure (weak scaling, no collective
on the data path); rank 0 prints the JSON line with the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FETI solves/s to 1e-8 rel. residual"
WORKLOADS = {
    "c2": "2D heat, two 32x32 Q1 patterns (conductivity 1 / 1000, seeded checkerboard) on 8x8 occurrences, "
          "u=0 on x=0, f~U(0,1), n_lambda=3904",
    "c1": "2D heat, one 8x8 Q1 pattern on 2x2 occurrences, u=0 on x=0, f~U(0,1), n_lambda=52",
    "c3": "3D elasticity, three 16^3 Q1 cube patterns, 4x6x8 occurrences with seeded cube rotations, clamped x=0, "
          "N(0,1) per dof, n_lambda=427392",
    "c4": "batched uneven 3D elasticity: hex patterns 8^3/12^3/16^3/24^3, 256 occurrences drawn with weights "
          "0.4/0.3/0.2/0.1, each pattern's occurrences one clamped block, all blocks solved in one structure, "
          "multivector width autotuned over {4,8,16,32}",
    "c5": "serving: structures arriving by a seeded Poisson process (mean 50/s), each 4-128 occurrences of one of "
          "6 resident patterns (2D heat 16^2/32^2/64^2, 3D elastic 8^3/12^3/16^3), admitted by device memory",
}
DEFAULTS = {  # per workload: local-product precision, multivector width, direction-history cap (GB; 0 = library)
    "c3": ("bf16x3", 4, 32.0), "c2": ("fp32", 8, 0.0), "c1": ("fp64", 4, 0.0), "c5": ("auto", 8, 0.0),
    "c4": ("auto", 0, 32.0),   # k = 0: autotuned
}
# Block iterations of the default workload (C3, k = 4, tol 1e-8): the count the library's solve needs on this
# structure, used to scale the oracle's sampled per-iteration cost to a whole solve.  k = 4 is the width the
# library's autotuner picks on C3 from {4, 8, 16, 32} (the direction-history work grows with k).
C3_ITERATIONS = 132
PHASE_KERNELS = {  # the kernels each phase launches
    "factor": "k_potrf_tile, k_trsm_tiles, k_update_pairs, k_tile_inverse, k_tri_*; n_b >= 1024: k_pinv_rows_tf32, "
              "k_tc_gemm<0> (S^dag = Y^T Y), k_split_bf16; else k_lauum, k_split_tf32/bf16",
    "coarse": "k_row_coefs, k_gtg, k_gemm_f64, d: k_tri_*",
    "local": "k_local_gemm / k_tc_gemm", "gather": "k_gather_tile, k_rotate_traces", "scatter": "k_scatter",
    "project": "k_gt_v, k_small_gemm, k_g_apply (FP64); k_split_pairs, k_gt_v_ds, k_small_gemm_ds, "
               "k_g_apply_ds(_rows) (mixed forms)",
    "gram": "k_group_wr, k_gram_split + k_reduce_chunks_dyn, k_eta_partial(_ds) + k_eta_group_sums",
    "reorth": "k_tall_update / k_tall_update_w<4|8|16|32>", "update": "k_split / k_perm_split, k_update",
    "recover": "k_tri_*, k_unpermute_rotate", "normalise": "k_normalise",
    "iterate": "k_persist (whole block iterations in one cooperative launch)",
    "outer": "FP64 residual: k_gather_tile, k_local_gemm<double> (n_b >= 1024: two triangular products with "
             "L_S^{-1}), k_scatter, projection",
}
PHASE_BOUND = {  # roofline resource of each phase's kernels
    "factor": "alu", "coarse": "alu", "local": "alu", "gather": "hbm", "scatter": "hbm", "project": "alu",
    "gram": "alu", "reorth": "alu", "update": "alu", "recover": "alu", "normalise": "alu", "iterate": "hbm",
    "outer": "alu",
}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# FP64 / FP32 SIMT peaks of GB300 derived from the unit counts and clock: 152 SMs x 2070 MHz x
# (FP32: 128 FMA lanes/SM -> 80.5 TFLOP/s; FP64: nominal 1.25 TFLOP/s, i.e. ~2 FMA/clk/SM).
FP64_PEAK_TFLOPS = 1.25
FP32_PEAK_TFLOPS = 152 * 2070e6 * 128 * 2 / 1e12


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed(base_seed, rank):
    """Every rank solves its own, independently seeded structure of the same shape (weak scaling)."""
    return base_seed + 1000003 * rank


def job_throughput(local_total_ms, steps, world, reduce_max=None):
    """Whole-job solves/s: every rank ran `steps` solves; the job time is the slowest rank's (max over ranks).
    reduce_max: callable taking a float and returning the max over ranks (None for one rank)."""
    total_ms = reduce_max(local_total_ms) if (reduce_max and world > 1) else local_total_ms
    return world * steps / (total_ms / 1e3), total_ms / steps


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
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
            self.f.close()

    def summary(self, gpu_index=0):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9 or p[0] != str(gpu_index):
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "samples": len(sm),
                "reasons": sorted(reasons)}


def h2d_bytes(prob):
    b = 0
    for pat in prob.patterns:
        K = pat.K
        b += K.indptr.size * 8 + K.indices.size * 4 + K.data.size * 8 + pat.bnd_nodes.size * 4
    for o in prob.occs:
        b += o.n_links * (4 + 1 + 4 + 1) + o.f_global.size * 8 + 9 * 8
    b += prob.n_lambda * 8 + prob.n_occ * 4
    return b


def fapply_bytes(prob, k, es):
    """Algorithmic bytes of one block F-apply (one Q = P^T F P Z over k columns): the local operators streamed
    once (sum_p n_b^2 / 2 entries of size es, the symmetric factor's half) + the block read and written in FP64
    (2 n_lambda k 8) + the coarse vectors (2 n_G k 8)."""
    nb = sum(p.n_b ** 2 / 2 for p in prob.patterns)
    n_G = sum(prob.patterns[o.pattern].kernel_dim for o in prob.occs)
    return nb * es + 2 * prob.n_lambda * k * 8 + 2 * n_G * k * 8


def run_ours(args, rank, world, local):
    import torch
    import paper_1208_6387_gb300.fetirp as F
    from fetirp_gen import config

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    prob = config(args.workload, seed=rank_seed(args.seed, rank), k=args.k or None)
    stream = torch.cuda.Stream(device=dev)
    if args.precision == "auto":   # the library's rule: FP32 SIMT for latency-bound structures, else tf32x3
        max_nb = max(p.n_b for p in prob.patterns)
        args.fprec = "fp32" if (max_nb <= 512 and prob.n_lambda <= 262144) else "tf32x3"
    else:
        args.fprec = args.precision
    autotune = None
    if not args.k:   # the library's autotuner picks the multivector width (untimed, before the steps)
        o = F.fetirp_default_options(precision=args.precision, tol=1e-8, inner_tol=args.inner_tol, device=local,
                                     history_bytes=int(args.history_gb * 1e9))
        o.cuda_stream = stream.cuda_stream
        c = F.fetirp_create(o)
        F.load_problem(c, prob)
        cand = (4, 8, 16, 32)
        best, times = F.fetirp_autotune_k(c, prob.n_lambda, prob.c, cand)
        F.fetirp_destroy(c)
        prob.k = best
        prob.groups = (np.arange(prob.n_occ) * best // prob.n_occ).astype(np.int32)
        autotune = {"candidates": list(cand), "solve_ms": [round(float(t), 2) for t in times], "best_k": best,
                    "grouping": "contiguous occurrence ids"}
    nu = F.n_u(prob)
    c_d = torch.tensor(prob.c, dtype=torch.float64, device=dev)
    lam_d = torch.empty(prob.n_lambda, dtype=torch.float64, device=dev)
    u_d = torch.empty(nu, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    hist_bytes = int(args.history_gb * 1e9)

    def make_ctx(precision, timing, mask=0):
        opts = F.fetirp_default_options(precision=precision, tol=1e-8, inner_tol=args.inner_tol, device=local,
                                        timing=timing, timing_mask=mask, history_bytes=hist_bytes)
        opts.cuda_stream = stream.cuda_stream
        c = F.fetirp_create(opts)
        F.load_problem(c, prob)
        return c

    def step(c):
        F.fetirp_factorize(c)
        return F.fetirp_solve_device(c, prob.n_lambda, c_d.data_ptr(), lam_d.data_ptr(), u_d.data_ptr())

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.zero_()

    # untimed probe: every phase bracketed by events (the phase table of one step, after a first step that also
    # builds the structure tables and captures the iteration graphs)
    ctx = make_ctx(args.precision, 1, 0)
    probe = []
    for _ in range(2):
        flush_l2()
        probe.append(step(ctx))
    F.fetirp_destroy(ctx)
    probe_ms = np.asarray(probe[-1]["phase_ms"])
    # timed: the phases the roofline keys read are bracketed by events (two event nodes per phase occurrence
    # inside the captured graphs); the others run without, as in a solve without timing
    timed_phases = ("factor", "coarse", "local", "gram", "reorth", "iterate")
    mask = sum(1 << F.PHASES.index(p) for p in timed_phases)
    ctx = make_ctx(args.precision, 1, mask)
    for _ in range(args.warmup):
        flush_l2()
        step(ctx)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    import tempfile
    clk_dir = tempfile.mkdtemp(prefix="fetirp_clocks_")
    clk = Clocks(os.path.join(clk_dir, f"clocks_rank{rank}.csv"))
    torch.cuda.synchronize()
    with clk:
        t0 = time.perf_counter()
        for i in range(args.steps):
            flush_l2()
            ev[i][0].record(stream)
            stats.append(step(ctx))
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]

    def reduce_max(x):
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    value, ms_per_step = job_throughput(sum(step_ms), args.steps, world, reduce_max)
    total_ms = ms_per_step * args.steps
    rel_res = max(s["rel_residual"] for s in stats)

    ph_ms = np.sum([s["phase_ms"] for s in stats], axis=0)
    ph_fl = np.sum([s["phase_flops"] for s in stats], axis=0)
    ph_by = np.sum([s["phase_bytes"] for s in stats], axis=0)
    ph_ln = np.sum([s["phase_launches"] for s in stats], axis=0)
    peaks, src = load_peaks()
    iters = float(np.mean([s["iterations"] for s in stats]))
    roof = roofline(args, prob, F, peaks, src, ph_ms, ph_fl, ph_ln, stats)
    roof["share_of_step"] = round(float(ph_ms[F.PHASES.index(roof["phase"])]) / total_ms, 4) if world == 1 else None
    roof["timed_phases_ms_per_step"] = {p: round(float(ph_ms[F.PHASES.index(p)]) / args.steps, 3)
                                        for p in timed_phases}
    roof["phases_ms_per_step_untimed_probe"] = {F.PHASES[i]: round(float(probe_ms[i]), 3)
                                                for i in range(len(F.PHASES))}
    # the pattern set-up (tile Cholesky, L_S^{-1}, S^+): FP64 flops counted by the library from the tile plans
    fi = F.PHASES.index("factor")
    setup_roof = None
    if ph_fl[fi] > 0 and ph_ms[fi] > 0:
        ach = float(ph_fl[fi]) / (float(ph_ms[fi]) / 1e3) / 1e12
        setup_roof = {"phase": "factor", "kernels": PHASE_KERNELS["factor"], "bound": "fp64",
                      "achieved": round(ach, 4), "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                      "frac": round(ach / FP64_PEAK_TFLOPS, 4),
                      "share_of_step": round(float(ph_ms[fi]) / total_ms, 4) if world == 1 else None,
                      "peak_source": "nominal FP64 rate (no measured FP64 peak on this pool)",
                      "work": "FP64 flops of the tile Cholesky (tile pairs with fill), L_S^{-1}, and S^+ for n_b < 1024 (larger "
                              "patterns form S^dag on the tensor cores), per step"}
    # the direction-history work (Gram products incl. eta, and the reorthogonalisation), its own key
    hg = [F.PHASES.index("gram"), F.PHASES.index("reorth")]
    hist_ms = float(sum(ph_ms[i] for i in hg))
    hist_by = float(sum(ph_by[i] for i in hg))
    history = {"kernels": PHASE_KERNELS["gram"] + "; " + PHASE_KERNELS["reorth"],
               "ms_per_step": round(hist_ms / args.steps, 3), "ms_per_iteration": round(hist_ms / args.steps / iters, 4),
               "bytes_per_step": hist_by / args.steps,
               "achieved_gbs": round(hist_by / (hist_ms / 1e3) / 1e9, 2) if hist_ms > 0 else None,
               "peak_gbs": peaks["hbm_gbs"], "frac": round(hist_by / (hist_ms / 1e3) / 1e9 / peaks["hbm_gbs"], 4)
               if hist_ms > 0 else None,
               "note": "algorithmic bytes of the history reads and block passes (library accounting), HBM of " + src}
    F.fetirp_destroy(ctx)

    def fapply_rate(precision, n_app):
        c = make_ctx(precision, 0)
        F.fetirp_prepare(c, prob.n_lambda, prob.c)
        k = prob.k
        V = torch.randn(prob.n_lambda, k, dtype=torch.float64, device=dev)
        Qo = torch.empty_like(V)
        prec = F.PRECISIONS[precision]
        for _ in range(3):
            F.fetirp_apply_block_device(c, k, V.data_ptr(), Qo.data_ptr(), prec)
        F.fetirp_device_status(c)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n_app):
            F.fetirp_apply_block_device(c, k, V.data_ptr(), Qo.data_ptr(), prec)
        b.record(stream)
        torch.cuda.synchronize()
        F.fetirp_device_status(c)
        F.fetirp_destroy(c)
        return n_app / (a.elapsed_time(b) / 1e3)

    fapply = {args.fprec: round(fapply_rate(args.fprec, 50), 2)}

    # the plain FP64 form of the same step (same k, same history cap), for comparison: one timed solve
    plain = None
    if args.precision != "fp64" and not args.no_fp64_reference:
        c = make_ctx("fp64", 0)
        if args.workload not in ("c3", "c4"):
            step(c)   # small structures: one untimed solve first (graph capture, buffers)
        times, its = [], []
        for _ in range(1 if args.workload in ("c3", "c4") else 3):
            flush_l2()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st = step(c)
            b.record(stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
            its.append(st["iterations"])
        F.fetirp_destroy(c)
        fapply["fp64"] = round(fapply_rate("fp64", 10 if args.workload in ("c3", "c4") else 50), 3)
        plain = {"time_to_solution_ms": round(statistics.median(times), 2), "iterations": its[-1],
                 "block_f_applies_per_s": fapply["fp64"],
                 "speedup_of_mixed_time_to_solution": round(statistics.median(times) / ms_per_step, 3),
                 "speedup_of_mixed_f_applies": round(fapply[args.fprec] / fapply["fp64"], 3)}

    # e2e: the public API from host buffers (create, patterns, occurrences, solve, outputs to host, destroy)
    e2e_times = []
    for i in range(3 if args.workload in ("c3", "c4") else max(2, min(args.steps, 5)) + 1):
        t = time.perf_counter()
        c2 = F.fetirp_create(F.fetirp_default_options(precision=args.precision, tol=1e-8, inner_tol=args.inner_tol,
                                                       device=local, history_bytes=hist_bytes))
        F.load_problem(c2, prob)
        F.fetirp_solve(c2, prob.n_lambda, prob.c, nu)
        F.fetirp_destroy(c2)
        if i > 0:
            e2e_times.append(time.perf_counter() - t)
    e2e_s = statistics.median(e2e_times)
    launches = int(np.mean([s["launches"] for s in stats]))
    out = {
        "metric": METRIC, "value": round(value, 4), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.fprec == "fp64" else "f64+" + args.fprec,
        "data": "synthetic (seeded Q1 meshes, rotations, loads; no datasets)",
        "config": {"workload": WORKLOADS[args.workload], "name": args.workload, "precision": args.precision,
                   "block_k": prob.k, "n_lambda": prob.n_lambda, "n_occ": prob.n_occ,
                   "l2": "operands larger than L2 and L2 flushed between steps (256 MB write)", "tol": 1e-8,
                   "history_gb": args.history_gb,
                   "step": "factorise patterns + coarse + d + block ORTHODIR + recovery"},
        "time_to_solution_ms": round(ms_per_step, 3),
        "setup_ms_per_step": round(float(ph_ms[F.PHASES.index("factor")] + ph_ms[F.PHASES.index("coarse")]) / args.steps, 2),
        "autotune": autotune,
        "iterations": stats[-1]["iterations"], "outer_steps": stats[-1]["outer_steps"],
        "rel_residual": rel_res,
        "block_f_applies_per_s": fapply,
        "plain_fp64": plain,
        "gpu_launches": launches * args.steps,
        "e2e": {"value": round(world / e2e_s, 4), "unit": "solves/s", "h2d_bytes_per_step": h2d_bytes(prob),
                "d2h_bytes_per_step": (prob.n_lambda + nu) * 8},
        "roofline": roof,
        "history_gram": history,
        "setup_roofline": setup_roof,
        "clocks": clk.summary(local),
        "wall_s": round(wall, 4),
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, prob, stats[-1]["iterations"])
    if world > 1:
        torch.distributed.destroy_process_group()
    return out


def roofline(args, prob, F, peaks, src, ph_ms, ph_fl, ph_ln, stats):
    """Roofline of the dominant kernel of the F-apply, from the library's per-launch CUDA events over the timed
    steps (events on the library's stream) and the algorithmic work of one launch.
    tf32x3 / bf16x3: k_tc_gemm, flops 2 sum_p n_b^2 R_p per launch (useful; three products are issued for each)
    against the tensor peak of the operand type: the measured sustained bf16 rate (bf16x3), times 1.1 / 2.25
    (the nominal tf32 / bf16 ratio) for tf32x3.
    Persistent iteration (FP32 / FP64 SIMT, latency-bound structures): k_persist, the F-apply bytes of every
    block iteration in the launch against the measured HBM copy rate."""
    loc, itp = F.PHASES.index("local"), F.PHASES.index("iterate")
    if ph_ln[itp] > 0:
        es = 8 if args.fprec == "fp64" else 4
        n_it = float(sum(s["iterations"] for s in stats))
        per_launch_ms = ph_ms[itp] / ph_ln[itp]
        bytes_per_launch = fapply_bytes(prob, prob.k, es) * n_it / ph_ln[itp]
        achieved = bytes_per_launch / (per_launch_ms / 1e3) / 1e9
        return {"kernel": "k_persist", "phase": "iterate", "bound": "hbm", "achieved": round(achieved, 3),
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 6),
                "traffic": None, "bytes_per_launch": bytes_per_launch, "launches": int(ph_ln[itp]),
                "ms_per_launch": round(per_launch_ms, 4),
                "peak_source": "hbm_gbs of " + src,
                "work": "F-apply bytes (operators once + 2 n_lambda k 8 + 2 n_G k 8) x block iterations per launch"}
    # one local product = 2 sum_p n_b^2 R_p useful flops; with a split reduction dimension (small blocks) it is
    # the product kernel plus the in-order sum of its partials, both inside the phase's events
    fl_one = sum(2.0 * p.n_b ** 2 * sum(1 for o in prob.occs if o.pattern == i) * prob.k
                 for i, p in enumerate(prob.patterns))
    n_prod = max(int(round(float(ph_fl[loc]) / fl_one)), 1) if fl_one > 0 else max(int(ph_ln[loc]), 1)
    per_launch_ms = ph_ms[loc] / n_prod
    flops_per_launch = ph_fl[loc] / n_prod
    achieved = flops_per_launch / (per_launch_ms / 1e3) / 1e12
    if args.fprec == "tf32x3":
        kern, bound = "k_tc_gemm (tcgen05 kind::tf32, 3 products)", "tensor"
        peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]) * 1.1 / 2.25
        note = f"tf32 tensor: bf16_tflops_sustained of {src} x 1.1/2.25 (nominal tf32/bf16 ratio)"
    elif args.fprec == "bf16x3":
        kern, bound = "k_tc_gemm (tcgen05 kind::f16, bf16 operands, 3 products)", "tensor"
        peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        note = f"bf16 tensor: bf16_tflops_sustained of {src}"
    elif args.fprec == "fp32":
        kern, bound, peak = "k_local_gemm<float>", "alu", FP32_PEAK_TFLOPS
        note = "FP32 SIMT peak derived from 152 SMs x 128 lanes x 2070 MHz"
    else:
        kern, bound, peak = "k_local_gemm<double>", "alu", FP64_PEAK_TFLOPS
        note = "FP64 nominal 1.25 TFLOP/s (152 SMs x 2070 MHz)"
    out = {"kernel": kern, "phase": "local", "bound": bound, "achieved": round(achieved, 3), "peak": round(peak, 2),
           "unit": "TFLOP/s", "frac": round(achieved / peak, 5), "traffic": None,
           "flops_per_launch": flops_per_launch, "launches": int(ph_ln[loc]), "products": n_prod,
           "ms_per_launch": round(per_launch_ms, 4),
           "peak_source": note, "work": "2 sum_p n_b^2 R_p per local product (R_p = occurrences of p x k); a product is one "
                   "k_tc_gemm launch, plus k_tc_reduce when small blocks split the reduction dimension"}
    if args.fprec in ("tf32x3", "bf16x3"):
        out["issued_frac"] = round(3 * achieved / peak, 4)
    return out


class OracleSampler:
    """Bounded sample of the oracle on a structure too large to solve on the host within the benchmark.  The
    oracle's set-up (FetiOracle: pattern factorisations, G, G^T G and its inverse) is timed in full once; each
    sample then times one F-apply of a k-column block through the oracle's generalized inverse restricted to
    n_sample_occ occurrences (scaled to all of them) and one projection.  Estimated solve time = set-up +
    n_it x (F-apply + 2 projections).  The oracle's history reorthogonalisation is left out, so the estimate
    favours the oracle."""

    def __init__(self, prob):
        from oracle.feti import FetiOracle
        self.prob = prob
        t = time.perf_counter()
        self.o = FetiOracle(prob, use_schur=False)
        self.t_setup = time.perf_counter() - t
        self.V = np.random.default_rng(5).standard_normal((prob.n_lambda, prob.k))

    def sample(self, n_it, n_sample_occ=8):
        o, prob, V = self.o, self.prob, self.V
        t = time.perf_counter()
        for s in range(n_sample_occ):
            o.Bs[s] @ o.kplus(s, o.Bs[s].T @ V)
        t_f = (time.perf_counter() - t) * prob.n_occ / n_sample_occ
        t = time.perf_counter()
        o.project(V)
        t_p = time.perf_counter() - t
        est = self.t_setup + n_it * (t_f + 2 * t_p)
        return est, (f"oracle set-up timed in full ({self.t_setup:.1f} s); one k={prob.k} F-apply on {n_sample_occ} "
                     f"of {prob.n_occ} occurrences ({t_f * n_sample_occ / prob.n_occ:.2f} s, scaled "
                     f"x{prob.n_occ / n_sample_occ:g}) and one projection ({t_p:.2f} s); solve = set-up + {n_it} "
                     f"iterations x (F-apply + 2 projections), reorthogonalisation not counted")


def oracle_step(prob):
    from oracle.feti import FetiOracle
    o = FetiOracle(prob)
    lam, it, _ = o.multivector(tol=1e-8, max_it=2000)
    o.recover(lam)
    return it


def cpu_baseline(args, prob, n_it):
    """The oracle as it stands (numpy/scipy FP64): one full solve of the workload when it finishes in seconds
    (C1, C2), else a bounded sample scaled to a solve."""
    cores = len(os.sched_getaffinity(0))
    if args.workload in ("c3", "c4"):
        est, what = OracleSampler(prob).sample(n_it)
        return {"value": round(1.0 / est, 6), "unit": "solves/s", "cores": cores, "kind": "oracle",
                "sample": what + f"; estimated {est:.1f} s per solve; numpy/scipy default BLAS threads"}
    t = time.perf_counter()
    it = oracle_step(prob)
    dt = time.perf_counter() - t
    return {"value": round(1.0 / dt, 5), "unit": "solves/s", "cores": cores,
            "kind": "oracle", "sample": f"one full solve of the same workload ({it} block iterations, "
                                        f"{dt:.1f} s; numpy/scipy default BLAS threads)"}


def run_reference(args, rank, world):
    """The oracle timed on the host cores (rank 0 only), same workload/metric; each step one full solve (C1, C2)
    or, for C3, one bounded sample scaled to a solve (the oracle's set-up, one sampled block F-apply and one
    projection; see _oracle_sample)."""
    from fetirp_gen import config
    if rank != 0:
        return None
    prob = config(args.workload, seed=args.seed, k=args.k or None)
    cores = len(os.sched_getaffinity(0))
    if args.workload == "c3":
        sampler = []

        def one():   # the set-up is timed once (first warm-up step), every step samples the iteration
            if not sampler:
                sampler.append(OracleSampler(prob))
            return sampler[0].sample(C3_ITERATIONS, n_sample_occ=4)
    else:
        def one():
            t = time.perf_counter()
            it = oracle_step(prob)
            return time.perf_counter() - t, f"one full oracle solve ({it} block iterations)"
    for _ in range(args.warmup):
        one()
    times, what = [], ""
    t0 = time.perf_counter()
    for _ in range(args.steps):
        est, what = one()
        times.append(est)
    wall = time.perf_counter() - t0
    value = args.steps / sum(times)
    sample = ("each step " + what) if args.workload != "c3" else ("each step a bounded sample: " + what)
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * sum(times) / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Q1 meshes, rotations, loads; no datasets)",
        "config": {"workload": WORKLOADS[args.workload], "name": args.workload, "block_k": prob.k,
                   "n_lambda": prob.n_lambda, "n_occ": prob.n_occ, "tol": 1e-8},
        "cpu_baseline": {"value": round(value, 6), "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 6), "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": round(wall, 3),
    }


def run_serving(args):
    """Continuous batching of whole structures over a resident library (fetirp_server_*): requests submitted at
    their Poisson arrival times, latency = submit -> result, throughput = requests / (last result - start)."""
    import threading
    import paper_1208_6387_gb300.fetirp as F
    from fetirp_gen import library_patterns, fill_structure, request_stream
    pats = library_patterns()
    lib = F.fetirp_create(F.fetirp_default_options())
    t = time.perf_counter()
    pids = []
    for p in pats:
        K = p.K.tocsr()
        pids.append(F.fetirp_create_pattern(lib, p.n_nodes, p.dpn, K.indptr, K.indices, K.data, p.bnd_nodes,
                                            p.kernel_dim))
    lib_s = time.perf_counter() - t
    reqs = request_stream(args.requests, args.rate, args.seed)
    probs = []
    for (_, pi, nocc, sd) in reqs:
        prob = fill_structure(pats[pi], nocc, seed=sd, k=args.k, rotate=pats[pi].dpn == 3)
        probs.append((pi, prob, F.structure_of(prob, {0: pids[pi]})))
    opts = F.fetirp_default_options(precision=args.precision, tol=1e-8, inner_tol=args.inner_tol,
                                    history_bytes=args.mem_budget // max(1, args.slots) // 2)
    srv = F.fetirp_server_create(lib, opts, args.slots, args.mem_budget)
    F.fetirp_server_set_batching(srv, args.batch)
    lat, stats_l, done_t = [None] * len(reqs), [None] * len(reqs), [None] * len(reqs)
    tickets = [None] * len(reqs)
    ready = threading.Event()

    def collector():
        for i in range(len(reqs)):
            while tickets[i] is None:
                ready.wait(0.001)
            _, prob, _ = probs[i]
            r = F.fetirp_server_wait(srv, tickets[i], prob.n_lambda, F.n_u(prob), -1.0, allow_noconv=True)
            lam, u, st, l = r
            lat[i], stats_l[i], done_t[i] = l, st, time.perf_counter()

    th = threading.Thread(target=collector)
    th.start()
    t0 = time.perf_counter()
    for i, (arr, _, _, _) in enumerate(reqs):
        dt = t0 + arr - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        tickets[i] = F.fetirp_server_submit(srv, probs[i][2])
        ready.set()
    th.join()
    t_end = max(done_t)
    F.fetirp_server_destroy(srv)
    lat_a = np.array(lat)
    conv = sum(1 for s in stats_l if s["rel_residual"] <= 1e-8)
    # the plain sequential FP64 form on a sample of the same requests (one context, one after the other)
    seq = F.fetirp_create_child(lib, F.fetirp_default_options(precision="fp64", tol=1e-8,
                                                             history_bytes=args.mem_budget // 2))
    seq_k = 8   # the plain FP64 form at its own best width (FP64 local products make wide blocks costly)
    ns = min(args.seq_sample, len(probs))
    ts = []
    for i in range(ns):
        pi, prob, _ = probs[i]
        F.fetirp_clear_occurrences(seq)
        for occ in prob.occs:
            F.fetirp_add_occurrence(seq, pids[pi], occ.rot.astype(float), occ.link_local_node, occ.link_global_comp,
                                    occ.link_lambda_row, occ.link_sign, occ.f_global)
        kk = min(seq_k, prob.n_occ)
        F.fetirp_set_groups(seq, kk, (np.arange(prob.n_occ) * kk // prob.n_occ).astype(np.int32))
        t = time.perf_counter()
        F.fetirp_solve(seq, prob.n_lambda, prob.c, F.n_u(prob), allow_noconv=True)
        ts.append(time.perf_counter() - t)
    F.fetirp_destroy(seq)
    F.fetirp_destroy(lib)
    value = len(reqs) / (t_end - t0)
    return {
        "metric": "served solves/s (p50/p99 latency) to 1e-8 rel. residual", "value": round(value, 3),
        "unit": "solves/s", "n_gpus": 1, "steps": len(reqs), "warmup": 0,
        "ms_per_step": round(1e3 * (t_end - t0) / len(reqs), 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f64+" + ("fp32|tf32x3" if args.precision == "auto" else args.precision),
        "data": "synthetic (seeded Q1 meshes, loads, Poisson arrivals; no datasets)",
        "config": {"workload": WORKLOADS["c5"], "name": "c5", "requests": len(reqs), "rate_per_s": args.rate,
                   "slots": args.slots, "batch": args.batch, "mem_budget_bytes": args.mem_budget,
                   "precision": args.precision,
                   "block_k": args.k},
        "latency_ms": {"p50": round(float(np.percentile(lat_a, 50)), 3),
                       "p99": round(float(np.percentile(lat_a, 99)), 3), "max": round(float(lat_a.max()), 3)},
        "converged": conv, "library_setup_s": round(lib_s, 3),
        "sequential_fp64": {"sample": ns, "block_k": seq_k, "solves_per_s": round(ns / sum(ts), 3) if ts else None,
                            "mean_ms": round(1e3 * float(np.mean(ts)), 3) if ts else None},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32", "tf32x3", "bf16x3", "auto"],
                    help="local-product arithmetic (default per workload: c3 bf16x3, c2 fp32, c4/c5 auto)")
    ap.add_argument("--k", type=int, default=None, help="multivector width (default per workload: c3 4, c2 8, c4 autotuned)")
    ap.add_argument("--inner-tol", type=float, default=0.0,
                    help="relative tolerance of the inner solves; 0 = the library's per-precision default")
    ap.add_argument("--workload", default="c3", choices=list(WORKLOADS))
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-reference", action="store_true")
    ap.add_argument("--history-gb", type=float, default=None,
                    help="cap on the direction history (GB); 0 = the library default (half of free memory); "
                         "default per workload: c3 32, c4 32, others 0")
    ap.add_argument("--requests", type=int, default=1000, help="serving workload: number of structures")
    ap.add_argument("--rate", type=float, default=50.0, help="serving workload: mean arrivals per second")
    ap.add_argument("--slots", type=int, default=4, help="serving workload: concurrent structures")
    ap.add_argument("--mem-budget", type=int, default=64 << 30, help="serving workload: device-memory budget")
    ap.add_argument("--seq-sample", type=int, default=40, help="serving workload: requests timed sequentially")
    ap.add_argument("--batch", type=int, default=1,
                    help="serving workload: structures of one pattern a slot may solve together (1 = none)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    d_prec, d_k, d_hist = DEFAULTS[args.workload]
    args.precision = args.precision or d_prec
    args.k = args.k or d_k
    args.history_gb = d_hist if args.history_gb is None else args.history_gb
    rank, world, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.workload == "c5":
        out = run_serving(args) if rank == 0 else None
    else:
        out = run_ours(args, rank, world, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
