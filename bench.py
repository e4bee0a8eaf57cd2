"""Benchmark of the fractional FEM hot path on one GB300 (or N independent replicas).

Headline workload: the convex parallelepiped - the unit cube cut into 24^3 cells x 6 tets
(82,944 tets, 331,776 Gauss points, 12,167 dofs), interior vertices jittered by +-0.15 h,
mapped by [[1, .3, 0], [0, 1, .2], [0, 0, .7]] - with alpha = (1.2, 1.5, 1.9), K = (1, 1, 1),
BF16 split-product contraction with FP32 accumulation, FP32 Cholesky and FP64 iterative
refinement, right-hand sides f = 1 and 16 seeded N(0, 1) columns.  One step = the whole
hot path: mesh records and transverse bins / template (mesh_upload), FP64 path walk +
closed-form derivative tables + contraction (assemble), load vector + factorisation +
refined solve of all 17 columns (solve).  Inputs (vertices, tets, nodal f) are resident
in HBM when the timed region starts; every step uploads, assembles, solves and frees.

metric: Gauss-point paths per second - one path = one Gauss point and one axis, both
directions walked and tabulated - through the whole step.

Sub-records: the 16^3 jittered cube (TF32 split products), the same step in the plain
FP64 form, and a batch of 64 uneven cube meshes with 16 right-hand sides each.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       [--workload parallelepiped24|cube16_jitter] [--precision bf16x3|tf32x3|fp32|fp64]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HEADLINE = "parallelepiped24"
DEFAULT_PRECISION = {"parallelepiped24": "bf16x3", "cube16_jitter": "tf32x3",
                     "parallelepiped16": "bf16x3"}
METRIC = "gauss_point_paths_per_s"
UNIT = "paths/s"
L2_FLUSH_BYTES = 256 << 20     # > 129 MB L2

# Peaks derived from unit counts and clocks (152 SMs, 2,070 MHz maximum SM clock): FP32 lanes
# 128 per SM (one FMA = 2 flops), FP64 rate 1/64 of FP32.  The measured HBM and BF16 peaks
# come from MEASURED_PEAKS.json; TF32 tensor = measured BF16 x the nominal 1.1 : 2.25 ratio.
SMS, SM_GHZ = 152, 2.070
FP32_FMA_TFLOPS = SMS * 128 * 2 * SM_GHZ / 1e3          # 80.5
FP32_ISSUE_TOPS = SMS * 128 * SM_GHZ / 1e3              # 40.3 T FP32 instructions/s
FP64_TFLOPS = FP32_FMA_TFLOPS / 64                      # 1.26
WALK_BYTES_PER_SEGMENT = 160      # one tet record read per walked segment
WALK_FP64_FLOPS_PER_SEGMENT = 25
DF_OPS_PER_PRODUCT = 13           # FP32 instructions of one double-float multiply-add
CHOL_TC_MIN_N = 4096              # the library's blocked tensor-core factorisation from this order


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# DRAM bytes (read + write) per launch from ncu captures of the kernels (summarised under
# profiles/), valid only for the source file they were taken on (sha256) and for the units
# of work of that capture; the bench scales them to its own launch by the units processed
# and reports null when the source has changed since the capture.
TRAFFIC = {
    # ncu capture of one launch on the 16^3 parallelepiped (16,301,215 segments)
    "k_walk_tables": {"source": "walk.cu",
                      "sha256": "f5c92935fc52fb0c9b1330c1e5b8263bad3af43b89dae583d9a101bc5830f08f",
                      "bytes": 189565952 + 598637568, "units": 16301215},
    # ncu capture of one 17-vector double-float launch on the 16^3 parallelepiped (units:
    # 14,392,119 nonzeros of the tables, read once per launch from their two list layouts)
    "k_apply_lists": {"source": "solve.cu",
                      "sha256": "338f5e8603fcac2521983a70e9b21d81327abaefc04680a6d409ed64289638c0",
                      "bytes": 433901312 + 5169152, "units": 14392119},
}

def _source_sha(name):
    try:
        with open(os.path.join(ROOT, "paper_1811_03339_gb300", "csrc", name), "rb") as fh:
            return hashlib.sha256(fh.read()).hexdigest()
    except OSError:
        return None


def measured_traffic(kernel, units):
    """ncu DRAM bytes of one launch of `kernel` scaled to `units` units of work, or None."""
    rec = TRAFFIC.get(kernel)
    if not rec or not units or _source_sha(rec["source"]) != rec["sha256"]:
        return None
    return rec["bytes"] * units / rec["units"]


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest of the ranks' values of x (x itself on one rank): the job takes as long as
    its slowest rank.  A collective when world > 1: every rank calls it."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank_step: float, steps: int, total_ms: float) -> float:
    """Units all ranks processed per second over the slowest rank's time (weak scaling: every
    rank processes the same units each step)."""
    return world * units_per_rank_step * steps / (total_ms / 1e3)


def kernel_rooflines(kms: dict, cnt: dict, n_dof: int, precision: str, peaks: dict,
                     workload: str, tc_factor=None) -> dict:
    """Roofline of every timed kernel class of one profiled step: achieved = algorithmic
    work of the class's launches / their summed CUDA-event time on the launch stream.

    walk_tables  HBM: 160 B (one tet record) per walked segment; FP64 side: 25 flops per
                 segment against the FP64 rate
    split        HBM: per table element 16 B read (L and R pairs) and the four operand halves
                 written (2 B each for BF16, 4 B for TF32); then, where the apply runs from
                 the nonzero lists, their entries (10 B per nonzero of L or W R in each of the
                 row-major and Gauss-point-major layouts), else the dense W R pair (8 B per
                 element)
    contract     tensor: algorithmic flops sum_g 4 nnz(L[g]) nnz(R[g]) per axis (when
                 counted) and the executed split-product MMA flops (3 x 2 D_b^2 G_b)
    factor       FP32 pipe: n^3 / 3 flops
    chain        HBM: one read of the factor's lower triangle (2 n^2 B for FP32) per launch
    apply        FP32 issue: 2 double-float multiply-adds (13 FP32 instructions each) per
                 nonzero table entry (of L and of R) and vector, when the nonzeros are counted
                 (else 4 per dense bin-table element pair)
    """
    out = {}
    hbm = float(peaks["hbm_gbs"])
    elems = cnt["table_bytes"] / 16.0          # table elements (hi + lo pairs) over the axes
    w = kms.get("walk_tables", (0, 0))
    if w[0] > 0:
        segs = cnt["segments"]
        gbs = WALK_BYTES_PER_SEGMENT * segs / (w[0] * 1e-3) / 1e9   # = per launch / launch time
        fl = WALK_FP64_FLOPS_PER_SEGMENT * segs / (w[0] * 1e-3) / 1e12
        out["walk_tables"] = {
            "kernel": "k_walk_tables", "bound": "hbm", "unit": "GB/s", "achieved": gbs,
            "peak": hbm, "frac": gbs / hbm, "launches": w[1], "launch_ms": w[0] / w[1],
            "traffic": measured_traffic("k_walk_tables", segs / w[1]),
            "algorithmic": f"{WALK_BYTES_PER_SEGMENT} B per walked segment x {segs} segments",
            "fp64_tflops": fl, "fp64_peak_tflops": FP64_TFLOPS, "fp64_frac": fl / FP64_TFLOPS}
    s = kms.get("split", (0, 0))
    if s[0] > 0:
        per = 16 + (8 if precision == "bf16x3" else 16 if precision == "tf32x3" else 0)
        snz = cnt.get("table_nnz") or 0
        slists = bool(snz) and cnt.get("apply_lists", True)
        nbytes = per * elems + (2 * 10 * snz if slists else 8 * elems)
        gbs = nbytes / (s[0] * 1e-3) / 1e9
        tail = (f"the nonzero lists, 2 x 10 B per nonzero x {snz} nonzeros" if slists else
                "the dense W R pair, 8 B per element")
        out["split"] = {"kernel": "k_split_ops (+ k_gp_lists)" if slists else "k_split_ops",
                        "bound": "hbm", "unit": "GB/s", "achieved": gbs,
                        "peak": hbm, "frac": gbs / hbm, "launches": s[1],
                        "launch_ms": s[0] / s[1], "traffic": None,
                        "algorithmic": f"{per} B per table element x {elems:.0f} elements, plus "
                                       + tail}
    c = kms.get("contract", (0, 0))
    if c[0] > 0:
        ratio = {"tf32x3": 1.1 / 2.25, "bf16x3": 1.0}.get(precision)
        executed = 3.0 * cnt["contract_flops"]
        if ratio is not None:
            peak = float(peaks.get("bf16_tflops", 1900.0)) * ratio
            ach = executed / (c[0] * 1e-3) / 1e12
            rec = {"kernel": "k_contract_tc", "bound": "tensor", "unit": "TFLOP/s",
                   "achieved": ach, "peak": peak, "frac": ach / peak,
                   "basis": "executed split-product MMA flops (3 x 2 D_b^2 G_b over the bins)"}
        else:
            peak = FP64_TFLOPS if precision == "fp64" else FP32_FMA_TFLOPS
            ach = cnt["contract_flops"] / (c[0] * 1e-3) / 1e12
            rec = {"kernel": "k_contract_simt", "bound": "alu", "unit": "TFLOP/s",
                   "achieved": ach, "peak": peak, "frac": ach / peak,
                   "basis": "dense bin flops 2 D_b^2 G_b"}
        alg = cnt.get("algorithmic_flops")
        if alg:
            rec["algorithmic_tflops"] = alg / (c[0] * 1e-3) / 1e12
            rec["executed_over_algorithmic"] = (executed if ratio is not None
                                                else cnt["contract_flops"]) / alg
        rec.update(launches=c[1], launch_ms=c[0] / c[1], traffic=None)
        out["contract"] = rec
    f = kms.get("factor", (0, 0))
    if f[0] > 0:
        fl = n_dof ** 3 / 3.0
        if tc_factor is None:
            tc_factor = n_dof >= CHOL_TC_MIN_N
        if precision != "fp64" and tc_factor:
            # blocked factorisation: the trailing updates (nearly all of n^3/3) run as three
            # TF32 split products on the tensor cores; the time is the factorisation's wall
            # time on the launch stream (diagonal chain and side-stream update together)
            peak = float(peaks.get("bf16_tflops", 1900.0)) * 1.1 / 2.25
            ach = 3.0 * fl / (f[0] * 1e-3) / 1e12
            out["factor"] = {"kernel": "k_cholp_trail (+ k_cholp_diag, k_cholp_panel)",
                             "bound": "tensor", "unit": "TFLOP/s", "achieved": ach, "peak": peak,
                             "frac": ach / peak, "launches": f[1], "launch_ms": f[0] / f[1],
                             "traffic": None,
                             "algorithmic": f"3 x n^3/3 split-product flops, n = {n_dof}; "
                                            f"{fl / (f[0] * 1e-3) / 1e12:.1f} TFLOP/s of n^3/3"}
        else:
            peak = FP64_TFLOPS if precision == "fp64" else FP32_FMA_TFLOPS
            ach = fl / (f[0] * 1e-3) / 1e12
            out["factor"] = {"kernel": "k_chol_tiles", "bound": "alu", "unit": "TFLOP/s",
                             "achieved": ach, "peak": peak, "frac": ach / peak, "launches": f[1],
                             "launch_ms": f[0] / f[1], "traffic": None,
                             "algorithmic": f"n^3/3 flops, n = {n_dof}",
                             "peak_basis": "CUDA-core FMA rate from unit counts and clocks"}
    ch = kms.get("chain", (0, 0))
    if ch[0] > 0:
        esz = 8 if precision == "fp64" else 4
        byt = esz * n_dof * n_dof / 2.0
        gbs = byt / (ch[0] / ch[1] * 1e-3) / 1e9
        out["chain"] = {"kernel": "k_solve_chain", "bound": "hbm", "unit": "GB/s",
                        "achieved": gbs, "peak": hbm, "frac": gbs / hbm, "launches": ch[1],
                        "launch_ms": ch[0] / ch[1], "traffic": None,
                        "algorithmic": "the factor's lower triangle once per launch"}
    a = kms.get("apply", (0, 0))
    if a[0] > 0 and cnt.get("apply_vectors"):
        nnz = cnt.get("table_nnz")
        if nnz:
            ops = 2 * DF_OPS_PER_PRODUCT * nnz * cnt["apply_vectors"]
            alg = (f"2 double-float multiply-adds ({DF_OPS_PER_PRODUCT} FP32 instructions each) "
                   f"per nonzero table entry and vector, {nnz} nonzeros of L and R, "
                   f"{cnt['apply_vectors']} vector-applies")
        else:
            ops = 4 * DF_OPS_PER_PRODUCT * elems * cnt["apply_vectors"]
            alg = (f"4 double-float multiply-adds ({DF_OPS_PER_PRODUCT} FP32 instructions each) "
                   f"per table element and vector, {elems:.0f} elements, "
                   f"{cnt['apply_vectors']} vector-applies")
        ach = ops / (a[0] * 1e-3) / 1e12
        lists = bool(nnz) and cnt.get("apply_lists", True)
        out["apply"] = {"kernel": "k_apply_lists" if lists else "k_apply_bin", "bound": "alu",
                        "unit": "T FP32 instr/s",
                        "achieved": ach, "peak": FP32_ISSUE_TOPS, "frac": ach / FP32_ISSUE_TOPS,
                        "launches": a[1], "launch_ms": a[0] / a[1],
                        "traffic": measured_traffic("k_apply_lists", nnz) if lists else None,
                        "algorithmic": alg,
                        "bytes_gbs": 16 * elems * cnt["apply_passes"] / (a[0] * 1e-3) / 1e9}
        if nnz:
            out["apply"]["nonzero_fraction_of_bin_tables"] = nnz / (2.0 * elems)
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------------
def _element_sum(o, w, gps, threads):
    """Wall time of the oracle's element sum over the Gauss points `gps`: one call, or with
    threads > 1 that many contiguous slices run at once, one oracle call per thread into its
    own matrix (the oracle's C code keeps no shared mutable state and ctypes releases the
    interpreter lock during a call)."""
    t0 = time.perf_counter()
    if threads <= 1:
        o.assemble_gps(w["alpha"], w["K"], gps)
    else:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(threads) as ex:
            for _ in ex.map(lambda part: o.assemble_gps(w["alpha"], w["K"], part) is None,
                            np.array_split(gps, threads)):
                pass
    return time.perf_counter() - t0


def oracle_sample(workload, mesh, F, gp_stride, n_chol, threads=0):
    """The oracle, as it stands, on a bounded sample of one step of `workload`: the whole
    mesh build, the element sum (walk, tables, sparse outer products) of every gp_stride-th
    Gauss point, the load vector, and a Cholesky factorisation + solve of the right-hand
    sides at size n_chol (an SPD stand-in: the textbook factorisation's arithmetic does not
    depend on the values).  The step time is extrapolated: lines x n_gp / sampled, factor x
    (n / n_chol)^3, solve x (n / n_chol)^2.  Single-threaded C.  With threads > 1 the
    sample's element sum is timed once more on that many threads (`_element_sum`), and
    "est_step_all_s" is the same step with that element sum and the single-threaded rest
    (the oracle's Cholesky is the textbook loop: it has no parallel form)."""
    import oracle
    from paper_1811_03339_gb300 import inputs
    w = inputs.WORKLOADS[workload]
    t0 = time.perf_counter()
    o = oracle.Oracle.from_mesh(mesh)
    t_mesh = time.perf_counter() - t0
    gps = np.arange(0, o.n_gp, gp_stride, dtype=np.int64)
    t_lines = _element_sum(o, w, gps, 1)
    t0 = time.perf_counter()
    o.load(F)
    t_load = time.perf_counter() - t0
    nrhs = 1 if F.ndim == 1 else F.shape[1]
    rng = np.random.default_rng(0)
    B = rng.standard_normal((n_chol, n_chol))
    M = B @ B.T / n_chol + np.eye(n_chol)
    t0 = time.perf_counter()
    Lc = oracle.cholesky(M)
    t_fac = time.perf_counter() - t0
    rhs = rng.standard_normal((n_chol, nrhs))
    t0 = time.perf_counter()
    oracle.chol_solve(Lc, rhs)
    t_sol = time.perf_counter() - t0
    n = o.n_dof
    scale = o.n_gp / len(gps)
    rest = t_mesh + t_load + t_fac * (n / n_chol) ** 3 + t_sol * (n / n_chol) ** 2
    out = {"paths": 3 * o.n_gp, "est_step_s": rest + t_lines * scale,
           "measured_s": t_mesh + t_lines + t_load + t_fac + t_sol,
           "sample": (f"oracle (single-threaded C) on a bounded sample of one {workload} "
                      f"step: mesh build (all {o.n_tets} tets), the element sum of every "
                      f"{gp_stride}-th Gauss point ({len(gps)} of {o.n_gp}, three axes), the "
                      f"load vector of {nrhs} columns, Cholesky + solve at n = {n_chol}; "
                      f"extrapolated to the whole step (lines x {scale:.0f}, "
                      f"factor x (n/{n_chol})^3, solve x (n/{n_chol})^2, n = {n})")}
    if threads > 1:
        t_all = _element_sum(o, w, gps, threads)
        out.update(est_step_all_s=rest + t_all * scale, lines_s=t_lines, lines_all_s=t_all,
                   est_factor_s=t_fac * (n / n_chol) ** 3)
    return out


# the all-core leg's thread count: each thread holds its own dense n x n matrix (1.2 GB at
# 12,167 dofs), so at most eight
def _oracle_threads():
    return max(1, min(8, os.cpu_count() or 1))


def cpu_baseline(workload, mesh, F):
    nt = _oracle_threads()
    try:
        r = oracle_sample(workload, mesh, F, gp_stride=4, n_chol=2048, threads=nt)
    except (MemoryError, OSError):   # a host without room for the threads' matrices
        nt = 1
        r = oracle_sample(workload, mesh, F, gp_stride=4, n_chol=2048)
    out = {"value": r["paths"] / r["est_step_s"], "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": r["sample"] + f"; {r['measured_s']:.1f} s of CPU work, estimated step "
                                   f"{r['est_step_s']:.1f} s"}
    if nt > 1:
        out["all_cores"] = {
            "value": r["paths"] / r["est_step_all_s"], "unit": UNIT, "cores": nt,
            "sample": (f"the same sample with its element sum on {nt} threads (contiguous "
                       f"slices of the sampled Gauss points, one unchanged oracle call per "
                       f"thread): {r['lines_all_s']:.2f} s wall against {r['lines_s']:.2f} s "
                       f"on one core; the mesh build, load vector, Cholesky and solve stay "
                       f"single-threaded (the textbook factorisation, "
                       f"{r['est_factor_s']:.0f} s of the estimated "
                       f"{r['est_step_all_s']:.1f} s step)")}
    return out


def run_reference(args):
    rank, world, _ = _dist_env()
    if rank != 0:
        return 0
    from paper_1811_03339_gb300 import inputs
    workload = args.workload
    mesh = inputs.workload_mesh(workload)
    F = inputs.workload_rhs(workload, mesh)
    est, measured = [], 0.0
    budget = 150.0
    t_start = time.perf_counter()
    sample = ""
    for it in range(args.warmup + args.steps):
        r = oracle_sample(workload, mesh, F, gp_stride=32, n_chol=1024)
        sample = r["sample"]
        if it >= args.warmup:
            est.append(r["est_step_s"])
            measured += r["measured_s"]
        if time.perf_counter() - t_start > budget and est:
            break
    paths = 3 * 4 * mesh.n_tets
    value = paths * len(est) / sum(est)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": world, "steps": len(est), "steps_requested": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(est) / len(est),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload, "tets": int(mesh.n_tets),
                   "gauss_points": 4 * int(mesh.n_tets), "paths_per_step": paths,
                   "alpha": list(inputs.WORKLOADS[workload]["alpha"]),
                   "K": list(inputs.WORKLOADS[workload]["K"])},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample + f"; each step one such sample ({measured / len(est):.1f} s "
                                            f"of CPU work), stopped early after {budget:.0f} s"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------
def _stage_dict(st):
    return dict(zip(["mesh", "bins", "walk_tables", "contract", "load", "factor",
                     "solve_refine"], [round(x, 4) for x in st]))


def measure_workload(args, torch, fem3, inputs, workload, precision, steps, warmup, dev, clk=None,
                     with_fp64=True, with_e2e=False, world=1):
    """Time one workload's step (CUDA events on torch's current stream, L2 flushed between
    steps), then profile one step (stage and kernel-class events) and, optionally, time the
    plain FP64 form and the end-to-end path through the C ABI with host buffers."""
    w = inputs.WORKLOADS[workload]
    mesh = inputs.workload_mesh(workload)
    alpha, K = w["alpha"], w["K"]
    F = inputs.workload_rhs(workload, mesh)
    nrhs = 1 if F.ndim == 1 else F.shape[1]
    verts_d = torch.from_numpy(mesh.verts).to(dev)
    tets_d = torch.from_numpy(mesh.tets).to(dev)
    F_d = torch.from_numpy(np.ascontiguousarray(F)).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    n_paths = 3 * 4 * mesh.n_tets
    stream = torch.cuda.current_stream()

    def step(prec, profile=False, keep=False):
        m = fem3.Mesh(verts_d, tets_d, bin_scale=args.bin_scale, profile=profile,
                      chol_tc=args.chol_tc)
        m.assemble(alpha, K, prec)
        u = m.solve(F_d, tol=args.tol)
        if keep:
            return m, u
        m.free()
        return None, u

    def timed(prec, k, warm):
        for _ in range(warm):
            step(prec)
        times = []
        for _ in range(k):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(prec)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        return times

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if clk is not None:
        with clk:
            times = timed(precision, steps, warmup)
    else:
        times = timed(precision, steps, warmup)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    total = max_over_ranks(sum(times), world, dev)
    out = {"workload": workload, "tets": int(mesh.n_tets), "gauss_points": 4 * int(mesh.n_tets),
           "paths_per_step": n_paths, "rhs_columns": nrhs, "alpha": list(alpha), "K": list(K),
           "precision": precision, "steps": steps, "ms_per_step": total / steps,
           "value": whole_job_rate(world, n_paths, steps, total)}

    # profiled step: stage and kernel-class events, counters
    m, u_mix = step(precision, profile=True, keep=True)
    m.sync()
    kms = m.kernel_ms()
    cnt = m.counters()
    cnt["algorithmic_flops"] = m.contract_work()
    cnt["table_nnz"] = m.table_nnz()
    cnt["apply_lists"] = m.apply_lists()
    out.update(dofs=int(m.n_dof), stages_ms=_stage_dict(m.stage_ms()),
               kernel_ms={k: {"ms": round(v[0], 4), "launches": v[1]} for k, v in kms.items()},
               segments_per_step=cnt["segments"], table_bytes=cnt["table_bytes"],
               gpu_launches_per_step=cnt["launches"],
               refinement={"iterations": m.iters, "final_rel_residual": m.resid,
                           "tol": args.tol},
               bins=[m.bin_stats(a) for a in range(3)], tc_tile=m.tc_tile()[0] or None)
    if precision != "fp64":
        passes = 0
        vecs = 0
        for _ in range(m.iters):
            vecs += nrhs
            passes += (nrhs + 7) // 8
        cnt["apply_vectors"], cnt["apply_passes"] = vecs, passes
    n_dof = m.n_dof
    m.free()
    tc_factor = args.chol_tc == 1 or (args.chol_tc == 0 and n_dof >= CHOL_TC_MIN_N)
    out["rooflines"] = kernel_rooflines(kms, cnt, n_dof, precision, _peaks()[0], workload,
                                        tc_factor)
    if out["rooflines"]:
        dom = max(out["rooflines"], key=lambda k: kms[k][0])
        out["dominant_kernel"] = dom
        out["dominant_share_of_kernel_time"] = kms[dom][0] / sum(v[0] for v in kms.values())

    if with_fp64 and precision != "fp64":
        t64 = timed("fp64", 2, 1)
        m64, u64 = step("fp64", profile=True, keep=True)
        m64.sync()
        out["fp64_form"] = {"ms_per_step": sum(t64) / len(t64),
                            "stages_ms": _stage_dict(m64.stage_ms())}
        m64.free()
        out["mixed_vs_fp64_speedup"] = out["fp64_form"]["ms_per_step"] / out["ms_per_step"]
        du = (u_mix - u64).reshape(-1, nrhs) if nrhs > 1 else (u_mix - u64)
        rel = torch.linalg.norm(du.reshape(-1, nrhs), dim=0) / torch.linalg.norm(
            u64.reshape(-1, nrhs), dim=0)
        out["u_rel_diff_mixed_vs_fp64_max"] = float(rel.max())

    if with_e2e:
        verts_h = torch.from_numpy(mesh.verts).pin_memory()
        tets_h = torch.from_numpy(mesh.tets).pin_memory()
        F_h = torch.from_numpy(np.ascontiguousarray(F)).pin_memory()
        e2e_t = []
        for it in range(warmup + steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mh = fem3.Mesh(verts_h.numpy(), tets_h.numpy(), bin_scale=args.bin_scale,
                           chol_tc=args.chol_tc)
            mh.assemble(alpha, K, precision)
            u = mh.solve(F_h.numpy(), tol=args.tol)
            u_host = u.cpu()
            e1.record(stream)
            torch.cuda.synchronize()
            mh.free()
            if it >= warmup:
                e2e_t.append(e0.elapsed_time(e1))
        out["e2e"] = {"value": whole_job_rate(world, n_paths, len(e2e_t),
                                              max_over_ranks(sum(e2e_t), world, dev)),
                      "unit": UNIT,
                      "h2d_bytes_per_step": int(mesh.verts.nbytes + mesh.tets.nbytes + F.nbytes),
                      "d2h_bytes_per_step": int(u_host.numel() * 8)}
    out["_mesh"] = mesh
    out["_F"] = F
    return out


def run_ours(args):
    import torch

    from paper_1811_03339_gb300 import fem3, inputs

    rank, world, local = _dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    workload = args.workload
    precision = args.precision or DEFAULT_PRECISION[workload]

    clk = ClockSampler(local)
    head = measure_workload(args, torch, fem3, inputs, workload, precision, args.steps,
                            args.warmup, dev, clk=clk, with_fp64=True, with_e2e=True,
                            world=world)
    sub = None
    if not args.no_sub:
        other = "cube16_jitter" if workload != "cube16_jitter" else HEADLINE
        sub = measure_workload(args, torch, fem3, inputs, other, DEFAULT_PRECISION[other],
                               max(5, min(args.steps, 20)), 3, dev, with_fp64=True,
                               world=world)
        for k in ("_mesh", "_F"):
            sub.pop(k)
    batch = None
    if not args.no_batch:
        batch = run_batch(args, torch, fem3, inputs, torch.cuda.current_stream())

    line = None
    if rank == 0:
        peaks, src = _peaks()
        mesh, F = head.pop("_mesh"), head.pop("_F")
        base = (cpu_baseline(workload, mesh, F)
                if (world == 1 and not args.no_cpu_baseline) else None)
        dom = head.get("dominant_kernel")
        roof = dict(head["rooflines"][dom]) if dom else None
        if roof is not None:
            roof["share_of_kernel_time"] = head["dominant_share_of_kernel_time"]
            roof["peak_source"] = ("measured (MEASURED_PEAKS.json)" if roof["unit"] in ("GB/s",)
                                   or roof["bound"] == "tensor" else
                                   "derived from unit counts and the 2,070 MHz clock")
        line = {
            "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"tf32x3": "f64 walk/tables, tf32x3 contraction, f32 factor, f64 refinement",
                      "bf16x3": "f64 walk/tables, bf16x3 contraction, f32 factor, f64 refinement",
                      "fp32": "f64 walk/tables, f32 contraction and factor, f64 refinement",
                      "fp64": "f64"}[precision],
            "data": "synthetic",
            "config": {"workload": workload, "tets": head["tets"],
                       "gauss_points": head["gauss_points"], "dofs": head["dofs"],
                       "paths_per_step": head["paths_per_step"],
                       "rhs_columns": head["rhs_columns"], "alpha": head["alpha"],
                       "K": head["K"], "precision": precision,
                       "parallelism": f"replicas{world}", "bin_scale": args.bin_scale,
                       "l2": "flushed (256 MB write) between timed steps"},
            "e2e": head["e2e"],
            "gpu_launches": head["gpu_launches_per_step"] * args.steps,
            "gpu_launches_note": f"{head['gpu_launches_per_step']} libfem3 kernel launches per "
                                 f"step (library counter)",
            "roofline": roof,
            "cpu_baseline": base,
            "clocks": clk.summary(),
            "fp64_form_ms_per_step": head.get("fp64_form", {}).get("ms_per_step"),
            "mixed_vs_fp64_speedup": head.get("mixed_vs_fp64_speedup"),
            "u_rel_diff_mixed_vs_fp64_max": head.get("u_rel_diff_mixed_vs_fp64_max"),
            "detail": {k: v for k, v in head.items() if k not in ("e2e",)},
            "peaks_source": src,
            "sub_workload": sub,
            "batch": batch,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_batch(args, torch, fem3, inputs, stream):
    """64 cube meshes with n ~ U{6..20} cells per side (6 tets per cell), alpha_i ~
    U(1.1, 1.9) per mesh and axis, K = 1, 16 N(0,1) nodal right-hand sides per mesh;
    mesh records uploaded once; one step = fem3_batch_run (walk, tables, contraction,
    load, factorisation and refinement of every mesh)."""
    specs = inputs.batch_specs(64, seed=3, nmin=6, nmax=20)
    meshes = [inputs.cube_mesh(sp["n"]) for sp in specs]
    alpha = np.array([sp["alpha"] for sp in specs])
    K = np.ones((len(specs), 3))
    fs = [torch.from_numpy(inputs.random_rhs(m.n_nodes, 16, seed=100 + i)).cuda()
          for i, m in enumerate(meshes)]
    paths = sum(3 * 4 * m.n_tets for m in meshes)
    b = fem3.Batch([(m.verts, m.tets) for m in meshes])

    def timed(precision, k, warm):
        for _ in range(warm):
            b.run(alpha, K, fs, precision, tol=args.tol)
        ts = []
        for _ in range(k):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            us = b.run(alpha, K, fs, precision, tol=args.tol)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return sum(ts) / len(ts), us

    ms_mix, u_mix = timed("tf32x3", 3, 1)
    iters = list(b.iters)
    ms_64, u_64 = timed("fp64", 1, 1)
    err = max(float(torch.linalg.norm(a - c) / torch.linalg.norm(c)) for a, c in zip(u_mix, u_64))
    out = {"workload": "64 Kuhn cubes, n ~ U{6..20} cells per side, 16 right-hand sides each",
           "tets": int(sum(m.n_tets for m in meshes)),
           "dofs": int(sum(b.n_dof)), "paths_per_step": paths,
           "ms_per_step": ms_mix, "paths_per_s": paths / (ms_mix / 1e3),
           "fp64_ms_per_step": ms_64, "mixed_vs_fp64_speedup": ms_64 / ms_mix,
           "u_rel_err_mixed_vs_fp64_max": err, "refinement_sweeps_max": max(iters),
           "precision": "tf32x3"}
    b.free()
    return out


def build_parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # about 30 steps of 50-80 ms keep the timed region long enough for several 200 ms
    # clock samples
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=HEADLINE,
                    choices=["parallelepiped24", "cube16_jitter", "parallelepiped16"])
    ap.add_argument("--precision", default=None, choices=["tf32x3", "bf16x3", "fp32", "fp64"],
                    help="default: bf16x3 for the parallelepiped, tf32x3 for the cube")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-mesh batched workload")
    ap.add_argument("--no-sub", action="store_true", help="skip the second workload")
    ap.add_argument("--tol", type=float, default=1e-10,
                    help="relative residual at which refinement stops (the mixed form targets "
                         "1e-8 relative solution error; the FP64 form is direct)")
    ap.add_argument("--chol-tc", type=int, default=0, choices=[-1, 0, 1],
                    help="FP32 factorisation: 1 the blocked tensor-core one, -1 the tile-task "
                         "one, 0 by size (tensor cores from 4,096 dofs)")
    ap.add_argument("--bin-scale", type=float, default=0.5,
                    help="transverse bin width in mean cell sizes (template granularity)")
    return ap


def main():
    args = build_parser().parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
