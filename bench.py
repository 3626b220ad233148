#!/usr/bin/env python
"""Benchmark: flux solves per second of the block low-rank cavity-radiation
hot path on one GB300 (or N independent replicas, one per GPU).

Workload (the closed-cylinder cavity): 19,936 inward-facing triangles
(R = 1, H = 4), emissivity U[0.3, 0.9], 64 temperature fields U[300, 1200] K,
leaf size 64, eta = 1, ACA tol 1e-5 (partial pivoting with sampled
verification), FP32 storage with FP32 accumulation, GMRES (restart 30) on the
reflection system to a relative residual of 1e-7 with FP64 Krylov vectors.

One step = the whole hot path on freshly uploaded inputs: facet geometry,
cluster tree, block tree, dense blocks, ACA, then the flux solve for all 64
fields (GMRES on 65 right-hand sides: 64 fields + the shared z = C^-1 eps,
and the flux epilogue).  value = fields solved per second.

Timing: W warm-up steps, then K steps between a barrier + synchronize; each
step is bracketed by CUDA events on the launching stream, and a 256 MiB
buffer is written between steps to flush L2 (129 MB).  The per-kernel
profile (CUDA events inside librad) gives the dominant kernel's duration for
the roofline; nvidia-smi samples clocks during the timed steps.

--impl reference times the FP64 CPU oracle (dense assembly, LU, flux) on the
host cores on a bounded sample of the same workload, extrapolated to the
full cavity.
"""
from __future__ import annotations

import argparse
import json
import math
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

import cavities as cv  # noqa: E402

METRIC = "flux solves/s"
UNIT = "solves/s"
SIGMA = 5.670374419e-8
RESTART = 30

# Workloads.  "cylinder" (the default line): closed cylinder, 19,936 facets,
# 64 fields, FP32 storage.  "sphere-mixed": level-6 icosphere, 81,920 facets,
# one field, BF16 low-rank factors + FP32 dense blocks, refinement with an
# FP32 accurate operator and FP64 residuals to 1e-8.
WORKLOADS = {
    "cylinder": dict(make=lambda: cv.config2(m=64), fields=64, leaf=64, eta=1.0, aca_tol=1e-5, solve_tol=1e-7,
                     factor="f32", near="f32", accurate=None, refine=False,
                     name="closed_cylinder_19936_64fields_fp32"),
    "sphere-mixed": dict(make=cv.config3, fields=1, leaf=64, eta=1.0, aca_tol=1e-6, solve_tol=1e-8,
                         factor="bf16", near="f32", accurate="f32", refine=True,
                         name="icosphere6_81920_1field_bf16_refined"),
    # Poisson stream (200 req/s) of transient-step solves on 12 resident
    # cavities (cubes, cylinders, spheres, 5k-200k facets), flux-solve server
    "served": dict(make=None, served=True, fields=1, leaf=64, eta=1.0, aca_tol=1e-6, solve_tol=1e-8,
                   factor="bf16", near="f32", accurate="f32", refine=True, slots=4, budget_gib=64,
                   name="served_poisson200_12cavities_bf16_refined"),
    # 256 boxes, 2k-40k facets each, one handle (forest), one field each
    "batch": dict(make=cv.config4, batch=True, fields=1, leaf=64, eta=1.0, aca_tol=1e-6, solve_tol=1e-7,
                  factor="f32", near="f32", accurate=None, refine=False,
                  name="batch_256_boxes_3.21M_facets_fp32"),
}
W = WORKLOADS["cylinder"]
FIELDS = W["fields"]
LEAF, ETA, ACA_TOL, SOLVE_TOL = W["leaf"], W["eta"], W["aca_tol"], W["solve_tol"]


def select_workload(name: str):
    global W, FIELDS, LEAF, ETA, ACA_TOL, SOLVE_TOL
    W = WORKLOADS[name]
    FIELDS = W["fields"]
    LEAF, ETA, ACA_TOL, SOLVE_TOL = W["leaf"], W["eta"], W["aca_tol"], W["solve_tol"]


class Work:
    """The workload's inputs: one cavity, or a batch concatenated facet-wise."""

    def __init__(self, W):
        made = W["make"]()
        cavs = made if W.get("batch") else [made]
        self.cavs = cavs
        self.counts = [c.n for c in cavs]
        self.off = np.concatenate([[0], np.cumsum(self.counts)]).astype(np.int64)
        self.verts = np.ascontiguousarray(np.concatenate([c.verts for c in cavs]))
        self.eps = np.concatenate([c.eps for c in cavs])
        self.T = np.concatenate([c.T[:, :W["fields"]] for c in cavs])
        self.n = int(self.off[-1])
        self.batch = bool(W.get("batch"))
        self.solves = W["fields"] * len(cavs)


def build(rad, work, verts):
    if work.batch:
        return rad.rad_build_htree_batch(verts, work.counts, LEAF, ETA)
    return rad.rad_build_htree(verts, LEAF, ETA)


PRODUCT_PATH = None   # --product-path: many-column product kernels (library default when None)
RECOMPRESS = 0.0      # --recompress-tol: truncation of the ACA crosses (0 = off)


def compress(rad, h):
    rad.rad_compress_aca(h, ACA_TOL, 64, "partial", W["factor"], W["near"], accurate_dtype=W["accurate"],
                         recompress_tol=RECOMPRESS)
    if PRODUCT_PATH is not None:
        rad.rad_htree_set_product_path(h, PRODUCT_PATH)


def solve(rad, h, eps, T, q=None):
    return rad.rad_solve_flux(h, eps, T, SIGMA, tol=SOLVE_TOL, restart=RESTART, max_iter=600, q=q,
                              refine=W["refine"], inner_tol=1e-4)
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- ranks
def max_over_ranks(value: float, device=None) -> float:
    """Max of `value` over all ranks of the default process group (replicas
    are timed independently; the job takes as long as its slowest rank)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_value(world: int, steps: int, total_ms: float, solves_per_step: int | None = None) -> float:
    """Whole-job throughput: every rank solves `solves_per_step` fields
    (default FIELDS) per step."""
    per = FIELDS if solves_per_step is None else solves_per_step
    return world * per * steps / (total_ms * 1e-3)


# ---------------------------------------------------------------- our arm
def run_ours(args, rank: int, world: int):
    import torch
    import paper_2305_06891_gb300 as rad

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    cav = Work(W)
    n = cav.n
    T_h = np.asfortranarray(cav.T)
    verts_d = torch.as_tensor(cav.verts, device=dev)
    eps_d = torch.as_tensor(cav.eps, device=dev)
    T_d = torch.as_tensor(cav.T, device=dev).t().contiguous().t()
    q_d = torch.empty((FIELDS, n), dtype=torch.float64, device=dev).t()
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(verts=verts_d, eps=eps_d, T=T_d, q=q_d):
        h = build(rad, cav, verts)
        compress(rad, h)
        q, info = solve(rad, h, eps, T, q=q)
        return h, info

    for _ in range(args.warmup):
        h, info = step()
        h.free()
    torch.cuda.synchronize()

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    clocks.start()
    launches0 = rad.rad_launch_count()
    rad.rad_profile_enable(True)
    times, infos = [], []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h, info = step()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        infos.append(info)
        st = rad.rad_htree_get_stats(h)
        h.free()
    torch.cuda.synchronize()
    prof = rad.rad_profile_read()
    rad.rad_profile_enable(False)
    launches = rad.rad_launch_count() - launches0
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(times), dev) if world > 1 else sum(times)

    # ---- one-off measurements (not in the timed region)
    extra = {}
    if rank == 0:
        extra = measure_extras(args, rad, torch, dev, cav, verts_d, eps_d, T_d, flush, stream)
    return dict(times=times, total_ms=total_ms, infos=infos, stats=st, prof=prof, launches=launches, clocks=clk,
                extra=extra, n=n, cav=cav, T_h=T_h)


def measure_extras(args, rad, torch, dev, cav, verts_d, eps_d, T_d, flush, stream):
    out = {}
    n = cav.n
    # single-RHS block matvec on the bench operator (HBM bound): plain
    # launches timed per kernel, then the autotuned, graph-replayed call
    h = build(rad, cav, verts_d)
    compress(rad, h)
    st = rad.rad_htree_get_stats(h)
    x = torch.as_tensor(SIGMA * cav.T[:, 0] ** 4, device=dev, dtype=torch.float32)
    y = torch.empty(n, dtype=torch.float32, device=dev)
    op_bytes = st["bytes_near"] + st["bytes_far"]   # the operator the product streams
    vec_bytes = 4 * (2 * n + 2 * st["sum_rank"])
    hbm, _, src = load_peaks()
    reps = 20

    def timed_calls(profile: bool):
        for _ in range(3):
            rad.rad_hmatvec(h, x, y)
        ts = []
        if profile:
            rad.rad_profile_enable(True)
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rad.rad_hmatvec(h, x, y)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        prof = {}
        if profile:
            prof = rad.rad_profile_read()
            rad.rad_profile_enable(False)
        return statistics.median(ts), prof

    ms_call, prof = timed_calls(True)
    kern_ms = sum(v[1] for k, v in prof.items() if k.startswith("hmv_")) / reps
    t0 = time.perf_counter()
    tuned = rad.rad_htree_autotune(h)
    tune_s = time.perf_counter() - t0
    ms_graph, _ = timed_calls(False)
    gbs = lambda ms: (op_bytes + vec_bytes) / (ms * 1e-3) / 1e9
    out["hmatvec"] = {
        "unit": "GB/s", "operator_bytes": op_bytes,
        "gbs_kernels": gbs(kern_ms) if kern_ms > 0 else None,
        "gbs_call": gbs(ms_call),
        "gbs_call_tuned_graph": gbs(ms_graph),
        "frac_kernels": gbs(kern_ms) / hbm if kern_ms > 0 else None,
        "frac_call_tuned_graph": gbs(ms_graph) / hbm,
        "peak_gbs": hbm, "peak_kind": src, "ms_kernels": kern_ms, "ms_call_median": ms_call,
        "ms_call_tuned_graph_median": ms_graph, "autotune": tuned, "autotune_s": tune_s,
        "per_kernel_ms": {k: v[1] / reps for k, v in prof.items()}}
    h.free()
    # the plain FP64 GPU path: same step with FP64 storage and arithmetic, one
    # cavity at a time (for a batch: the first 16 cavities, solves/s)
    if not args.no_fp64:
        sample = cav.cavs[:16] if cav.batch else cav.cavs
        ts64 = []
        for it in range(2):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for c in sample:
                vd = torch.as_tensor(c.verts, device=dev)
                h = rad.rad_build_htree(vd, LEAF, ETA)
                rad.rad_compress_aca(h, ACA_TOL, 64, "partial", "f64", "f64")
                q, info = rad.rad_solve_flux(h, torch.as_tensor(c.eps, device=dev),
                                             torch.as_tensor(np.asfortranarray(c.T[:, :FIELDS]), device=dev),
                                             SIGMA, tol=SOLVE_TOL, restart=RESTART, max_iter=600)
                h.free()
            e1.record(stream)
            torch.cuda.synchronize()
            if it:
                ts64.append(e0.elapsed_time(e1))
        solves = FIELDS * len(sample)
        out["fp64_path"] = {"ms_per_step": ts64[0], "value": solves / (ts64[0] * 1e-3), "unit": UNIT,
                            "cavities": len(sample), "gmres_iters": info["iters"],
                            "max_rel_residual": info["max_rel_residual"]}
    # end to end through the C ABI with host buffers (copies inside)
    verts_h = np.ascontiguousarray(cav.verts)
    T_h = np.asfortranarray(cav.T)
    q_h = np.empty((n, FIELDS), order="F")
    e2e = []
    for it in range(max(2, min(args.steps, 5)) + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = build(rad, cav, verts_h)
        compress(rad, h)
        solve(rad, h, cav.eps, T_h, q=q_h)
        t1 = time.perf_counter()
        h.free()
        if it:
            e2e.append(t1 - t0)
    out["e2e"] = {"value": cav.solves / statistics.median(e2e), "unit": UNIT,
                  "h2d_bytes_per_step": int(verts_h.nbytes + cav.eps.nbytes + T_h.nbytes),
                  "d2h_bytes_per_step": int(q_h.nbytes), "ms_per_step": 1e3 * statistics.median(e2e)}
    return out


# DRAM bytes (read + write) per launch of a workload's dominant kernel, from
# the ncu capture summarised in profiles/ (kept only while the kernel is
# unchanged since that capture).
TRAFFIC = {("cylinder", "hmm_rows"): 284.72e6 + 6.27e6}


def roofline(prof: dict, st: dict, steps: int, clocks: dict, nc: int):
    """Dominant kernel of the timed steps and its roofline."""
    hbm, smax, src = load_peaks()
    if not prof:
        return None
    name, (cnt, ms) = max(prof.items(), key=lambda kv: kv[1][1])
    wl = next(k for k, v in WORKLOADS.items() if v is W)
    traffic = TRAFFIC.get((wl, name)) if PRODUCT_PATH in (None, 0) else None
    avg_s = ms / cnt * 1e-3
    fp32_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * smax * 1e6 / 1e12
    if name == "hmm_rows":
        flops = 2.0 * nc * (st["near_entries"] + st["far_u_entries"])
        ach = flops / avg_s / 1e12
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": ach / fp32_peak, "traffic": traffic, "launches": cnt, "avg_ms": ms / cnt,
                "peak_note": f"FP32 FFMA: {SM_COUNT} SMs x {FP32_LANES_PER_SM} lanes x 2 x {smax:.0f} MHz (of derived)"}
    if name == "hmm_far_vt":
        flops = 2.0 * nc * st["far_v_entries"]
        ach = flops / avg_s / 1e12
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": ach / fp32_peak, "traffic": None, "launches": cnt, "avg_ms": ms / cnt,
                "peak_note": f"FP32 FFMA: {SM_COUNT} SMs x {FP32_LANES_PER_SM} lanes x 2 x {smax:.0f} MHz"}
    if name in ("aca_partial", "near_assemble"):
        # view-factor entry evaluations: ~ 24 FP32 + 3 FP64 operations each
        ents = st["aca_entries"] if name == "aca_partial" else st["near_entries"]
        flops = 27.0 * ents / steps * steps
        ach = flops / avg_s / 1e12
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": ach / fp32_peak, "traffic": None, "launches": cnt, "avg_ms": ms / cnt,
                "peak_note": "entry evaluations x 27 flops vs FP32 issue peak"}
    # vector-bound GMRES kernels and the rest: HBM
    return {"kernel": name, "bound": "hbm", "achieved": None, "peak": hbm, "unit": "GB/s", "frac": None,
            "traffic": None, "launches": cnt, "avg_ms": ms / cnt}


# ---------------------------------------------------------------- oracle arm
def oracle_step(work, rows_sample=1024, lu_n=3072, seed=0):
    """Seconds the FP64 oracle needs for one step of the workload (all its
    cavities and fields), measured on a bounded sample and extrapolated:
    returns (seconds, description)."""
    sizes = sorted(work.counts)
    probe = next(c for c in work.cavs if c.n == sizes[len(sizes) // 2])   # median-size cavity
    a, b, c, desc = _oracle_coeffs(probe, min(rows_sample, probe.n), min(lu_n, probe.n), seed)
    total = sum(a * m * m + b * m ** 3 + 2.0 * c * m * m * (FIELDS + 1) for m in work.counts)
    if work.batch:
        desc += f"; extrapolated to the {len(work.counts)} cavities by their sizes"
    return total, desc


def _oracle_coeffs(cav, rows_sample, lu_n, seed):
    """Time the oracle on one cavity: F assembly on `rows_sample` rows, and the
    direct solve + flux on its first `lu_n` facets.  Returns per-unit costs
    (seconds per F entry, per n^3 of the LU, per n^2 and column of a product)
    and a description."""
    from oracle import geometry, radiosity, viewfactor
    n = cav.n
    f = geometry.facets_from_triangles(cav.verts)
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(n, rows_sample, replace=False))
    t0 = time.perf_counter()
    viewfactor.rows(f, rows)
    a = (time.perf_counter() - t0) / (rows_sample * n)
    sub = np.arange(lu_n)
    Fs = viewfactor.dense(f.subset(sub))
    T = cav.T[sub, :FIELDS]
    t0 = time.perf_counter()
    q, Y, z = radiosity.solve_flux(Fs, cav.eps[sub], T, SIGMA)
    t_solve = time.perf_counter() - t0
    # dense LU is O(n^3); the flux products F @ [Y z] are O(n^2): split the
    # measured time into the two by timing the product alone
    t0 = time.perf_counter()
    _ = Fs @ np.concatenate([Y.reshape(lu_n, -1), z[:, None]], axis=1)
    t_mm = time.perf_counter() - t0
    t_lu = max(t_solve - 2 * t_mm, 1e-9)
    b = t_lu / lu_n ** 3
    c = t_mm / (lu_n ** 2 * (FIELDS + 1))
    desc = (f"F rows {rows_sample}/{n} of a {n}-facet cavity (assembly x n^2); direct solve + flux on its "
            f"leading {lu_n} facets (LU x n^3, F@[Y z] x n^2); {FIELDS} field(s) per cavity")
    return a, b, c, desc


def accuracy_vs_oracle(work, samples=512, cols=4, seed=7, no_fp64=False):
    """Error of the GPU solves against the FP64 oracle, stated per result:
    the reflection system C Y = B (Eq. 11) is solved on the GPU with the
    workload's settings (and with the plain FP64 path), and the residual
    B - C Y is evaluated on `samples` random rows with exact FP64 rows of F
    from the oracle.  Reported as max over rows and columns of |r_i| / max|b|
    per column (per cavity for a batch).  Runs on the host beside the CPU
    baseline, outside the timed region."""
    import torch
    import paper_2305_06891_gb300 as rad
    from oracle import geometry, viewfactor
    n = work.n
    eta = SIGMA * np.concatenate([c.T[:, :1] for c in work.cavs]) ** 4 if work.batch else SIGMA * work.T[:, :cols] ** 4
    B = np.asfortranarray(np.concatenate([work.eps[:, None] * eta, work.eps[:, None]], axis=1))
    rows = np.sort(np.random.default_rng(seed).choice(n, min(samples, n), replace=False))
    cav_of = np.searchsorted(work.off, rows, side="right") - 1
    dev = torch.device("cuda", torch.cuda.current_device())
    verts_d = torch.as_tensor(work.verts, device=dev)
    paths = {"ours": (W["factor"], W["near"], W["accurate"], W["refine"])}
    if not no_fp64:
        paths["fp64_path"] = ("f64", "f64", None, False)
    out = {"check": f"residual of C Y = B on {len(rows)} random rows with exact FP64 oracle rows of F; "
                    f"B = [eps*sigma*T^4 for {B.shape[1] - 1} field(s), eps]", "rows": int(len(rows))}
    exact = {}
    for k in np.unique(cav_of):
        c = work.cavs[k]
        loc = rows[cav_of == k] - work.off[k]
        exact[k] = (rows[cav_of == k], viewfactor.rows(geometry.facets_from_triangles(c.verts), loc))
    for label, (fac, near, acc, refine) in paths.items():
        h = build(rad, work, verts_d)
        rad.rad_compress_aca(h, ACA_TOL, 64, "partial", fac, near, accurate_dtype=acc,
                             recompress_tol=RECOMPRESS if label == "ours" else 0.0)
        Y, info = rad.rad_solve_reflection(h, work.eps, B, tol=SOLVE_TOL, restart=RESTART, max_iter=600,
                                           refine=refine, inner_tol=1e-4)
        h.free()
        worst = 0.0
        for k, (glob, Fr) in exact.items():
            o0, o1 = work.off[k], work.off[k + 1]
            R = B[glob] - (Y[glob] - (1.0 - work.eps[glob])[:, None] * (Fr @ Y[o0:o1]))
            worst = max(worst, float((np.abs(R).max(axis=0) / np.abs(B[o0:o1]).max(axis=0)).max()))
        out[label] = {"max_rel_residual_exact_rows": worst, "solver_rel_residual": info["max_rel_residual"]}
    return out


def run_reference(args):
    cores = os.cpu_count()
    if W.get("served"):
        work = None
        pool, reqs = cv.config5_stream()
        est = lambda seed: served_oracle_estimate(pool, reqs, seed)
        solves = len(reqs)
    else:
        work = Work(W)
        est = lambda seed: oracle_step(work, seed=seed)
        solves = work.solves
    for _ in range(args.warmup):
        est(0)
    vals = []
    t0 = time.perf_counter()
    for s in range(args.steps):
        t, desc = est(s)
        vals.append(t)
    elapsed = time.perf_counter() - t0
    t = statistics.median(vals)
    value = solves / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(work),
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": UNIT, "cores": cores, "sample": desc,
                             "wall_s": elapsed},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dict(work=None):
    d = {"workload": W["name"], "fields": FIELDS, "leaf_size": LEAF, "eta_adm": ETA, "aca_tol": ACA_TOL,
         "aca_pivoting": "partial, stop checked on a residual probe in every row and column",
         "recompress_tol": RECOMPRESS,
         "solve_tol": SOLVE_TOL, "gmres_restart": RESTART,
         "storage": f"{W['near']} near + {W['factor']} factors",
         "accumulation": "f32 (operator), f64 (Krylov, inner products, residuals)",
         "l2": "flushed between timed steps (256 MiB write)", "parallelism": "replicas"}
    if work is not None and work.batch:
        d["cavities"] = len(work.counts)
        d["facets_total"] = work.n
        d["solves_per_step"] = work.solves
        d["handle"] = "one batch handle (forest of cluster trees), per-cavity Krylov problems"
    if W["refine"]:
        d["refinement"] = f"{W['accurate']} accurate operator, double-float (FP64-grade) residual accumulation, inner GMRES tol 1e-4"
    return d


def run_served(args):
    """The served workload: one pass of the request stream warms the server
    (builds every operator); each timed step replays the stream with its
    arrival times through the public server API (host arrays in and out)."""
    import torch
    import paper_2305_06891_gb300 as rad
    pool, reqs = cv.config5_stream()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    srv = rad.Server(slots=W["slots"], hbm_budget_bytes=W["budget_gib"] << 30, leaf_size=LEAF, eta_adm=ETA,
                     aca_tol=ACA_TOL, factor_dtype=W["factor"], near_dtype=W["near"],
                     accurate_dtype=W["accurate"], tol=SOLVE_TOL, restart=RESTART, max_iter=600,
                     refine=W["refine"], inner_tol=1e-4, recompress_tol=RECOMPRESS)
    ids = [srv.add_cavity(v) for v in pool]

    def stream():
        t0 = time.perf_counter()
        tickets = []
        for arr, c, e, T in reqs:
            dt = t0 + arr - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets.append(srv.submit(ids[c], e, T, SIGMA))
        infos = [srv.wait(t)[1] for t in tickets]
        return time.perf_counter() - t0, infos

    for _ in range(max(1, args.warmup)):
        stream()
    clocks = ClockSampler(0)
    clocks.start()
    l0 = rad.rad_launch_count()
    walls, infos = [], []
    for _ in range(args.steps):
        w, inf = stream()
        walls.append(w)
        infos += inf
    launches = rad.rad_launch_count() - l0
    clk = clocks.stop()
    st = srv.stats()
    # capacity: the same requests submitted at once (no arrival gaps)
    t0 = time.perf_counter()
    tickets = [srv.submit(ids[c], e, T, SIGMA) for _, c, e, T in reqs]
    for t in tickets:
        srv.wait(t)
    burst = time.perf_counter() - t0
    srv.close()
    lat = np.array([i["latency_ms"] for i in infos])
    total = sum(walls)
    value = len(infos) / total
    # the dominant kernel: one product on the largest pool operator
    big = int(np.argmax([v.shape[0] for v in pool]))
    h = rad.rad_build_htree(torch.as_tensor(pool[big], device=dev), LEAF, ETA)
    rad.rad_compress_aca(h, ACA_TOL, 64, "partial", W["factor"], W["near"], accurate_dtype=W["accurate"],
                         recompress_tol=RECOMPRESS)
    hst = rad.rad_htree_get_stats(h)
    n = pool[big].shape[0]
    x = torch.ones(n, dtype=torch.float32, device=dev)
    y = torch.empty_like(x)
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)
    for _ in range(3):
        rad.rad_hmatvec(h, x, y)
    rad.rad_profile_enable(True)
    for _ in range(20):
        flush.zero_()
        rad.rad_hmatvec(h, x, y)
    torch.cuda.synchronize()
    prof = rad.rad_profile_read()
    rad.rad_profile_enable(False)
    h.free()
    kms = sum(v[1] for k, v in prof.items() if k.startswith("hmv_")) / 20
    op_bytes = hst["bytes_near"] + hst["bytes_far"] + 4 * (2 * n + 2 * hst["sum_rank"])
    hbm, _, src = load_peaks()
    ach = op_bytes / (kms * 1e-3) / 1e9
    # the plain FP64 single-cavity path on the same requests, operators
    # resident (built before timing), one request after another
    fp64 = None
    if not args.no_fp64:
        hs = {}
        for c in sorted(set(c for _, c, _, _ in reqs)):
            hh = rad.rad_build_htree(torch.as_tensor(pool[c], device=dev), LEAF, ETA)
            rad.rad_compress_aca(hh, ACA_TOL, 64, "partial", "f64", "f64")
            hs[c] = hh
        t0 = time.perf_counter()
        for _, c, e, T in reqs:
            rad.rad_solve_flux(hs[c], e, T, SIGMA, tol=SOLVE_TOL, restart=RESTART, max_iter=600)
        t64 = time.perf_counter() - t0
        for hh in hs.values():
            hh.free()
        fp64 = {"value": len(reqs) / t64, "unit": UNIT, "ms_per_request": 1e3 * t64 / len(reqs),
                "note": "FP64 storage and arithmetic, operators resident, requests one after another"}
    h2d = sum(e.nbytes + T.nbytes for _, _, e, T in reqs) * args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(config_dict(), requests_per_step=len(reqs), rate_per_s=200.0, cavities=len(pool),
                       facets=[int(v.shape[0]) for v in pool], slots=W["slots"], hbm_budget_gib=W["budget_gib"]),
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "max": float(lat.max()), "mean_service": float(np.mean([i["service_ms"] for i in infos])),
                       "mean_queue": float(np.mean([i["queue_ms"] for i in infos]))},
        "server": st,
        "capacity": {"value": len(reqs) / burst, "unit": UNIT,
                     "note": "the stream's requests submitted at once; value above is paced by the 200/s arrivals"},
        "gpu_launches": int(launches), "clocks": clk,
        "roofline": {"kernel": "single_phase_a + single_phase_b (one product, largest pool operator)",
                     "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                     "traffic": None, "peak_kind": src, "avg_ms": kms},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": int(h2d // args.steps),
                "d2h_bytes_per_step": int(sum(T.nbytes for _, _, _, T in reqs)),
                "note": "the served value itself is end to end: host arrays through rad_server_submit/wait"},
        "max_rel_residual": float(max(i["max_rel_residual"] for i in infos)),
    }
    if fp64:
        line["fp64_path"] = fp64
        line["speedup_vs_fp64_gpu"] = value / fp64["value"]
    if not args.no_cpu_baseline:
        t, desc = served_oracle_estimate(pool, reqs)
        line["cpu_baseline"] = {"value": len(reqs) / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": desc}
    print(json.dumps(line), flush=True)


def served_oracle_estimate(pool, reqs, seed=0):
    """The oracle factors each request's cavity (no reuse); per-unit costs
    measured on a bounded sample of the median pool cavity, extrapolated to
    every request's cavity by its size.  Returns (seconds, description)."""
    sizes = sorted(v.shape[0] for v in pool)
    probe_n = sizes[len(sizes) // 2]
    probe_v = next(v for v in pool if v.shape[0] == probe_n)
    rng = np.random.default_rng(seed)
    probe = cv.Cavity("probe", probe_v, rng.uniform(0.3, 0.9, probe_n), rng.uniform(300, 1200, (probe_n, 1)), {})
    a, b, c, desc = _oracle_coeffs(probe, min(1024, probe_n), min(3072, probe_n), seed)
    t = sum(a * pool[k].shape[0] ** 2 + b * pool[k].shape[0] ** 3 + 4.0 * c * pool[k].shape[0] ** 2
            for _, k, _, _ in reqs)
    return t, desc + f"; extrapolated to each of the {len(reqs)} requests' cavities"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--workload", default="cylinder", choices=sorted(WORKLOADS))
    ap.add_argument("--product-path", type=int, choices=[0, 1], default=None,
                    help="many-column product: 0 CUDA-core tiles, 1 tensor cores (default: library choice)")
    ap.add_argument("--recompress-tol", type=float, default=None,
                    help="truncate every ACA cross at this relative accuracy (default: the workload's setting)")
    args = ap.parse_args()
    select_workload(args.workload)
    global PRODUCT_PATH, RECOMPRESS
    PRODUCT_PATH = args.product_path
    RECOMPRESS = W.get("recompress", 0.0) if args.recompress_tol is None else args.recompress_tol
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))

    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return 0
    if W.get("served"):
        if rank == 0:
            run_served(args)
        return 0

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    r = run_ours(args, rank, world)
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0
    st = r["stats"]
    times = r["times"]
    ms_per_step = r["total_ms"] / args.steps
    value = job_value(world, args.steps, r["total_ms"], r["cav"].solves)
    nc = FIELDS + 1
    steps = args.steps
    prof = {k: (v[0], v[1]) for k, v in r["prof"].items() if not k.startswith("host_")}
    host = {k: v[1] / args.steps for k, v in r["prof"].items() if k.startswith("host_")}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic", "config": config_dict(r["cav"]),
        "latency_ms": {"p50": float(np.percentile(times, 50)), "p99": float(np.percentile(times, 99))},
        "gpu_launches": int(r["launches"]),
        "clocks": r["clocks"],
        "roofline": roofline(prof, st, steps, r["clocks"], nc),
        "kernels_ms_per_step": {k: v[1] / steps for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])},
        "host_phases_ms_per_step": dict(sorted(host.items(), key=lambda kv: -kv[1])),
        "gmres": {"iters": r["infos"][-1]["iters"], "restarts": r["infos"][-1]["restarts"],
                  "matvecs": r["infos"][-1]["matvecs"], "max_rel_residual": r["infos"][-1]["max_rel_residual"]},
        "operator": {k: st[k] for k in ("n_blocks", "n_admissible", "near_entries", "far_entries", "sum_rank",
                                         "max_rank_used", "n_dense_fallback", "bytes_near", "bytes_far")},
    }
    ex = r["extra"]
    line["e2e"] = ex.get("e2e")
    line["hmatvec"] = ex.get("hmatvec")
    if "fp64_path" in ex:
        line["fp64_path"] = ex["fp64_path"]
        line["speedup_vs_fp64_gpu"] = value / world / ex["fp64_path"]["value"]
    if not args.no_cpu_baseline:
        t, desc = oracle_step(r["cav"])
        line["cpu_baseline"] = {"value": r["cav"].solves / t, "unit": UNIT, "cores": os.cpu_count(),
                                "kind": "oracle", "sample": desc}
        # (a batch's FP64 path would hold a ~100 GB operator: ours only there)
        line["accuracy"] = accuracy_vs_oracle(r["cav"], no_fp64=args.no_fp64 or r["cav"].batch)
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
