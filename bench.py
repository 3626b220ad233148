#!/usr/bin/env python
"""Benchmark: flux solves per second of the block low-rank cavity-radiation
hot path on one GB300 (or N independent replicas, one per GPU).

Headline workload (the closed-cylinder cavity): 19,936 inward-facing
triangles (R = 1, H = 4), emissivity U[0.3, 0.9], 64 temperature fields
U[300, 1200] K, leaf size 64, eta = 1, ACA tol 1e-5 (partial pivoting, stop
checked on a residual probe in every row and column), FP32 storage with FP32
accumulation, GMRES (restart 30) on the reflection system to a relative
residual of 1e-7 with FP64 Krylov vectors.

One step = the whole hot path on inputs resident in device memory: facet
geometry, cluster tree, block tree, dense blocks, ACA, then the flux solve
for all 64 fields (GMRES on 65 right-hand sides: 64 fields + the shared
z = C^-1 eps, and the flux epilogue).  value = fields solved per second.

Timing: W warm-up steps, then K steps between a barrier + synchronize; each
step is bracketed by CUDA events on the launching stream, and a 256 MiB
buffer is written between steps to flush L2 (129 MB).  The timed steps run
without instrumentation; a separate profiled pass of the same steps (CUDA
events around every library kernel, on its launch stream) gives the kernel
table and the dominant kernel's roofline.  nvidia-smi samples clocks during
the timed steps.

Accuracy: the GPU flux and product against the full dense FP64 oracle (all
19,936^2 entries, LAPACK LU), whose timed phases are also the CPU baseline.

The default run adds the other workloads as keys of the same line:
``workloads.sphere_mixed`` (level-6 icosphere, 81,920 facets, BF16 factors +
refinement), ``workloads.batch`` (256 boxes, 3.21 M facets, one handle) and
``workloads.served`` (Poisson stream of 200 requests/s on 12 resident
cavities, continuous batching, p50/p99 latency), each with its plain FP64 GPU
path and its accuracy against exact oracle rows.

--impl reference times the FP64 CPU oracle (dense assembly, LU, flux) on the
host cores on a bounded sample of the same workload, extrapolated to the
full cavity.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
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


def workload_key() -> str:
    return next(k for k, v in WORKLOADS.items() if v is W)


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


FP32_LANES_PER_SM = 128


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


def load_bf16_peak():
    """Dense BF16 tensor throughput (TFLOP/s) sustained over seconds: the
    peak of a kernel timed inside a long step."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["bf16_tflops_sustained"]), "measured"
    except Exception:
        return 1700.0, "fallback"


def sm_count(dev=None) -> int:
    import torch
    return int(torch.cuda.get_device_properties(dev if dev is not None else 0).multi_processor_count)


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip() + f" ({platform.machine()})"
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.machine()


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


def timed_steps(step, steps, stream, flush):
    """CUDA-event time of each of `steps` calls of step(); L2 flushed before
    each.  Returns (times_ms, last result)."""
    import torch
    times, res = [], None
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = step()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        if res is not None and hasattr(res[0], "free"):
            res[0].free()
    return times, res


# ---------------------------------------------------------------- our arm
def run_ours(args, rank: int, world: int, profile_steps: int | None = None, e2e: bool = True):
    """The timed steps (uninstrumented), then a profiled pass of the same
    steps on rank 0.  Returns the measurements."""
    import torch
    import paper_2305_06891_gb300 as rad

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    cav = Work(W)
    n = cav.n
    verts_d = torch.as_tensor(cav.verts, device=dev)
    eps_d = torch.as_tensor(cav.eps, device=dev)
    T_d = torch.as_tensor(cav.T, device=dev).t().contiguous().t()
    q_d = torch.empty((FIELDS, n), dtype=torch.float64, device=dev).t()
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    stats = {}

    def step():
        h = build(rad, cav, verts_d)
        compress(rad, h)
        q, info = solve(rad, h, eps_d, T_d, q=q_d)
        stats.update(rad.rad_htree_get_stats(h))
        return h, info

    timed_steps(step, args.warmup, stream, flush)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    clocks.start()
    launches0 = rad.rad_launch_count()
    times, (_, info) = timed_steps(step, args.steps, stream, flush)
    launches = rad.rad_launch_count() - launches0
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(times), dev) if world > 1 else sum(times)

    # ---- profiled pass (not timed for the value): per-kernel CUDA events
    prof, prof_times = {}, []
    if rank == 0:
        k = profile_steps or min(args.steps, 5)
        # a pass that ran far slower than the timed steps (a disturbance of
        # the GPU or the host while it ran) is taken again, once: its per-kernel
        # table is what the roofline and the kernel shares are read from
        for attempt in range(2):
            rad.rad_profile_enable(True)
            prof_times, _ = timed_steps(step, k, stream, flush)
            torch.cuda.synchronize()
            prof = rad.rad_profile_read()
            rad.rad_profile_enable(False)
            if statistics.median(prof_times) <= 1.5 * statistics.median(times):
                break
    extra = {}
    if rank == 0:
        extra = measure_extras(args, rad, torch, dev, cav, verts_d, flush, stream, e2e=e2e)
    return dict(times=times, total_ms=total_ms, info=info, stats=stats, prof=prof, prof_times=prof_times,
                launches=launches, clocks=clk, extra=extra, n=n, cav=cav, dev=dev)


def measure_extras(args, rad, torch, dev, cav, verts_d, flush, stream, e2e=True):
    out = {}
    n = cav.n
    # single-RHS block matvec on the bench operator (HBM bound): plain
    # launches timed per kernel, then the autotuned, graph-replayed call
    h = build(rad, cav, verts_d)
    compress(rad, h)
    st = rad.rad_htree_get_stats(h)
    fdt = torch.float64 if W["near"] == "f64" else torch.float32
    x = torch.as_tensor(SIGMA * cav.T[:, 0] ** 4, device=dev, dtype=fdt)
    y = torch.empty(n, dtype=fdt, device=dev)
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
        info = None
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
    if e2e:
        verts_h = np.ascontiguousarray(cav.verts)
        T_h = np.asfortranarray(cav.T)
        q_h = np.empty((n, FIELDS), order="F")
        ts = []
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
                ts.append(t1 - t0)
        out["e2e"] = {"value": cav.solves / statistics.median(ts), "unit": UNIT,
                      "h2d_bytes_per_step": int(verts_h.nbytes + cav.eps.nbytes + T_h.nbytes),
                      "d2h_bytes_per_step": int(q_h.nbytes), "ms_per_step": 1e3 * statistics.median(ts)}
    return out


# DRAM bytes (read + write) per launch of a workload's dominant kernel on a
# product path (0 CUDA cores, 1 tensor cores), from the ncu capture
# summarised in profiles/ (kept only while the kernel is unchanged since that
# capture).
TRAFFIC = {("cylinder", "hmm_rows", 1): 524.12e6 + 9.98e6,
           ("cylinder", "hmm_far_vt", 1): 253.13e6 + 69.50e6}


def roofline(prof: dict, st: dict, steps: int, nc: int, sms: int):
    """Dominant kernel of the profiled steps and its roofline."""
    hbm, smax, src = load_peaks()
    if not prof:
        return None
    name, (cnt, ms) = max(prof.items(), key=lambda kv: kv[1][1])
    path = int(st.get("product_path", 0))
    traffic = TRAFFIC.get((workload_key(), name, path))
    avg_s = ms / cnt * 1e-3
    fp32_peak = sms * FP32_LANES_PER_SM * 2 * smax * 1e6 / 1e12
    note = f"FP32 FFMA: {sms} SMs x {FP32_LANES_PER_SM} lanes x 2 x {smax:.0f} MHz (of derived)"
    base = {"kernel": name, "launches": cnt, "avg_ms": ms / cnt,
            "measured": f"CUDA events around every launch on its stream, profiled pass of {steps} steps"}
    if name in ("hmm_rows", "hmm_far_vt") and path == 1:
        # tensor cores: every FP32 operand in three BF16 pieces, six BF16
        # partial products per FP32 multiply-add (padding not counted)
        ents = st["near_entries"] + st["far_u_entries"] if name == "hmm_rows" else st["far_v_entries"]
        flops = 6 * 2.0 * nc * ents
        ach = flops / avg_s / 1e12
        bf16, bsrc = load_bf16_peak()
        return dict(base, bound="tensor", achieved=ach, peak=bf16, unit="TFLOP/s", frac=ach / bf16, traffic=traffic,
                    peak_note=f"dense BF16, sustained (of {bsrc}); achieved counts the six BF16 partial products of "
                              "the three-way split per FP32 multiply-add")
    if name == "hmm_rows":
        flops = 2.0 * nc * (st["near_entries"] + st["far_u_entries"])
        ach = flops / avg_s / 1e12
        return dict(base, bound="alu", achieved=ach, peak=fp32_peak, unit="TFLOP/s", frac=ach / fp32_peak,
                    traffic=traffic, peak_note=note)
    if name == "hmm_far_vt":
        flops = 2.0 * nc * st["far_v_entries"]
        ach = flops / avg_s / 1e12
        return dict(base, bound="alu", achieved=ach, peak=fp32_peak, unit="TFLOP/s", frac=ach / fp32_peak,
                    traffic=traffic, peak_note=note)
    if name in ("aca_partial", "near_assemble"):
        # view-factor entry evaluations: ~ 24 FP32 + 3 FP64 operations each
        ents = st["aca_entries"] if name == "aca_partial" else st["near_entries"]
        ach = 27.0 * ents / avg_s / 1e12
        return dict(base, bound="alu", achieved=ach, peak=fp32_peak, unit="TFLOP/s", frac=ach / fp32_peak,
                    traffic=None, peak_note="entry evaluations x 27 flops vs " + note)
    # vector-bound GMRES kernels and the rest: HBM
    return dict(base, bound="hbm", achieved=None, peak=hbm, unit="GB/s", frac=None, traffic=None)


# ---------------------------------------------------------------- oracle
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


def _oracle_coeffs(cav, rows_sample, lu_n, seed, fields=None):
    """Time the oracle on one cavity: F assembly on `rows_sample` rows, and the
    direct solve + flux on its first `lu_n` facets.  Returns per-unit costs
    (seconds per F entry, per n^3 of the LU, per n^2 and column of a product)
    and a description."""
    from oracle import geometry, radiosity, viewfactor
    fields = FIELDS if fields is None else fields
    n = cav.n
    f = geometry.facets_from_triangles(cav.verts)
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(n, rows_sample, replace=False))
    t0 = time.perf_counter()
    viewfactor.rows(f, rows)
    a = (time.perf_counter() - t0) / (rows_sample * n)
    sub = np.arange(lu_n)
    Fs = viewfactor.dense(f.subset(sub))
    T = cav.T[sub, :fields]
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
    c = t_mm / (lu_n ** 2 * (fields + 1))
    desc = (f"F rows {rows_sample}/{n} of a {n}-facet cavity (assembly x n^2); direct solve + flux on its "
            f"leading {lu_n} facets (LU x n^3, F@[Y z] x n^2); {fields} field(s) per cavity")
    return a, b, c, desc


def dense_oracle(work):
    """The whole step by the FP64 oracle on the full cavity, timed by phase:
    dense assembly of every F entry, the direct LU solve of C [Y z] = [eps
    eta, eps] with the flux of Eq. (12), and the flux products F [Y z] alone
    (timed again to split the LU from the products).  Also the exact
    products F X (X = sigma T^4) for the accuracy check."""
    from oracle import geometry, radiosity, viewfactor
    c = work.cavs[0]
    f = geometry.facets_from_triangles(c.verts)
    t0 = time.perf_counter()
    F = viewfactor.dense(f)
    t_asm = time.perf_counter() - t0
    t0 = time.perf_counter()
    q, Y, z = radiosity.solve_flux(F, c.eps, c.T[:, :FIELDS], SIGMA)
    t_solve = time.perf_counter() - t0
    t0 = time.perf_counter()
    _ = F @ np.concatenate([Y, z[:, None]], axis=1)
    t_mm = time.perf_counter() - t0
    Yx = F @ (SIGMA * c.T[:, :FIELDS] ** 4)
    del F
    phases = {"assembly_s": t_asm, "lu_solve_s": max(t_solve - t_mm, 0.0), "flux_products_s": t_mm}
    return q, Yx, phases


def single_thread_sample(n_sub=3072):
    """The oracle phases on the leading `n_sub` facets of the workload's
    (first) cavity in a child process limited to one BLAS thread."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", str(n_sub), "--workload", workload_key()]
    try:
        r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=600)
        return json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as e:
        return {"error": str(e)[:200]}


def oracle_sample_main(n_sub):
    from oracle import geometry, radiosity, viewfactor
    c = Work(W).cavs[0]
    sub = np.arange(min(n_sub, c.n))
    f = geometry.facets_from_triangles(c.verts[sub])
    t0 = time.perf_counter()
    F = viewfactor.dense(f)
    t_asm = time.perf_counter() - t0
    t0 = time.perf_counter()
    q, Y, z = radiosity.solve_flux(F, c.eps[sub], c.T[sub, :FIELDS], SIGMA)
    t_solve = time.perf_counter() - t0
    t0 = time.perf_counter()
    _ = F @ np.concatenate([Y, z[:, None]], axis=1)
    t_mm = time.perf_counter() - t0
    m = len(sub)
    N = c.n
    # extrapolation to the full cavity: assembly and products x (N/m)^2, LU x (N/m)^3
    full = t_asm * (N / m) ** 2 + max(t_solve - t_mm, 0.0) * (N / m) ** 3 + t_mm * (N / m) ** 2
    print(json.dumps({"facets": m, "threads": 1, "assembly_s": t_asm, "lu_solve_s": max(t_solve - t_mm, 0.0),
                      "flux_products_s": t_mm, "full_step_s_extrapolated": full,
                      "value_extrapolated": FIELDS / full, "unit": UNIT}))


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def max_field_err(a, b):
    return float(max(np.linalg.norm(a[:, j] - b[:, j]) / np.linalg.norm(b[:, j]) for j in range(b.shape[1])))


def gpu_solutions(work, fac, near, acc, refine, recompress):
    """Flux of all fields and the product F X (X = sigma T^4) from the GPU
    with the given storage, as host arrays."""
    import torch
    import paper_2305_06891_gb300 as rad
    dev = torch.device("cuda", torch.cuda.current_device())
    h = build(rad, work, torch.as_tensor(work.verts, device=dev))
    rad.rad_compress_aca(h, ACA_TOL, 64, "partial", fac, near, accurate_dtype=acc, recompress_tol=recompress)
    q, info = rad.rad_solve_flux(h, work.eps, np.asfortranarray(work.T), SIGMA, tol=SOLVE_TOL, restart=RESTART,
                                 max_iter=600, refine=refine, inner_tol=1e-4)
    X = SIGMA * work.T ** 4
    xdt = torch.float64 if near == "f64" else torch.float32
    Y = rad.rad_hmatvec(h, torch.as_tensor(np.ascontiguousarray(X), device=dev, dtype=xdt)).cpu().numpy()
    h.free()
    return np.asarray(q), Y, info


def dense_accuracy_and_baseline(work, args):
    """Accuracy of the GPU flux and product against the full dense FP64
    oracle, and the oracle's own timed phases (the CPU baseline)."""
    cores = os.cpu_count()
    q_ref, Y_ref, phases = dense_oracle(work)
    step_s = sum(phases.values())
    paths = {"ours": (W["factor"], W["near"], W["accurate"], W["refine"], RECOMPRESS)}
    if not args.no_fp64:
        paths["fp64_path"] = ("f64", "f64", None, False, 0.0)
    acc = {"oracle": f"full dense FP64: all {work.n}^2 entries of F (centroid rule), LAPACK LU of C, Eq. (12)",
           "error": "||v - v_ref||_2 / ||v_ref||_2 over all facets and fields; max over fields of the same per field"}
    for label, (fac, near, a, refine, rc) in paths.items():
        q, Y, info = gpu_solutions(work, fac, near, a, refine, rc)
        acc[label] = {"flux_rel_err": rel_err(q, q_ref), "flux_rel_err_max_field": max_field_err(q, q_ref),
                      "product_rel_err": rel_err(Y, Y_ref), "product_rel_err_max_field": max_field_err(Y, Y_ref),
                      "solver_rel_residual": info["max_rel_residual"]}
    st1 = single_thread_sample()
    base = {"value": work.solves / step_s, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"the whole step on the full cavity, measured (not extrapolated): dense assembly of "
                       f"{work.n}^2 entries, LU solve of {FIELDS + 1} right-hand sides, flux products; "
                       f"numpy/LAPACK with {cores} threads"),
            "cpu_model": cpu_model(), "phases_s": phases, "step_s": step_s, "single_thread": st1}
    return acc, base


def accuracy_vs_oracle(work, samples=512, cols=4, seed=7, no_fp64=False):
    """Error of the GPU solves against the FP64 oracle on cavities too large
    to assemble densely: the reflection system C Y = B (Eq. 11) is solved on
    the GPU with the workload's settings (and with the plain FP64 path), and
    the residual B - C Y is evaluated on `samples` random rows with exact
    FP64 rows of F.  Reported as max over rows and columns of |r_i| / max|b|
    per column (per cavity for a batch), with the error bound
    ||e||_inf <= ||r||_inf / (1 - max(1 - eps) max_i sum_j F_ij) from the
    exact row sums of the sampled rows."""
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
    smax = 0.0
    for k in np.unique(cav_of):
        c = work.cavs[k]
        loc = rows[cav_of == k] - work.off[k]
        Fr = viewfactor.rows(geometry.facets_from_triangles(c.verts), loc)
        exact[k] = (rows[cav_of == k], Fr)
        smax = max(smax, float(Fr.sum(axis=1).max()))
    rho = float((1.0 - work.eps).max())
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
        out[label] = {"max_rel_residual_exact_rows": worst, "solver_rel_residual": info["max_rel_residual"],
                      "error_bound": worst / max(1e-300, 1.0 - rho * smax)}
    out["bound_terms"] = {"max_one_minus_eps": rho, "max_exact_row_sum": smax}
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
    desc = ""
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
                             "wall_s": elapsed, "cpu_model": cpu_model(),
                             "note": "ms_per_step is the oracle's time for one whole step, extrapolated from the "
                                     "bounded sample each step times"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dict(work=None):
    d = {"workload": W["name"], "fields": FIELDS, "leaf_size": LEAF, "eta_adm": ETA, "aca_tol": ACA_TOL,
         "aca_pivoting": "partial, stop checked on a residual probe in every row and column",
         "recompress_tol": RECOMPRESS,
         "solve_tol": SOLVE_TOL, "gmres_restart": RESTART,
         "storage": f"{W['near']} near + {W['factor']} factors",
         "accumulation": ("f64 (operator, Krylov, inner products)" if W["near"] == "f64" else
                          "f32 (operator), f64 (Krylov, inner products, residuals)"),
         "l2": "flushed between timed steps (256 MiB write)", "parallelism": "replicas"}
    tc = PRODUCT_PATH == 1 or (PRODUCT_PATH is None and W["near"] != "f64")
    d["many_column_product"] = ("tensor cores (tcgen05): FP32 operands split into three BF16 pieces, six partial "
                                "products, FP32 accumulation" if tc else
                                f"CUDA-core tiles ({'FP64' if W['near'] == 'f64' else 'FP32'} FMA)")
    if work is not None and work.batch:
        d["cavities"] = len(work.counts)
        d["facets_total"] = work.n
        d["solves_per_step"] = work.solves
        d["handle"] = "one batch handle (forest of cluster trees), per-cavity Krylov problems"
    if W["refine"]:
        d["refinement"] = f"{W['accurate']} accurate operator, double-float (FP64-grade) residual accumulation, inner GMRES tol 1e-4"
    return d


def kernel_tables(prof, steps):
    kern = {k: v for k, v in prof.items() if not k.startswith("host_")}
    host = {k: v[1] / steps for k, v in prof.items() if k.startswith("host_")}
    return ({k: v[1] / steps for k, v in sorted(kern.items(), key=lambda kv: -kv[1][1])},
            dict(sorted(host.items(), key=lambda kv: -kv[1])), kern)


def solver_workload_summary(name, args):
    """A secondary solver workload (sphere-mixed or batch), measured like the
    headline: timed steps, the plain FP64 GPU path, accuracy on exact oracle
    rows, the oracle's bounded-sample time."""
    import torch
    select_workload(name)
    steps = max(3, min(args.steps, 5 if name == "batch" else 10))
    r = run_ours(argparse.Namespace(**dict(vars(args), steps=steps, warmup=2)), 0, 1, profile_steps=1,
                 e2e=name != "batch")
    ms = r["total_ms"] / steps
    value = r["cav"].solves / (ms * 1e-3)
    kern, host, _ = kernel_tables(r["prof"], 1)
    d = {"metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": ms, "steps": steps, "warmup": 2,
         "dtype": "f32" if W["factor"] == "f32" else "bf16+f32", "config": config_dict(r["cav"]),
         "gpu_launches": int(r["launches"]), "clocks": r["clocks"],
         "gmres": {k: r["info"][k] for k in ("iters", "restarts", "matvecs", "max_rel_residual", "refinements")},
         "kernels_ms_per_step": dict(list(kern.items())[:8]),
         "hmatvec": r["extra"].get("hmatvec")}
    if "fp64_path" in r["extra"]:
        d["fp64_path"] = r["extra"]["fp64_path"]
        d["speedup_vs_fp64_gpu"] = value / r["extra"]["fp64_path"]["value"]
    if "e2e" in r["extra"]:
        d["e2e"] = r["extra"]["e2e"]
    if not args.no_cpu_baseline:
        t, desc = oracle_step(r["cav"])
        d["cpu_baseline"] = {"value": r["cav"].solves / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": desc + " (extrapolated)"}
        d["accuracy"] = accuracy_vs_oracle(r["cav"], no_fp64=args.no_fp64 or r["cav"].batch)
    torch.cuda.empty_cache()
    return d


def served_summary(args, steps=None):
    """The served workload: one pass of the request stream warms the server
    (builds every operator); each timed pass replays the stream with its
    arrival times through the public server API (host arrays in and out)."""
    import torch
    import paper_2305_06891_gb300 as rad
    select_workload("served")
    steps = steps or args.steps
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
    for _ in range(steps):
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
    h2d = sum(e.nbytes + T.nbytes for _, _, e, T in reqs) * steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16+f32", "data": "synthetic",
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
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": int(h2d // steps),
                "d2h_bytes_per_step": int(sum(T.nbytes for _, _, _, T in reqs)),
                "note": "the served value itself is end to end: host arrays through rad_server_submit/wait"},
        "max_rel_residual": float(max(i["max_rel_residual"] for i in infos)),
    }
    if fp64:
        line["fp64_path"] = fp64
        line["speedup_vs_fp64_gpu"] = value / fp64["value"]
        line["speedup_vs_fp64_gpu_at_capacity"] = (len(reqs) / burst) / fp64["value"]
    if not args.no_cpu_baseline:
        t, desc = served_oracle_estimate(pool, reqs)
        line["cpu_baseline"] = {"value": len(reqs) / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": desc}
    torch.cuda.empty_cache()
    return line


def hlu_summary(args):
    """The block LU of C (paper §5.1-5.2) on two operators: the unit cube
    (768 facets, FP64, eps_rel 1e-4) and the headline cylinder (19,936
    facets, FP32, eps_rel 1e-3): factor time and storage, one substitution,
    and the flux solve with and without the factors as GMRES preconditioner.
    The cube's direct apply is checked against the oracle's dense solve."""
    import torch
    import paper_2305_06891_gb300 as rad
    from oracle import geometry, radiosity, viewfactor
    dev = torch.device("cuda", 0)
    out = {}
    cases = (("cube_768_f64", cv.config1(), 32, 1e-8, "f64", 1e-4, 1e-10, 1),
             ("cylinder_19936_f32", cv.config2(m=64), 64, 1e-5, "f32", 1e-3, 1e-7, 64))
    for name, c, leaf, acatol, dt, lutol, stol, fields in cases:
        h = rad.rad_build_htree(torch.as_tensor(c.verts, device=dev), leaf, 1.0)
        rad.rad_compress_aca(h, acatol, 64, "partial", dt, dt)
        ed = torch.as_tensor(c.eps, device=dev)
        Td = torch.as_tensor(np.asfortranarray(c.T[:, :fields]), device=dev)
        fms = []
        lu = None
        for _ in range(3):
            if lu is not None:
                lu.free()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lu = rad.rad_hlu_factor(h, ed, lutol)
            fms.append(1e3 * (time.perf_counter() - t0))
        st = rad.rad_hlu_get_stats(lu)
        b = torch.as_tensor(np.random.default_rng(0).uniform(size=(c.n, fields + 1)), device=dev)
        sms = []
        for _ in range(4):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x = rad.rad_hlu_solve(lu, b)
            torch.cuda.synchronize()
            sms.append(1e3 * (time.perf_counter() - t0))
        d = {"facets": c.n, "precision": dt, "eps_rel": lutol, "factor_ms": statistics.median(fms),
             "stored_entries": st["dense_entries"] + st["lowrank_entries"], "dense_lu_entries": c.n * c.n,
             "lowrank_leaves": st["n_lowrank"], "max_rank": st["max_rank"],
             "substitution_ms": statistics.median(sms[1:]), "substitution_steps": st["solve_launches"],
             "substitution_columns": fields + 1}
        for label, pre in (("gmres", None), ("gmres_hlu_preconditioned", lu)):
            rad.rad_solve_flux(h, ed, Td, SIGMA, tol=stol, restart=RESTART, max_iter=600, precond=pre)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            q, info = rad.rad_solve_flux(h, ed, Td, SIGMA, tol=stol, restart=RESTART, max_iter=600, precond=pre)
            torch.cuda.synchronize()
            ms = 1e3 * (time.perf_counter() - t0)
            d[label] = {"iters": info["iters"], "ms": ms, "solves_per_s": fields / (ms * 1e-3),
                        "max_rel_residual": info["max_rel_residual"]}
        if c.n <= 5000:
            F = viewfactor.dense(geometry.facets_from_triangles(c.verts))
            C = radiosity.reflection_matrix(F, c.eps)
            xe = np.linalg.solve(C, b.cpu().numpy())
            d["direct_apply_rel_err"] = rel_err(x.cpu().numpy(), xe)
        out[name] = d
        lu.free()
        h.free()
    return out


def served_oracle_estimate(pool, reqs, seed=0):
    """The oracle factors each request's cavity (no reuse); per-unit costs
    measured on a bounded sample of the median pool cavity, extrapolated to
    every request's cavity by its size.  Returns (seconds, description)."""
    sizes = sorted(v.shape[0] for v in pool)
    probe_n = sizes[len(sizes) // 2]
    probe_v = next(v for v in pool if v.shape[0] == probe_n)
    rng = np.random.default_rng(seed)
    probe = cv.Cavity("probe", probe_v, rng.uniform(0.3, 0.9, probe_n), rng.uniform(300, 1200, (probe_n, 1)), {})
    a, b, c, desc = _oracle_coeffs(probe, min(1024, probe_n), min(3072, probe_n), seed, fields=1)
    t = sum(a * pool[k].shape[0] ** 2 + b * pool[k].shape[0] ** 3 + 4.0 * c * pool[k].shape[0] ** 2
            for _, k, _, _ in reqs)
    return t, desc + f"; extrapolated to each of the {len(reqs)} requests' cavities"


def headline_line(args, world, r):
    st = r["stats"]
    ms_per_step = r["total_ms"] / args.steps
    value = job_value(world, args.steps, r["total_ms"], r["cav"].solves)
    nc = FIELDS + 1
    ksteps = max(1, len(r["prof_times"]))
    kern, host, kern_raw = kernel_tables(r["prof"], ksteps)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if W["near"] == "f64" else "f32", "data": "synthetic",
        "config": config_dict(r["cav"]),
        "latency_ms": {"p50": float(np.percentile(r["times"], 50)), "p99": float(np.percentile(r["times"], 99))},
        "gpu_launches": int(r["launches"]),
        "clocks": r["clocks"],
        "roofline": roofline(kern_raw, st, ksteps, nc, sm_count(r["dev"])),
        "profiled_pass": {"steps": ksteps, "ms_per_step": statistics.mean(r["prof_times"]) if r["prof_times"] else None,
                          "note": "kernel and host-phase tables come from this separate, instrumented pass"},
        "kernels_ms_per_step": kern,
        "host_phases_ms_per_step": host,
        "gmres": {k: r["info"][k] for k in ("iters", "restarts", "matvecs", "max_rel_residual")},
        "operator": {k: st[k] for k in ("n_blocks", "n_admissible", "near_entries", "far_entries", "sum_rank",
                                         "max_rank_used", "n_dense_fallback", "bytes_near", "bytes_far")},
    }
    ex = r["extra"]
    line["e2e"] = ex.get("e2e")
    line["hmatvec"] = ex.get("hmatvec")
    if "fp64_path" in ex:
        line["fp64_path"] = ex["fp64_path"]
        line["speedup_vs_fp64_gpu"] = value / world / ex["fp64_path"]["value"]
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-workloads", action="store_true",
                    help="headline line only (skip the sphere, batch and served keys)")
    ap.add_argument("--workload", default="cylinder", choices=sorted(WORKLOADS))
    ap.add_argument("--product-path", type=int, choices=[0, 1], default=None,
                    help="many-column product: 0 CUDA-core tiles, 1 tensor cores (default: library choice)")
    ap.add_argument("--recompress-tol", type=float, default=None,
                    help="truncate every ACA cross at this relative accuracy (default: the workload's setting)")
    ap.add_argument("--oracle-sample", type=int, default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    select_workload(args.workload)
    global PRODUCT_PATH, RECOMPRESS
    PRODUCT_PATH = args.product_path
    RECOMPRESS = W.get("recompress", 0.0) if args.recompress_tol is None else args.recompress_tol
    if args.oracle_sample is not None:
        oracle_sample_main(args.oracle_sample)
        return 0
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))

    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return 0
    if W.get("served"):
        if rank == 0:
            print(json.dumps(served_summary(args)), flush=True)
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
    line = headline_line(args, world, r)
    if not args.no_cpu_baseline:
        if not r["cav"].batch and r["cav"].n <= 40000:
            line["accuracy"], line["cpu_baseline"] = dense_accuracy_and_baseline(r["cav"], args)
        else:
            t, desc = oracle_step(r["cav"])
            line["cpu_baseline"] = {"value": r["cav"].solves / t, "unit": UNIT, "cores": os.cpu_count(),
                                    "kind": "oracle", "sample": desc + " (extrapolated)", "cpu_model": cpu_model()}
            # (a batch's FP64 path would hold a ~100 GB operator: ours only there)
            line["accuracy"] = accuracy_vs_oracle(r["cav"], no_fp64=args.no_fp64 or r["cav"].batch)
    if world == 1 and args.workload == "cylinder" and not args.no_workloads:
        head = args.workload
        wl = {}
        for name, key in (("sphere-mixed", "sphere_mixed"), ("batch", "batch")):
            try:
                wl[key] = solver_workload_summary(name, args)
            except Exception as e:   # report, never hide: the key carries the failure
                wl[key] = {"error": f"{type(e).__name__}: {e}"[:300]}
        try:
            wl["served"] = served_summary(args, steps=3)
        except Exception as e:
            wl["served"] = {"error": f"{type(e).__name__}: {e}"[:300]}
        try:
            wl["hlu"] = hlu_summary(args)
        except Exception as e:
            wl["hlu"] = {"error": f"{type(e).__name__}: {e}"[:300]}
        select_workload(head)
        line["workloads"] = wl
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
