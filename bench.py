"""Benchmark of the Burton-Miller collocation BEM hot path on one GB300 (or N independent replicas).

Workload (default): star-shaped scatterer r(t) = 1 + 0.3 cos 5t, k_e = 20, k_i = 30 (eps_i = 2.25),
4096 constant elements (8192 complex unknowns), 4-point Gauss-Legendre, 64 incident plane waves
uniform on [0, 2 pi) solved as one multi-right-hand-side block, far field at 32 angles.

One step = the whole hot path on one batch: element geometry, assembly of A, plane-wave right-hand
sides, GMRES solves of all 64 columns to relative residual `--tol`, far fields.  The headline `value`
is the mixed-precision path (complex FP32 storage and Krylov basis, FP64 refinement); the plain FP64
GPU path runs the same step for comparison (`fp64` key).  The CPU oracle solves the whole workload on
the host cores (`cpu_baseline`), and its LU solution is the reference of the `accuracy` key.

The same line carries secondary keys, each with its own clock record: `sweep` (256 random stars solved
as one batch) and `serving` (a Poisson stream of 2000 requests through the continuous-batching loop,
p50/p99 latency), both with an FP64 comparator on identical problems, and `sec7_sweeps` (the iteration
studies of Sec. 7.1 and 7.2: circle, concentric circles and junction disk, GMRES iterations against N,
omega and eps for the proposed and the compared arrangements, one batch each).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--fp64-steps S]
                       [--workload star|sweep|serving|omega_eps] [--no-secondary] [--requests R]
Other workloads print one leg alone: `sweep`, `serving`, and `omega_eps` (the frequency and contrast
sweeps of Sec. 7.1 and 7.2 as batched launches).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "BEM solves/s (mixed vs FP64 GPU at err<=1e-6)"
# Roofline inputs from ncu counts of single launches on the benchmarked star (r = 1 + 0.3 cos 5t, N_e = 4096,
# 64 right-hand sides; profiles/assemble_star4096.md, profiles/gemm_tc_star4096_64rhs.md):
#  * k_assemble issues 3.342e9 warp instructions (smsp__inst_executed.sum) over the FP64 pipe (per-pair
#    geometry, phase k r) and the FP32 pipe (double-float node geometry, Bessel values and Gauss sums); neither
#    pipe alone binds, so its roofline is the issue rate: 4 warp instructions per clock per SM.  Scaled to other
#    sizes by the number of element pairs.  DRAM traffic 1.0159 GB written + 0.95 MB read per launch.
#  * the multi-RHS GEMM streams the FP16 split copy of A once per launch: 2 x 2 bytes per real entry; DRAM
#    traffic 564.2 MB read + 6.4 MB written per launch (a relaxed launch, A's and Bt's hi parts only: 274.0 +
#    6.3 MB), scaled by the matrix size.
#  * the refinement residual runs 16 FP32 operations per complex multiply-add on the FP32 pipe (four exact
#    products summed with an offset accumulator, four operations each; the per-run offsets and the
#    double-float fold are not counted), 128 operations per clock per SM; with the tensor-core product the
#    small terms hi x_lo + lo x_hi are two FP16x3 GEMMs (11 kernels per residual, 12 with a K split).
ASM_WARP_INST_N4096 = 3.34192383e9
ASM_DRAM_BYTES_N4096 = 1.015926e9 + 0.951808e6
GEMM_DRAM_BYTES_N4096 = 564.2304e6 + 6.43072e6
GEMM_DRAM_BYTES_RELAXED_N4096 = 273.995776e6 + 6.288384e6
RESID_FP32_OPS_PER_CMAC = 16
RESID_LAUNCHES_TC = 11
SM_COUNT, SM_CLOCK_HZ = 152, 2.07e9
ISSUE_PEAK_G = SM_COUNT * 4 * SM_CLOCK_HZ / 1e9          # G warp instructions / s
FP32_PEAK_T = SM_COUNT * 128 * SM_CLOCK_HZ / 1e12        # T FP32 thread operations / s
UNIT = "solves/s"
N_RHS = 64
N_FF = 32


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, max clock, throttle reasons, GPU utilisation)."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, util, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
            if len(f) >= 10:
                try:
                    util.append(float(f[9]))
                except ValueError:
                    pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "gpu_util_pct_mean": statistics.mean(util) if util else None}


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    return ws, rank, local


def barrier_max(ws, value):
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------------------------------------
# CPU oracle legs
# ------------------------------------------------------------------------------------------------

def oracle_full(wp, ang, tol, gmres_cols=1, single_rows=128):
    """The oracle on the whole workload, on every host core: the full matrix (rows split over spawned
    processes, the oracle's arithmetic unchanged), the right-hand sides and a direct solve of all columns
    (LAPACK LU, multi-threaded).  Also, for context: the single-process assembly time, extrapolated from
    `single_rows` rows (labelled as such), and the paper's solver (the oracle's unrestarted MGS-GMRES) on
    `gmres_cols` columns.  Returns (timings dict, LU solutions n_rhs x 2N)."""
    import oracle as O
    workers = O.default_workers()
    n2 = 2 * wp.n_elem
    t0 = time.perf_counter()
    A = O.assemble_parallel(wp, Q=4, workers=workers)
    t_asm = time.perf_counter() - t0
    t0 = time.perf_counter()
    el = O.elements(wp)
    Bm = np.stack([O.rhs_planewave(wp, t, el=el) for t in ang], 1)
    X = O.solve_lu(A, Bm).T.copy()
    t_lu = time.perf_counter() - t0
    out = {"cores": workers, "assembly_s": t_asm, "rhs_and_lu_s": t_lu, "n_rhs": len(ang)}
    if single_rows:
        rows = np.linspace(0, n2 - 1, single_rows).astype(int)
        t0 = time.perf_counter()
        O.assemble_rows(wp, rows, Q=4, el=el)
        out["single_process_assembly_s"] = (time.perf_counter() - t0) * n2 / single_rows
        out["single_process_assembly_extrapolated_from_rows"] = single_rows
    if gmres_cols:
        t0 = time.perf_counter()
        its = [O.gmres(A, Bm[:, c], tol=tol)[1] for c in range(gmres_cols)]
        out["gmres_s_per_column"] = (time.perf_counter() - t0) / gmres_cols
        out["gmres_iters"] = its
    return out, X


def run_reference(args):
    """The oracle as the reference arm: every timed step is the whole workload (full assembly on all host
    cores + LU solve of the 64 plane waves); warm-up steps run a small star."""
    ws, rank, _ = dist_setup(args)
    if rank != 0:
        return
    wp = W.cfg_star_c2()
    ang = W.plane_wave_angles(N_RHS)
    small = W.cfg_star_c2(256)
    for _ in range(args.warmup):
        oracle_full(small, ang, args.tol, gmres_cols=0, single_rows=0)
    t = []
    info = {}
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        info, _ = oracle_full(wp, ang, args.tol, gmres_cols=0, single_rows=0)
        t.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(t))
    value = N_RHS / (ms / 1e3)
    sample = (f"the whole workload each step: assembly of all {2 * wp.n_elem} rows on {info['cores']} host "
              f"processes + LU solve of {N_RHS} right-hand sides (not extrapolated)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wp.name, "n_elem": wp.n_elem, "n_rhs": N_RHS},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
                             "sample": sample, "extrapolated": False},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------------
# GPU legs
# ------------------------------------------------------------------------------------------------

def roofline(prof, nel, hbm, src):
    """Roofline entry of the dominant kernel: the phase with the most device time among those with a model.

    prof maps a phase name to (milliseconds, launches) of one profiled step (the "relaxed" entry counts the
    tensor-core products that multiplied the FP16 hi parts alone); nel is the element count of the workload;
    hbm the HBM peak in GB/s and src where it comes from."""
    models = ("assemble", "matvec", "residual")
    ph, (ph_ms, ph_n) = max(((k, v) for k, v in prof.items() if k in models), key=lambda kv: kv[1][0])
    n2 = 2 * nel
    scale = (nel / 4096.0) ** 2
    roof = {"kernel": ph, "launches": ph_n, "avg_launch_ms": ph_ms / ph_n, "traffic": None}
    if ph == "assemble":
        avg_s = ph_ms / ph_n / 1e3
        ach = ASM_WARP_INST_N4096 * scale / avg_s / 1e9
        roof.update({"kernel": "k_assemble (issue-bound: FP64 geometry + double-float Bessel on FP32)", "bound": "alu",
                     "achieved": ach, "peak": ISSUE_PEAK_G, "unit": "G warp instructions/s", "frac": ach / ISSUE_PEAK_G,
                     "traffic": ASM_DRAM_BYTES_N4096 * scale, "algorithmic_bytes_per_launch": 64 * nel * nel,
                     "peak_source": "derived: 152 SMs x 4 issue slots/clk x 2.07 GHz"})
    elif ph == "matvec":
        # one kernel per product: the GEMM (its stream-K reduction is timed as the "reduce" phase); the launch
        # count leaves out the gated launches queued after convergence, which do no work
        # relaxed launches (inexact GMRES: A's FP16 remainder dropped) stream half of A's bytes; the algorithmic
        # bytes and the traffic are the averages over the profiled step's full and relaxed launches
        avg_s = ph_ms / ph_n / 1e3
        n_rel = min(ph_n, prof.get("relaxed", (0.0, 0))[1])
        full_b = n2 * n2 * 8 + 2 * N_RHS * n2 * 8             # A (2 x FP16 per real entry) + X + Y
        rel_b = n2 * n2 * 4 + 2 * N_RHS * n2 * 8              # A's FP16 hi part + X + Y
        bytes_per = ((ph_n - n_rel) * full_b + n_rel * rel_b) / ph_n
        ach = bytes_per / avg_s / 1e9
        traffic = None
        if GEMM_DRAM_BYTES_RELAXED_N4096 is not None:
            traffic = ((ph_n - n_rel) * GEMM_DRAM_BYTES_N4096 + n_rel * GEMM_DRAM_BYTES_RELAXED_N4096) / ph_n * scale
        roof.update({"kernel": "k_gemm_tc (tcgen05 FP16x3 multi-RHS GEMM; its stream-K reduction is the reduce phase)",
                     "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                     "peak_source": src, "algorithmic_bytes_per_launch": bytes_per,
                     "relaxed_launches": n_rel, "full_launches": ph_n - n_rel,
                     "traffic": traffic,
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one full and one relaxed "
                                       "launch at N_e = 4096 (profiles/gemm_tc_star4096_64rhs.md), averaged like the "
                                       "algorithmic bytes and scaled by the matrix size"})
    else:
        # launches per refinement residual: 11 (12 with a K split) with the tensor-core small terms
        n_gemm = max(1, ph_n // RESID_LAUNCHES_TC)
        avg_s = ph_ms / n_gemm / 1e3
        ops = RESID_FP32_OPS_PER_CMAC * n2 * n2 * N_RHS
        ach = ops / avg_s / 1e12
        roof.update({"kernel": "k_resid_df_gemm (double-float residual: exact products on the FP32 pipe)", "bound": "alu",
                     "launches": n_gemm, "avg_launch_ms": ph_ms / n_gemm, "achieved": ach, "peak": FP32_PEAK_T,
                     "unit": "T FP32 operations/s", "frac": ach / FP32_PEAK_T,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz"})

    return roof


def _load_lib():
    import torch
    import paper_2312_12787_gb300 as P
    from paper_2312_12787_gb300 import build as Bd
    Bd.build()
    P.load()
    return torch, P


def elements_per_wavelength(wp):
    """N_e x (interior wavelength 2 pi / k_i) / (boundary length): how finely the mesh resolves the interior field."""
    length = 0.0
    for sgm in wp.segments:
        xy = np.asarray(sgm.xy, float)
        d = np.diff(np.vstack([xy, xy[:1]]) if sgm.closed else xy, axis=0)
        length += float(np.hypot(d[:, 0], d[:, 1]).sum())
    return wp.n_elem * 2.0 * np.pi / (max(wp.k) * length)


def sweep_leg(args, clock_index=0):
    """The random-star sweep (256 stars, N_e U[128, 2048], k_e U[1, 40]) solved as one batch by the mixed
    engine, and the same 256 problems through the plain FP64 single-problem path one after another."""
    torch, P = _load_lib()
    stars = W.cfg_random_stars_c4()
    res = {}
    for leg in ("warmup", "timed"):
        kw = dict(tol=args.tol, max_iter=args.max_iter, inner_tol=args.inner_tol, orth_passes=args.orth_passes)
        probs = [P.Problem.from_workload(wp, prec="mixed", **kw) for wp in stars]
        xs = [torch.empty(p.bem_num_unknowns(), dtype=torch.complex128, device="cuda") for p in probs]
        bt = P.Batch(len(stars), sum(p.bem_num_unknowns() for p in probs), **kw)
        torch.cuda.synchronize()
        with ClockSampler(clock_index) as clk:
            t0 = time.perf_counter()
            st, it, rs = bt.bem_batch_solve_planewave(probs, np.zeros(len(stars)), xs)
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
        res[leg] = (t, it, rs, xs, clk.summary())
        bt.close()
        for p in probs:
            p.close()
    t, it, rs, xs, clocks = res["timed"]
    # the FP64 comparator on the identical problems (one warm-up solve first)
    it64, rs64, err = [], [], []
    q = P.Problem.from_workload(stars[0], prec="fp64", tol=args.tol, max_iter=600)
    q.bem_solve_planewave([0.0], torch.empty((1, q.bem_num_unknowns()), dtype=torch.complex128, device="cuda"))
    q.close()
    torch.cuda.synchronize()
    with ClockSampler(clock_index) as clk64:
        t0 = time.perf_counter()
        x64s = []
        for wp in stars:
            q = P.Problem.from_workload(wp, prec="fp64", tol=args.tol, max_iter=600)
            x64 = torch.empty((1, q.bem_num_unknowns()), dtype=torch.complex128, device="cuda")
            _, i64, r64 = q.bem_solve_planewave([0.0], x64)
            q.close()
            it64.append(int(i64[0]))
            rs64.append(float(r64[0]))
            x64s.append(x64[0])
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
    for xm, x64 in zip(xs, x64s):
        err.append((torch.linalg.vector_norm(xm - x64) / torch.linalg.vector_norm(x64)).item())
    # draws with fewer than 2 elements per interior wavelength are kept for throughput, not for accuracy claims
    epw = np.array([elements_per_wavelength(wp) for wp in stars])
    resolved = epw >= 2.0
    return {"metric": "random-star sweep solves/s (one mixed batch) vs FP64 one problem at a time",
            "value": len(stars) / t, "unit": "solves/s", "wall_s": t, "n_problems": len(stars),
            "iters_mean": float(np.mean(it)), "max_rel_resid": float(np.max(rs)), "tol": args.tol,
            "clocks": clocks,
            "fp64": {"value": len(stars) / t64, "unit": "solves/s", "wall_s": t64, "iters_mean": float(np.mean(it64)),
                     "max_rel_resid": float(np.max(rs64)), "clocks": clk64.summary()},
            "speedup_mixed_over_fp64": t64 / t,
            "max_rel_diff_mixed_vs_fp64": float(np.max(err)),
            "max_rel_diff_mixed_vs_fp64_resolved": float(np.max(np.asarray(err)[resolved])) if resolved.any() else None,
            "elements_per_interior_wavelength": {"min": float(epw.min()), "median": float(np.median(epw)),
                                                 "max": float(epw.max()), "below_2": int((~resolved).sum())},
            "config": {"workload": "256 random stars (seed 2312): lobes 3-7, amplitude U[0.1, 0.4], "
                                   "N_e U[128, 2048], k_e U[1, 40], contrast U[1.2, 2.0]; one plane wave each",
                       "l2": "sum of the matrices 12 GB (> L2)"}}


def serving_leg(args, clock_index=0):
    """The Poisson request stream through the continuous-batching loop (mixed), and the identical requests
    through the plain FP64 single-problem path one at a time in arrival order."""
    torch, P = _load_lib()
    from paper_2312_12787_gb300 import serve
    stream = W.cfg_serving_c5(count=args.requests)
    requests = [(t, wp, 0.0) for t, wp in stream]
    srv = serve.Server(max_slots=256, pool_unknowns=1 << 22, hbm_budget_bytes=96 << 30, tol=args.tol,
                       max_iter=args.max_iter, inner_tol=args.inner_tol, orth_passes=args.orth_passes)
    warm = W.cfg_serving_c5(count=8, seed=7)
    srv.run([(0.0, wp, 0.0) for _, wp in warm], time_limit_s=600)      # warm-up (kernel loading, autotuning)
    with ClockSampler(clock_index) as clk:
        stm = srv.run(requests, time_limit_s=3600)
    srv.close()
    with ClockSampler(clock_index) as clk64:
        st64 = serve.serve_fp64_sequential(requests, tol=args.tol, time_limit_s=3600)
    big = sum(serve.c32_matrix_bytes(wp) > 8e9 for _, wp, _ in requests)
    return {"metric": "serving solves/s and p50/p99 latency: continuous batching (mixed) vs FP64 one at a time",
            "mixed": stm.summary() | {"clocks": clk.summary()},
            "fp64_sequential": st64.summary() | {"clocks": clk64.summary()},
            "speedup_mixed_over_fp64": st64.wall_s / stm.wall_s if stm.wall_s > 0 else None,
            "tol": args.tol, "requests": len(requests), "matrix_free_requests": int(big),
            "config": {"workload": f"Poisson stream (seed 2313), {len(requests)} requests at 200/s: circles, ellipses "
                                   "(aspect U[1, 4]), 2-material junction disks; N_e log-uniform [256, 16384], "
                                   "k_e U[1, 50], contrast U[1.2, 2.0]; matrix-free above 8 GB of complex FP32 "
                                   "matrix (mixed path); the FP64 path stores every matrix",
                       "identical_requests": True}}


def omega_eps_leg(args):
    """The iteration studies of Sec. 7.1 (unit circle: GMRES iterations vs omega and vs eps_2) and Sec. 7.2
    (concentric circles: vs omega and vs eps_2 = 1/eps_3; the junction disk: vs N, omega and eps_3) for the
    proposed ("mod") arrangement and the others the paper compares ("orig": beta = -alpha on the standard rows
    only; "conv": conventional), each as one batch of all its problems."""
    torch, P = _load_lib()

    def run_batch(cases, form):
        res = {}
        for leg in ("warmup", "timed"):
            probs = [P.Problem.from_workload(wp, prec="mixed", form=form, tol=args.tol, max_iter=1000)
                     for _, _, wp in cases]
            xs = [torch.empty(p.bem_num_unknowns(), dtype=torch.complex128, device="cuda") for p in probs]
            bt = P.Batch(len(probs), sum(p.bem_num_unknowns() for p in probs), form=form, tol=args.tol,
                         max_iter=1000)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, it, rs = bt.bem_batch_solve_planewave(probs, np.zeros(len(probs)), xs)
            torch.cuda.synchronize()
            res[leg] = (time.perf_counter() - t0, it, rs)
            bt.close()
            for p in probs:
                p.close()
        t, it, rs = res["timed"]
        kinds = np.array([c[0] for c in cases])
        r = {"solves_per_s": len(cases) / t, "wall_s": t, "max_rel_resid": float(np.max(rs)),
             "iters_vs_omega": [int(v) for v in it[kinds == "omega"]],
             "iters_vs_eps": [int(v) for v in it[kinds == "eps"]]}
        if np.any(kinds == "n"):
            r["iters_vs_n"] = [int(v) for v in it[kinds == "n"]]
        return r
    circ = W.cfg_omega_eps_sweep()
    conc = W.cfg_concentric_sweep()
    junc = W.cfg_junction_sweep()
    with ClockSampler(0) as clk:
        out = {"circle": {f: run_batch(circ, f) for f in ("mod", "conv")},
               "concentric": {f: run_batch(conc, f) for f in ("mod", "orig", "conv")},
               "junction": {f: run_batch(junc, f) for f in ("mod", "orig", "conv")}}
    return {"metric": "omega / eps sweeps of Sec. 7 (one batch per geometry and arrangement, mixed)",
            "value": out["circle"]["mod"]["solves_per_s"], "unit": "solves/s", "tol": args.tol,
            "results": out, "clocks": clk.summary(),
            "circle_omega": [c[1] for c in circ if c[0] == "omega"],
            "circle_eps_2": [c[1] for c in circ if c[0] == "eps"],
            "concentric_omega": [c[1] for c in conc if c[0] == "omega"],
            "concentric_eps_3": [c[1] for c in conc if c[0] == "eps"],
            "junction_n": [c[1] for c in junc if c[0] == "n"],
            "junction_omega": [c[1] for c in junc if c[0] == "omega"],
            "junction_eps_3": [c[1] for c in junc if c[0] == "eps"],
            "config": {"workload": "unit circle, 600 elements: 64 omega in [0.5, 20] (eps_2 = 2), 64 eps_2 in "
                                   "[1.1, 10] (omega = 5); concentric circles, 600 + 1200 elements: 32 omega "
                                   "in [0.5, 10] (eps_i = i), 32 eps_3 in [0.1, 10] with eps_2 = 1/eps_3 "
                                   "(omega = 5); junction disk (3/4 of the elements on the circle, 1/4 on the "
                                   "diameter, eps_i = i): N in 266..3198 at omega = 5, 32 omega in [0.5, 10] and "
                                   "32 eps_3 in [0.1, 10] with eps_2 = 1/eps_3 (omega = 5) at N = 1066; Q = 4, "
                                   "tolerance 1e-8, mixed precision"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed_tc", choices=["mixed", "mixed_tc"])
    ap.add_argument("--tol", type=float, default=1e-8, help="relative residual target of both paths (paper: 1e-8)")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle leg (then the accuracy reference is "
                                                          "the FP64 GPU path at tol 1e-12)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison leg (profiling runs)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg (profiling runs)")
    ap.add_argument("--no-secondary", action="store_true", help="star: skip the sweep and serving keys")
    ap.add_argument("--n-elem", type=int, default=4096, help="elements of the star (smaller cases for ncu)")
    ap.add_argument("--max-iter", type=int, default=400)
    ap.add_argument("--inner-tol", type=float, default=1e-5, help="inner GMRES tolerance of the mixed path")
    ap.add_argument("--orth-passes", type=int, default=0, help="Gram-Schmidt passes of the mixed path (0 = auto)")
    ap.add_argument("--workload", default="star", choices=["star", "serving", "sweep", "omega_eps"],
                    help="star: the 64-RHS star (default line, with the sweep and serving keys); serving: the "
                         "Poisson request stream alone; sweep: 256 random stars in one batch alone; omega_eps: the "
                         "omega and eps sweeps of Sec. 7.1 and 7.2, one batch per arrangement")
    ap.add_argument("--requests", type=int, default=2000, help="serving: number of requests")
    ap.add_argument("--n-rhs", type=int, default=64, help="star: incident angles per step (64 = the workload)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "star":
        leg = {"sweep": sweep_leg, "serving": serving_leg, "omega_eps": omega_eps_leg}[args.workload]
        print(json.dumps(leg(args)), flush=True)
        return

    import torch
    ws, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    import paper_2312_12787_gb300 as P
    from paper_2312_12787_gb300 import build as B
    B.build()
    P.load()

    global N_RHS
    N_RHS = args.n_rhs
    wp = W.cfg_star_c2(args.n_elem)
    ang = W.plane_wave_angles(N_RHS)
    ffa = np.linspace(0.0, 2 * np.pi, N_FF, endpoint=False)
    stream = torch.cuda.current_stream()

    def make(prec):
        p = P.Problem.from_workload(wp, prec=prec, tol=args.tol, max_iter=args.max_iter, inner_tol=args.inner_tol,
                                    orth_passes=args.orth_passes if prec != "fp64" else 0)
        n2 = p.bem_num_unknowns()
        x = torch.empty((N_RHS, n2), dtype=torch.complex128, device="cuda")
        ff = torch.empty((N_RHS, N_FF), dtype=torch.complex128, device="cuda")
        return p, x, ff

    def step(p, x, ff):
        p.bem_assemble(stream)
        st, it, rs = p.bem_solve_planewave(ang, x, stream)
        p.bem_far_field(x, ffa, ff, n_rhs=N_RHS, stream=stream)
        return st, it, rs

    # ---- mixed path (headline) ----
    p, x, ff = make(args.prec)
    for _ in range(args.warmup):
        step(p, x, ff)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    iters, resids = [], []
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            evs[k][0].record(stream)
            st, it, rs = step(p, x, ff)
            evs[k][1].record(stream)
            iters.append(it.copy())
            resids.append(rs.copy())
        torch.cuda.synchronize()
    barrier(ws)
    times = [a.elapsed_time(b) for a, b in evs]
    total_ms = barrier_max(ws, sum(times))
    # phase breakdown from one more (untimed) step with per-launch CUDA events; the timed steps run without
    # them, which lets the tensor-core iterations replay as a CUDA graph
    p.bem_profile_enable(True)
    step(p, x, ff)
    torch.cuda.synchronize()
    prof = p.bem_profile_read()
    p.bem_profile_enable(False)
    x_mixed = x.clone()
    ms_step = total_ms / args.steps
    value = ws * N_RHS * args.steps / (total_ms / 1e3)
    lat = sorted(times)
    p50 = lat[len(lat) // 2]
    p99 = lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)]

    # ---- FP64 path: the same step ----
    fp64 = None
    x64 = None
    acc = {"tol": args.tol, "iters_mixed_max": int(np.max(iters[-1])), "iters_mixed_mean": float(np.mean(iters[-1])),
           "max_rel_resid_mixed": float(np.max(resids[-1]))}
    if not args.no_fp64:
        p64, x64, ff64 = make("fp64")
        step(p64, x64, ff64)
        torch.cuda.synchronize()
        t64 = []
        for _ in range(max(1, args.fp64_steps)):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st64, it64, rs64 = step(p64, x64, ff64)
            b.record(stream)
            torch.cuda.synchronize()
            t64.append(a.elapsed_time(b))
        fp64_ms = statistics.median(t64)
        p64.close()
        acc["iters_fp64_max"] = int(np.max(it64))
        acc["iters_fp64_mean"] = float(np.mean(it64))
        fp64 = {"value": N_RHS / (fp64_ms / 1e3), "unit": UNIT, "ms_per_step": fp64_ms,
                "speedup_mixed_over_fp64": fp64_ms / ms_step, "iters_max": int(np.max(it64))}

    # ---- end to end through the host-buffer entry point ----
    nel = wp.n_elem
    e2e = None
    if not args.no_e2e:
        e2e_ms = []
        h2d = nel * (4 * 8 + 2 * 4) + N_RHS * 8 + N_FF * 8
        d2h = N_RHS * 2 * nel * 16 + N_RHS * N_FF * 16
        for k in range(4):   # one warm-up call, the median of three timed ones
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            q = P.Problem.from_workload(wp, prec=args.prec, tol=args.tol, max_iter=args.max_iter)
            q.bem_solve_planewave_host(ang, ff_angles=ffa, want_traces=True, stream=stream)
            q.close()
            torch.cuda.synchronize()
            if k:
                e2e_ms.append(1e3 * (time.perf_counter() - t0))
        e2e = {"value": N_RHS / (statistics.median(e2e_ms) / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    hbm, src = _peaks()
    roof = roofline(prof, nel, hbm, src)
    n2 = 2 * nel

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c32 storage + f64 refinement", "data": "synthetic",
        "config": {"workload": wp.name, "n_elem": nel, "n_unknowns": n2, "n_rhs": N_RHS, "quad": 4,
                   "prec": args.prec, "tol": args.tol, "inner_tol": args.inner_tol, "orth_passes": args.orth_passes,
                   "far_field_angles": N_FF,
                   "l2": "inputs larger than L2 (A is 0.54 GB complex FP32 + 0.54 GB remainder)"},
        "latency_ms": {"p50": p50, "p99": p99, "unit": "ms per 64-solve batch"},
        "fp64": fp64,
        "accuracy": acc,
        "phases_ms": {k: round(v[0], 3) for k, v in prof.items() if v[1] and k != "relaxed"},   # one profiled step
        "roofline": roof,
        # the assembly kernel's own rate: Gauss nodes x the (two) domains of every element pair of one interface
        "assembly": ({"ms_per_launch": prof["assemble"][0] / prof["assemble"][1],
                      "hankel_pairs_per_launch": 4 * 2 * nel * nel,
                      "hankel_pairs_per_s": 4 * 2 * nel * nel / (prof["assemble"][0] / prof["assemble"][1] / 1e3)}
                     if prof.get("assemble", (0, 0))[1] else None),
        "e2e": e2e,
        "gpu_launches": int(sum(v[1] for k, v in prof.items() if k != "relaxed")) * args.steps,
        "clocks": clk.summary(),
    }
    # ---- CPU oracle (rank 0, N = 1): timed on the whole workload; its LU solution is the accuracy reference ----
    if rank == 0 and ws == 1 and not args.no_cpu:
        info, X = oracle_full(wp, ang, args.tol)
        v = N_RHS / (info["assembly_s"] + info["rhs_and_lu_s"])
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
                                "sample": f"the whole workload: assembly of all {n2} rows on {info['cores']} "
                                          f"host processes + LU solve of {N_RHS} right-hand sides (not "
                                          "extrapolated); the single-process assembly time is extrapolated from "
                                          "128 rows; the oracle's GMRES is timed on one column",
                                "extrapolated": False, **info}
        Xd = torch.as_tensor(X, device="cuda")
        nrm = torch.linalg.vector_norm(Xd, dim=1)
        acc["reference"] = "oracle LU solution (FP64, CPU)"
        acc["max_rel_err_mixed"] = (torch.linalg.vector_norm(x_mixed - Xd, dim=1) / nrm).max().item()
        if x64 is not None:
            acc["max_rel_err_fp64"] = (torch.linalg.vector_norm(x64 - Xd, dim=1) / nrm).max().item()
    elif x64 is not None:
        pr = P.Problem.from_workload(wp, prec="fp64", tol=1e-12, max_iter=args.max_iter)
        xr = torch.empty_like(x64)
        pr.bem_solve_planewave(ang, xr, stream)
        pr.close()
        nrm = torch.linalg.vector_norm(xr, dim=1)
        acc["reference"] = "FP64 GPU path at tol 1e-12"
        acc["max_rel_err_mixed"] = (torch.linalg.vector_norm(x_mixed - xr, dim=1) / nrm).max().item()
        acc["max_rel_err_fp64"] = (torch.linalg.vector_norm(x64 - xr, dim=1) / nrm).max().item()
    p.close()
    # ---- secondary keys: the batched sweep and the serving stream (rank 0) ----
    if rank == 0 and not args.no_secondary:
        line["sweep"] = sweep_leg(args, local)
        line["serving"] = serving_leg(args, local)
        line["sec7_sweeps"] = omega_eps_leg(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
