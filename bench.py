"""Benchmark: Poisson solves/s to 1e-8 relative residual on the icosphere x8 mesh.

Workload (the configuration the headline metric is quoted on): unit
icosphere subdivided 8 times with midpoints projected to radius 1
(655,362 vertices, 1,310,720 triangles), 7 multigrid levels (162 ... 655,362
vertices), constant-nullspace gauge, right-hand side = sum of real spherical
harmonics of degree 1..16 with N(0,1) coefficients (seed 1), flexible
MG-preconditioned CG with FP32 V-cycles inside an FP64 outer iteration --
FP64 residual, dot products (products and sums), updates and gauge
projection (--mode mixed) -- to relative residual 1e-8.  One step = one
complete solve with b resident in HBM.  The line also reports the other
modes (f64: all FP64; mixed_ff: float-float outer iteration; mixed_f32dot:
FP64 updates with FP32 dot products), their speed-ups over f64, and the true
FP64 residual of every returned solution.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs independent replicas of the solve on its own
GPU (the solve has no data-parallel split); `value` is the total solves/s of
all ranks over the slowest rank's time.  `--impl reference` times the FP64
CPU oracle on the host (rank 0 only) on the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

# The CPU oracle (cpu_baseline, --impl reference) is timed on one core: BLAS and OpenMP pools default to one
# thread unless the caller sets them (before numpy loads its BLAS).  The GPU path does no host arithmetic.
for _var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_var, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "Poisson solves/s to 1e-8 rel. residual; V-cycle MDOF/s; HBM GB/s vs peak"
NSUB, NLEVELS, TOL, SEED = 8, 7, 1e-8, 1
WORKLOAD = "icosphere_l8_gauge_sh16_mgpcg_1e-8"
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2

# Algorithmic bytes per row of each kernel kind (K = stencil slots per row,
# FP32 cycle vectors / FP64 outer vectors, int32 columns).  A gathered vector
# is counted once per row (its entries are reused from cache by neighbours).
def bytes_per_row(kind, K, mode, cheb, outer=False):
    mixed = mode != "f64"
    ff = mode == "mixed_ff"
    d64 = mode == "mixed"  # FP64 dot products with the FP64 residual
    f = 4 if mixed else 8  # cycle precision
    if kind == "smooth0":
        return K * f + f + f + (f if cheb else 0)
    if kind == "smoothdots":
        # the last smoothing step (operator, b = r32, x, direction, new x) plus *0, free mask, previous z
        # (and the FP64 residual with FP64 *0 in mode mixed)
        if d64:
            return K * 4 + K * 4 + 3 * 4 + (4 if cheb else 0) + 8 + 1 + 8 + 4
        return K * 4 + K * 4 + 3 * 4 + (4 if cheb else 0) + 4 + 1 + 4
    if kind == "smooth01":
        # operator, diagonal, b, the new x (two steps, nu = 2: no direction is written)
        return K * 4 + K * f + 3 * f
    if kind == "smooth":
        # with nu = 2 each Chebyshev step reads or writes one direction vector
        return K * 4 + K * f + 3 * f + (f if cheb else 0)
    if kind == "residual":
        return K * 4 + K * f + 3 * f
    if kind == "spmv64":
        if ff:
            return K * 12 + 4 + 8 + 4  # col, w32 + wlo, p_i (f32), q hi+lo, *0 (f32)
        return K * 4 + K * 8 + 8 + 8 + 8  # col, w64, p_i, q, *0
    if kind == "update":
        if ff:
            # p, q, x and r (hi+lo, read and write); fused: the diagonal and the first smoothing step's x, d
            return 4 + 8 + 16 + 16 + (12 if outer else 0)
        if d64:
            # p, q, x and r (read and write), r32; fused: the diagonal and the first smoothing step's x, d
            return 8 + 8 + 16 + 16 + 4 + (12 if outer else 0)
        return 8 + 8 + 16 + 16 + (4 if mixed else 0)
    if kind == "zdots":
        # mixed: *0 (f64), free, z, r (f64), z_old (f32); mixed_f32dot / ff: *0 (f32), free, z, r32, z_old;
        # f64: z, zn write, *0, r, z_old, free
        if d64:
            return 8 + 1 + 4 + 8 + 4
        return (4 + 1 + 4 + 4 + 4) if mixed else (8 + 8 + 8 + 8 + 8 + 1)
    if kind == "pupd":
        if ff:
            return 1 + 4 + 4 + 8  # free, z, z_old write, p (f32) read and write
        return (1 + 4 + 4 + 16) if mixed else (8 + 1 + 8 + 16)
    return None


def fp64_per_row(kind, mode):
    """FP64 instructions per row of the FP64-pipe-bound outer kernels (0: not FP64-bound).  Mode mixed:
    q = L p in the difference form (6 subtractions, 6 FMAs) with <p, q>*0 (a product, an FMA); the update
    (x, r, ||r||^2: 3 FMAs, the FP32 rounding of r); the four *0 dot products of z (a product, 3 FMAs, an
    add; z widened by integer instructions); the direction (a subtraction, an FMA)."""
    if mode == "mixed":
        return {"spmv64": 14, "update": 4, "smoothdots": 5, "zdots": 5, "pupd": 2}.get(kind, 0)
    if mode == "mixed_f32dot":
        return {"spmv64": 14, "update": 3, "pupd": 1}.get(kind, 0)
    if mode == "f64":
        return {"spmv64": 21, "update": 3, "zdots": 6, "pupd": 2}.get(kind, 0)
    return 0


def restrict_bytes(n_f, n_c, K, f):
    return n_c * K * 4 + n_f * f + n_c * f


def prolong_bytes(n_f, n_c, f):
    return 2 * n_f * f + (n_f - n_c) * 8 + n_c * f


def kernel_bytes(entry, hier, mode, cheb):
    """Algorithmic bytes moved by one launch of a profiled kernel."""
    lvl = entry["level"]
    n = entry["rows"]
    K = hier.ell_width[lvl]
    f = 4 if mode != "f64" else 8
    kind = entry["kind"]
    if kind == "restrict":
        extra = 0
        if getattr(hier, "fuse", 0) & 8 and lvl - 1 > 0:
            extra = hier.nv[lvl - 1] * (3 * f)  # the coarse level's first smoothing step: diagonal in, x and d out
        return restrict_bytes(n, hier.nv[lvl - 1], K, f) + extra
    if kind == "prolong":
        return prolong_bytes(n, hier.nv[lvl - 1], f)
    nc = hier.nv[lvl - 1] if lvl > 0 else 0
    if kind == "resrestrict":
        # fine operator, x and b once; the coarse right-hand side written
        return n * (K * 4 + K * f + 2 * f) + nc * f
    if kind == "prolsmooth":
        # operator, diagonal, b, x in and out, the direction (Chebyshev), the coarse correction and parents
        return n * (K * 4 + K * f + 4 * f + (f if cheb else 0)) + nc * f + (n - nc) * 8
    if kind in ("patchdown", "patchup"):
        # halo tiles, per row of the level once (the ring rows a tile recomputes are not counted): the
        # operator, b, the diagonal (down) or the uncorrected iterate (up), the new iterate; the coarse
        # right-hand side (down) or the coarse correction and the midpoint parents (up)
        return n * (K * 4 + K * f + 3 * f) + nc * f + ((n - nc) * 8 if kind == "patchup" else 0)
    per = bytes_per_row(kind, K, mode, cheb, outer=bool(getattr(hier, "fuse", 0) & 16))
    return None if per is None else per * n


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# Device sources each measured kernel is compiled from (single-right-hand-side kernels: kernels.cuh and
# coarse_cycle.cuh; batched kernels: the device part of batch.cu, everything before its host-side section,
# and the kernels.cuh helpers it includes).
KERNEL_SOURCES = {"single": ("kernels.cuh", "coarse_cycle.cuh"), "batched": ("batch.cu", "kernels.cuh")}
DEVICE_PART_END = {"batch.cu": b"// host side\n"}


def kernels_hash(group="single"):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[group]:  # the device code the counters were taken on
        with open(os.path.join(ROOT, "paper_2508_12501_gb300", "csrc", f), "rb") as fh:
            data = fh.read()
        end = DEVICE_PART_END.get(f)
        if end is not None and end in data:
            data = data[:data.index(end)]
        h.update(data)
    return h.hexdigest()[:16]


def ncu_traffic(kind):
    """DRAM bytes per launch of `kind` from the committed ncu summary, if it was taken on the current kernels."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    ent = d.get("kernels", {}).get(kind)
    if ent is None or ent.get("kernels_hash") != kernels_hash(ent.get("sources", "single")):
        return None
    return float(ent["dram_bytes_per_launch"])


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        # raw samples; the JSON line carries their summary
        self.path = os.path.join(os.environ.get("DEC_BENCH_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"dec_bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu is not None:
                cmd += ["-i", str(self.gpu)]
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower() in ("active", "1"):
                        reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------
# oracle arm / CPU baseline
# ----------------------------------------------------------------------------

def oracle_setup(smoother="chebyshev"):
    from oracle import multigrid as omg
    v, t = W.icosahedron()
    oh = omg.build_hierarchy(v, t, NSUB, NLEVELS, "gauge", sphere=True, opts=omg.MGOptions(smoother=smoother))
    b = W.sh_sum(oh.finest.mesh.verts, W.sh_coefficients(SEED))
    return oh, b


_ORACLE_CPU = {"cpu_s": 0.0, "wall_s": 0.0}


def oracle_time(oh, b, nsolve):
    from oracle import multigrid as omg
    ts = []
    res = None
    c0, w0 = time.process_time(), time.perf_counter()
    for _ in range(nsolve):
        t0 = time.perf_counter()
        res = omg.pcg_solve(oh, b, TOL, 100)
        ts.append(time.perf_counter() - t0)
    _ORACLE_CPU["cpu_s"] = time.process_time() - c0
    _ORACLE_CPU["wall_s"] = time.perf_counter() - w0
    return ts, res


def cpu_cores_used():
    """Cores the last timed oracle solves kept busy: the process's CPU time (all its threads, e.g. a
    multithreaded BLAS) over the wall time, at least 1."""
    w = _ORACLE_CPU["wall_s"]
    return max(1.0, round(_ORACLE_CPU["cpu_s"] / w, 1)) if w > 0 else 1.0


def workload_config(args, nv, world):
    """The `config` object of the JSON line; both arms print the same one."""
    return {"workload": WORKLOAD, "nv": nv, "levels": NLEVELS, "smoother": args.smoother, "cycle": "V(2,2)",
            "mode": args.mode, "tol": TOL, "l2": "256 MB buffer written before every step (flush)",
            "parallelism": f"replicas x{world}"}


def run_reference(args, rank):
    if rank != 0:
        return 0
    oh, b = oracle_setup(args.smoother)
    oracle_time(oh, b, args.warmup)
    ts, res = oracle_time(oh, b, args.steps)
    tot = sum(ts)
    value = args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, oh.finest.mesh.nv, int(os.environ.get("WORLD_SIZE", "1"))),
        "reference_solver": "oracle flexible MG-PCG, FP64 throughout, numpy/scipy on the host (1 thread)",
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cpu_cores_used(), "kind": "oracle",
                         "sample": f"{args.steps} complete oracle solves of the full workload ({res.iters} iterations each)"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "iters": res.iters, "rel_res": res.rel_res,
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# batched workload: 64 right-hand sides on the icosphere x7 plus 32 squares
# ----------------------------------------------------------------------------

def batched_workload(torch, dev, flush, stream, steps, tune=True):
    import paper_2508_12501_gb300 as P
    v, t = W.icosahedron()
    hi = P.Hierarchy(P.Mesh(v, t), 7, 6, bc="gauge", sphere=True)
    pos = hi.table(-1, "verts")
    hs, ks = [hi], [64]
    bs = [torch.as_tensor(np.stack([W.sh_sum(pos, W.sh_coefficients(100 + j)) for j in range(64)], axis=1)
                          .reshape(-1), device=dev)]
    vs, ts = W.unit_square()
    seed = 200
    for nsub in (6, 7, 8, 9):
        hq = P.Hierarchy(P.Mesh(vs, ts), nsub, nsub - 1, bc="dirichlet")
        for _ in range(8):
            hs.append(hq)
            ks.append(1)
            bs.append(torch.as_tensor(W.uniform_field(hq.n, seed), device=dev))
            seed += 1
    # block size, interleave width k (0: every right-hand side of a hierarchy in one group, up to the block
    # size) and sweeps per smoothing call
    cands = [dict(block=bl, kgroup=kg, nu=nu, smoother="chebyshev", solver="mgpcg")
             for bl in (256, 512) for kg in (0, 8, 16, 32) for nu in (1, 2, 3)]
    if tune:
        best, best_ms, table = P.tune_batch(hs, ks, bs, tol=TOL, candidates=cands, reps=2)
    else:  # the library's defaults (block 256, one group per hierarchy, Chebyshev nu = 2, MG-PCG)
        best, table = dict(block=256, kgroup=0, nu=2, smoother="chebyshev", solver="mgpcg"), []

    def timed(B, fn):
        for _ in range(2):
            fn()
        evs, st = [], None
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize(dev)
        return sum(a.elapsed_time(c) for a, c in evs) / 1e3, st

    B = P.Batch(hs, ks, **best)
    xs = [None]

    def fwd():
        xs[0], st = B.solve(bs, tol=TOL)
        return st
    tot, st = timed(B, fwd)
    # the adjoint of every solve: dJ/du = u (J = 1/2 ||u||^2 per right-hand side), dJ/db and dJ/d*1
    us = [x.reshape(h.n, -1) for x, h in zip(xs[0], hs)]
    tot_b, stb = timed(B, lambda: B.solve_backward(us, us, tol=TOL)[2])
    # the same batch by FP64 iterative refinement around the FP32 cycles
    Bm = P.Batch(hs, ks, **dict(best, solver="mg"))
    tot_m, stm = timed(Bm, lambda: Bm.solve(bs, tol=TOL)[1])
    torch.cuda.nvtx.range_push("batched_time_smooth")  # the launches profiles/ captures of k_b_smooth
    ms, by = B.time_smooth(20)
    torch.cuda.nvtx.range_pop()
    peak, src = peaks()
    return {
        "workload": "64 SH right-hand sides on icosphere x7 (163,842 V) + 32 unit squares at levels 6-9 "
                    "(8 per level), FP32 cycles inside FP64 flexible MG-PCG per right-hand side, to 1e-8",
        "rhs_solves_per_s": sum(ks) * steps / tot, "batch_ms": 1e3 * tot / steps, "iters": st.iters,
        "max_rel_res": st.max_rel_res, "dof": st.dof,
        "mdof_per_s_per_iter": st.dof * st.iters * steps / tot / 1e6, "gpu_launches_per_solve": st.launches,
        "adjoint": {"rhs_solves_per_s": sum(ks) * steps / tot_b, "batch_ms": 1e3 * tot_b / steps,
                    "iters": stb.iters, "max_rel_res": stb.max_rel_res,
                    "what": "dJ/db and dJ/d*1 of every right-hand side (adjoint MG-PCG on the same batch)"},
        "refinement": {"rhs_solves_per_s": sum(ks) * steps / tot_m, "batch_ms": 1e3 * tot_m / steps,
                       "passes": stm.iters, "max_rel_res": stm.max_rel_res},
        "tuned": best, "tuner_table": [[o["block"], o["kgroup"], round(tm, 4)] for o, tm in table],
        "roofline_smooth": {"bound": "hbm", "achieved": by / (ms * 1e-3) / 1e9, "peak": peak, "peak_source": src,
                            "unit": "GB/s", "frac": by / (ms * 1e-3) / 1e9 / peak, "algorithmic_bytes": by,
                            "avg_launch_ms": ms, "traffic": ncu_traffic("batched_smooth"),
                            "timing": "20 back-to-back launches of the finest-level sweep between two CUDA events"},
    }


# ----------------------------------------------------------------------------
# V-cycle convergence factor of each smoother, GPU next to the oracle
# ----------------------------------------------------------------------------

def convergence_factors(torch, dev):
    import paper_2508_12501_gb300 as P
    from oracle import multigrid as omg
    out = []
    cases = [("icosphere x6 (40,962 V), gauge", W.icosahedron, 6, 5, "gauge", True),
             ("unit square x7 (16,641 V), Dirichlet", W.unit_square, 7, 6, "dirichlet", False)]
    for label, base, nsub, nl, bc, sph in cases:
        v, t = base()
        for smoother in ("jacobi", "chebyshev", "mcgs"):
            for gamma in (1, 2, "F"):
                fc = gamma == "F"
                g = 1 if fc else gamma
                h = P.Hierarchy(P.Mesh(v, t), nsub, nl, bc=bc, sphere=sph, smoother=smoother, gamma=g, fcycle=fc)
                oh = omg.build_hierarchy(v, t, nsub, nl, bc, sphere=sph,
                                         opts=omg.MGOptions(smoother=smoother, gamma=g, fcycle=fc))
                b = W.uniform_field(h.n, 71)
                _, st = h.solve(torch.as_tensor(b, device=dev), solver="mg", mode="f64", tol=1e-10, maxit=100)
                ref = omg.mg_solve(oh, b, 1e-10, 100)
                out.append({"mesh": label, "smoother": smoother, "cycle": {1: "V(2,2)", 2: "W(2,2)", "F": "F(2,2)"}[gamma],
                            "gpu": round((st.rel_res / st.rel_res0) ** (1.0 / st.iters), 4),
                            "oracle": round(omg.convergence_factor(ref.history), 4),
                            "gpu_cycles": st.iters, "oracle_cycles": ref.iters})
    return out


def _timed(torch, dev, stream, fn, reps):
    """Mean milliseconds of fn() over reps calls after one warm-up call (CUDA events on the solve stream)."""
    fn()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = None
    for _ in range(reps):
        r = fn()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1) / reps, r


def _oracle_clock(fn, reps=1):
    """(mean seconds, CPU seconds / wall seconds, last result) of fn() on the host."""
    c0, w0 = time.process_time(), time.perf_counter()
    r = None
    for _ in range(reps):
        r = fn()
    wall = time.perf_counter() - w0
    cores = max(1.0, round((time.process_time() - c0) / wall, 1)) if wall > 0 else 1.0
    return wall / reps, cores, r


def oracle_other_configs():
    """The FP64 CPU oracle timed on the other workloads (one thread; hierarchy builds excluded).
    Returns {config key: cpu_baseline object}; long workloads are timed on a bounded sample and
    extrapolated, as each `sample` says."""
    from oracle import adjoint as oadj, multigrid as omg, porous as opor
    from oracle.mesh import d0_matrix
    out = {}
    v, t = W.unit_square()
    # standalone FP64 V(2,2) Jacobi MG, unit square x5 to 1e-10
    oh = omg.build_hierarchy(v, t, 5, 5, "dirichlet")
    b = W.rhs_sin_square(oh.finest.mesh.verts)
    sec, cores, r = _oracle_clock(lambda: omg.mg_solve(oh, b, 1e-10, 100), 10)
    out["standalone_mg"] = {"value": 1.0 / sec, "unit": "solves/s", "cores": cores, "kind": "oracle",
                            "sample": f"10 complete oracle MG solves ({r.iters} cycles each)"}
    # batched: 64 SH right-hand sides on icosphere x7 + 32 squares (8 per level 6..9), refinement to 1e-8 with
    # FP64 Chebyshev V(2,2) cycles; a sample of 2 icosphere and 4 square solves (one per level), extrapolated
    vi, ti = W.icosahedron()
    ohi = omg.build_hierarchy(vi, ti, 7, 6, "gauge", sphere=True, opts=omg.MGOptions(smoother="chebyshev"))
    pos = ohi.finest.mesh.verts
    ts_ico = []
    for j in (0, 1):
        bj = W.sh_sum(pos, W.sh_coefficients(100 + j))
        sec, cores_i, _ = _oracle_clock(lambda: omg.mg_solve(ohi, bj, TOL, 100))
        ts_ico.append(sec)
    del ohi
    t_sq = 0.0
    for nsub, seed in zip((6, 7, 8, 9), (200, 208, 216, 224)):
        ohq = omg.build_hierarchy(v, t, nsub, nsub - 1, "dirichlet", opts=omg.MGOptions(smoother="chebyshev"))
        bq = W.uniform_field(ohq.finest.mesh.nv, seed)
        sec, _, _ = _oracle_clock(lambda: omg.mg_solve(ohq, bq, TOL, 100))
        t_sq += 8 * sec
    t_all = 64 * statistics.mean(ts_ico) + t_sq
    out["batched"] = {"value": 96 / t_all, "unit": "RHS solves/s", "cores": cores_i, "kind": "oracle",
                      "sample": "2 icosphere x7 and 4 square solves (one per level 6-9) of the batch, FP64 MG "
                                "refinement to 1e-8, extrapolated to the 96 right-hand sides (64 x icosphere "
                                "mean + 8 x each square level)"}
    # differentiable solve: unit square x10 (1,050,625 V), log-normal *1, forward MG-PCG to 1e-8, adjoint solve,
    # dJ/db and dJ/d*1
    oh = omg.build_hierarchy(v, t, 10, 9, "dirichlet", star1_scale=W.lognormal_factors(3147776, 2),
                             opts=omg.MGOptions(smoother="chebyshev"))
    lev = oh.finest
    b = W.uniform_field(lev.mesh.nv, 3)
    ut = W.u_target_square(lev.mesh.verts)
    d0 = d0_matrix(lev.mesh).astype(np.float64)

    def fwd_bwd():
        u = omg.pcg_solve(oh, b, TOL, 100).x
        mu = omg.pcg_solve(oh, (u - ut) * lev.free, TOL, 100).x
        return lev.star0 * mu * lev.free, -(d0 @ mu) * (d0 @ u)
    sec, cores, _ = _oracle_clock(fwd_bwd)
    out["adjoint"] = {"value": 1e3 * sec, "unit": "ms per forward + backward", "cores": cores, "kind": "oracle",
                      "sample": "one oracle forward MG-PCG solve and one adjoint MG-PCG solve to 1e-8 with both "
                                "gradients"}
    del oh, lev, d0
    # porous rollout: unit square x9, forward Euler, the oracle's direct pressure solves; 3 steps extrapolated
    from oracle import mesh as omesh
    m9 = omesh.refine(v, t, 9)[0][-1]
    lev9 = omg.make_level(m9, "gauge")
    prm = opor.PorousParams()
    prm.dt = 0.5 * (1.0 / 512) ** 2 / (4 * prm.kappa)
    xy = m9.verts
    fixed = (xy[:, 1] == 0.0) | (xy[:, 1] == 1.0)
    pot = opor.potential(xy, prm)
    T0 = W.porous_initial_T(xy, 0)
    sec, cores, _ = _oracle_clock(lambda: opor.step(lev9, T0, pot, fixed, prm), 3)
    out["porous"] = {"value": 1.0 / sec, "unit": "steps/s", "cores": cores, "kind": "oracle",
                     "sample": "3 oracle forward-Euler steps (direct sparse pressure solve each) on the unit "
                               "square x9; 2000 steps would take 2000 / value seconds"}
    return out


def other_configs(torch, dev, stream):
    """The scope table's other workloads (standalone MG, the differentiable solve, the porous rollout)."""
    import math
    import paper_2508_12501_gb300 as P
    out = {}
    v, t = W.unit_square()
    # standalone FP64 V(2,2) multigrid, unit square x5, against the discrete closed form
    h = P.Hierarchy(P.Mesh(v, t), 5, 5, bc="dirichlet")
    xy = h.table(-1, "verts")
    s0 = h.table(-1, "star0")
    b = torch.as_tensor(W.rhs_sin_square(xy), device=dev)
    ms, (x, st) = _timed(torch, dev, stream, lambda: h.solve(b, solver="mg", mode="f64", tol=1e-10, maxit=100), 50)
    hh = 1.0 / 32
    u_h = 2 * math.pi ** 2 / (8.0 / hh ** 2 * math.sin(math.pi * hh / 2) ** 2) * W.u_sin_square(xy)
    d = x.cpu().numpy() - u_h
    out["standalone_mg"] = {
        "workload": "unit square x5 (1,089 V), 5-level V(2,2) Jacobi, Dirichlet, RHS -Delta sin(pi x) sin(pi y), "
                    "FP64 MG to 1e-10", "ms_per_solve": ms, "solves_per_s": 1e3 / ms, "iters": st.iters,
        "conv_factor": (st.rel_res / st.rel_res0) ** (1.0 / st.iters),
        "rel_err_vs_discrete_closed_form": float(np.sqrt(np.sum(s0 * d * d) / np.sum(s0 * u_h * u_h)))}
    del h
    # differentiable solve: forward and adjoint on unit square x10 with log-normal *1
    h = P.Hierarchy(P.Mesh(v, t), 10, 9, bc="dirichlet", smoother="chebyshev")
    s1 = h.table(-1, "star1") * W.lognormal_factors(h.ne[-1], 2)
    h.set_star1(torch.as_tensor(s1, device=dev))
    xy = h.table(-1, "verts")
    s0d = torch.as_tensor(h.table(-1, "star0"), device=dev)
    b = torch.as_tensor(W.uniform_field(h.n, 3), device=dev)
    ut = torch.as_tensor(W.u_target_square(xy), device=dev)

    def fwd_bwd(mode):
        u, sf = h.solve(b, mode=mode, tol=1e-8)
        gb, gs, sb = h.solve_backward(u, s0d * (u - ut), mode=mode, tol=1e-8)
        return sf, sb
    ms, (sf, sb) = _timed(torch, dev, stream, lambda: fwd_bwd("mixed"), 5)
    ms_ff, _ = _timed(torch, dev, stream, lambda: fwd_bwd("mixed_ff"), 5)
    ms_64, _ = _timed(torch, dev, stream, lambda: fwd_bwd("f64"), 5)

    def finest_roofline(mode):
        # the finest level's cycle kernels in one forward solve, timed by event pairs in the solve's graph;
        # at 1,050,625 rows a sweep moves 67 MB (FP32 cycles) or 109 MB (FP64): per-level working sets at or
        # above L2, where the scope table asks for the HBM fraction
        h.profile(1)
        h.solve(b, mode=mode, tol=1e-8)
        torch.cuda.synchronize(dev)
        ent = h.profile_read()
        h.profile(0)
        peak, src = peaks()
        kern = {}
        for e in ent:
            if e["kind"] not in ("smooth", "residual", "restrict", "prolong"):
                continue
            by = kernel_bytes(e, h, mode, True)
            avg = e["total_ms"] / max(1, e["launches"])
            gbs = by / (avg * 1e-3) / 1e9
            kern[e["kind"]] = {"algorithmic_bytes": by, "avg_launch_ms": avg, "achieved_gbs": gbs,
                               "frac": gbs / peak}
        return {"peak": peak, "peak_source": src, "unit": "GB/s", "kernels": kern,
                "timing": "event pair around each launch inside the solve's iteration graph (in-solve)"}
    roof_mixed, roof_64 = finest_roofline("mixed"), finest_roofline("f64")
    out["adjoint"] = {
        "workload": "unit square x10 (1,050,625 V), log-normal *1 (sigma 0.5, seed 2), b U[-1,1] (seed 3), "
                    "J = 1/2 ||u - sin(2 pi x) sin(pi y)||^2_*0, dJ/db and dJ/d*1, MG-PCG mixed (FP32 cycles, "
                    "FP64 outer) to 1e-8",
        "ms_forward_backward": ms, "forward_iters": sf.iters, "backward_iters": sb.iters,
        "ms_forward_backward_mixed_ff": ms_ff, "ms_forward_backward_f64": ms_64,
        "speedup_vs_f64": ms_64 / ms, "roofline_finest_mixed": roof_mixed, "roofline_finest_f64": roof_64}
    del h
    # porous convection: 2000 explicit steps with checkpoints every 100, then the checkpointed adjoint
    h = P.Hierarchy(P.Mesh(v, t), 9, 8, bc="gauge", restriction="star0")
    xy = h.table(-1, "verts")
    fixed = torch.as_tensor(((xy[:, 1] == 0.0) | (xy[:, 1] == 1.0)).astype(np.uint8), device=dev)
    T0 = torch.as_tensor(W.porous_initial_T(xy, 0), device=dev)
    kappa, nsteps, ce = 2.0, 2000, 100
    dt = 0.5 * (1.0 / 512) ** 2 / (4 * kappa)
    ck = torch.empty((nsteps // ce + 1) * h.n, dtype=torch.float64, device=dev)
    top = torch.as_tensor(xy[:, 1] == 1.0, device=dev).double()
    gradF = -kappa * torch.as_tensor(h.table(-1, "star0"), device=dev) * h.laplace0_apply(top)
    T = T0.clone()
    Pr = torch.zeros_like(T)
    h.porous_step(T, Pr, fixed, 10, dt, tol=1e-8, mode="mixed")  # warm-up
    ms_f, _ = _timed(torch, dev, stream, lambda: h.porous_step(T0.clone(), torch.zeros_like(T0), fixed, nsteps, dt,
                                                               checkpoints=ck, ckpt_every=ce, tol=1e-8,
                                                               mode="mixed"), 1)
    ms_b, (g, sb) = _timed(torch, dev, stream, lambda: h.porous_backward(T0, torch.zeros_like(T0), fixed, nsteps, gradF,
                                                                         dt, ckpt_every=ce, tol=1e-8,
                                                                         mode="mixed"), 1)
    out["porous"] = {
        "workload": "unit square x9 (263,169 V), T0 = 100 - 200 y + 1e-3 U[-1,1] (seed 0), 2000 forward-Euler "
                    "steps, dt = h^2/(8 kappa), pressure MG-PCG mixed (FP32 cycles, FP64 outer) to 1e-8 (warm "
                    "start), checkpoints every 100 steps; adjoint of the top-boundary heat flux",
        "rollout_ms": ms_f, "steps_per_s": nsteps / (ms_f * 1e-3), "adjoint_ms": ms_b,
        "forward_plus_adjoint_ms": ms_f + ms_b, "grad_norm": float(torch.linalg.vector_norm(g))}

    # the paper's porous run (Sec. 3.2.2) on its 16,641-vertex mesh: Gaussian T0, walls at -100 / +100,
    # adaptive Tsit5 at rtol 1e-9 over the first 1 % of its interval; MG-PCG pressure solves in mixed_ff
    # to 1e-8 against FP64 ones to 1e-12 (the stand-in for the paper's LU reference)
    h7 = P.Hierarchy(P.Mesh(v, t), 7, 6, bc="gauge", restriction="star0")
    xy7 = h7.table(-1, "verts")
    T7 = W.gaussian_initial_T(xy7, (0.5, 0.5))
    T7 = np.where(xy7[:, 1] == 1.0, -100.0, np.where(xy7[:, 1] == 0.0, 100.0, T7))
    T7 = torch.as_tensor(T7, device=dev)
    fx7 = torch.as_tensor(((xy7[:, 1] == 0.0) | (xy7[:, 1] == 1.0)).astype(np.uint8), device=dev)
    t_end = 5e-3
    runs = {}
    for key, kw in (("mg", dict(tol=1e-8, mode="mixed_ff")), ("fp64", dict(tol=1e-12, mode="f64", maxit=300))):
        Tk = T7.clone()
        Pk = torch.zeros_like(Tk)

        def run():  # from the initial state every call (the warm-up call included)
            Tk.copy_(T7)
            Pk.zero_()
            return h7.porous_rk(Tk, Pk, fx7, t_end, 1e-6, rtol=1e-9, atol=1e-6, **kw)
        ms_k, st_k = _timed(torch, dev, stream, run, 1)
        runs[key] = (Tk, st_k, ms_k)
    Tm, stm, msm = runs["mg"]
    rmse = float(torch.sqrt(torch.mean((Tm - runs["fp64"][0]) ** 2)))
    out["porous_tsit5"] = {
        "workload": "unit square x7 (16,641 V, the paper's porous mesh), T0 = 400 x Gaussian(centre, I/2), walls "
                    "-100 / +100, adaptive Tsit5 (rtol 1e-9, atol 1e-6) from t = 0 to 5e-3, pressure MG-PCG mixed_ff "
                    "to 1e-8 (warm start)",
        "ms": msm, "accepted_steps": stm["naccept"], "rejected_steps": stm["nreject"], "rhs_evals": stm["nfev"],
        "rhs_evals_per_s": stm["nfev"] / (msm * 1e-3), "pressure_iters": stm["pressure_iters"],
        "rmse_vs_fp64_pressure": rmse, "fp64_pressure_ms": runs["fp64"][2],
        "fp64_pressure_accepted_steps": runs["fp64"][1]["naccept"]}
    return out


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def replica_throughput(local_s, steps, world, device):
    """Whole-job throughput of `world` independent replicas that each ran `steps` solves in local_s seconds:
    all ranks' solves over the slowest rank's time (max over ranks by all_reduce; no data moves between
    replicas).  Returns (value, max seconds)."""
    tot = local_s
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([local_s], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        tot = float(tt.item())
    return steps * world / tot, tot


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="mixed", choices=["mixed", "mixed_ff", "mixed_f32dot", "f64"])
    ap.add_argument("--smoother", default="chebyshev", choices=["jacobi", "chebyshev"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-all-levels", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-only", action="store_true",
                    help="only the batched workload, with the library's default batch options (no tuner); prints "
                         "its results as one JSON line (the command line of the batched-smoother ncu capture)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the standalone-MG, differentiable-solve and porous-rollout measurements")
    ap.add_argument("--host-loop", action="store_true",
                    help="host-driven iteration loop (same kernels; profilers cannot see conditional graphs)")
    ap.add_argument("--only-solves", action="store_true",
                    help="warm-up and timed solves only (the command line used for the ncu launch list)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank)

    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    import paper_2508_12501_gb300 as P

    if args.batched_only:
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
        out = batched_workload(torch, dev, flush, torch.cuda.current_stream(dev), args.steps, tune=False)
        if rank == 0:
            print(json.dumps({"metric": "batched RHS solves/s to 1e-8", "value": out["rhs_solves_per_s"],
                              "unit": "RHS solves/s", "batched": out}), flush=True)
        return 0

    v, t = W.icosahedron()
    h = P.Hierarchy(P.Mesh(v, t), NSUB, NLEVELS, bc="gauge", sphere=True, smoother=args.smoother)
    n = h.n
    b_host = W.sh_sum(h.table(-1, "verts"), W.sh_coefficients(SEED))
    b = torch.as_tensor(b_host, device=dev)
    x = torch.empty_like(b)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()

    def timed_solves(k, mode, profile=0):
        if profile:
            h.profile(profile)
        evs = []
        st = None
        launches = 0
        for _ in range(k):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, st = h.solve(b, x, solver="mgpcg", mode=mode, tol=TOL, host_loop=args.host_loop)
            e1.record(stream)
            evs.append((e0, e1))
            launches += st.launches
        torch.cuda.synchronize(dev)
        ms = [a.elapsed_time(c) for a, c in evs]
        prof = h.profile_read() if profile else None
        if profile:
            h.profile(0)
        return ms, st, launches, prof

    # warm-up (builds the iteration graphs)
    for _ in range(args.warmup):
        h.solve(b, x, solver="mgpcg", mode=args.mode, tol=TOL, host_loop=args.host_loop)
        if not args.only_solves:
            h.solve(b, x, solver="mgpcg", mode="f64", tol=TOL)
    barrier()

    gpu_idx = None
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    if cvd:
        ids = [s for s in cvd.split(",") if s.strip()]
        gpu_idx = ids[local] if local < len(ids) else None
    else:
        gpu_idx = local
    clocks = ClockSampler(gpu_idx)
    clocks.start()

    # ---- timed region: K solves, L2 flushed before each, CUDA events per solve
    barrier()
    ms, st, launches, _ = timed_solves(args.steps, args.mode)
    barrier()
    clk = clocks.stop()
    x_mixed = x.clone()
    value, tot_s = replica_throughput(sum(ms) / 1e3, args.steps, world, dev)
    errors = {}
    if args.only_solves:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "solves/s", "iters": st.iters,
                              "gpu_launches": launches, "ms_per_step": 1e3 * tot_s / args.steps}), flush=True)
        return 0

    # ---- the other precision modes of the same solve, and the true FP64
    # residual of every returned solution (dec_residual in FP64)
    s0v = torch.as_tensor(h.table(-1, "star0"), device=dev)
    bp = b - (s0v * b).sum() / s0v.sum()  # the gauge projection the solver applies to b

    def true_rel(xv):
        return float(torch.linalg.vector_norm(h.residual(bp, xv)) / torch.linalg.vector_norm(bp))
    modes = {args.mode: {"solves_per_s": value / world, "iters": st.iters, "rel_res": st.rel_res,
                         "true_rel_res": true_rel(x_mixed)}}
    sols = {args.mode: x_mixed}
    for m in ("mixed", "mixed_ff", "mixed_f32dot", "f64"):
        if m == args.mode:
            continue
        try:
            for _ in range(2):
                h.solve(b, x, solver="mgpcg", mode=m, tol=TOL, host_loop=args.host_loop)
            msm, stm, _, _ = timed_solves(args.steps, m)
            sols[m] = x.clone()
            modes[m] = {"solves_per_s": args.steps / (sum(msm) / 1e3), "iters": stm.iters, "rel_res": stm.rel_res,
                        "true_rel_res": true_rel(sols[m])}
        except Exception as ex:  # noqa: BLE001
            errors["mode_" + m] = repr(ex)
    v64 = modes.get("f64", {}).get("solves_per_s")
    x_f64 = sols.get("f64")
    for m in modes:
        modes[m]["speedup_vs_f64"] = (modes[m]["solves_per_s"] / v64) if v64 else None

    # ---- live per-kernel timing of the same solves (event pairs on the solve stream)
    mixed = args.mode != "f64"
    cheb = args.smoother == "chebyshev"
    rows, roof, vroof = [], None, None
    try:
        _, _, _, prof = timed_solves(args.steps, args.mode, profile=2 if args.profile_all_levels else 1)
        for e in prof or []:
            by = kernel_bytes(e, h, args.mode, cheb)
            avg = e["total_ms"] / max(1, e["launches"])
            rows.append(dict(e, avg_ms=avg, bytes=by, gbs=(by / (avg * 1e-3) / 1e9) if by else None))
        peak, peak_src = peaks()
        tot_ms = sum(r["total_ms"] for r in rows) or 1.0

        def hbm_roof(r):
            # achieved: algorithmic bytes over the kernel's own duration inside the solve (an event pair around
            # each launch in the captured iteration graph, on the solve stream, L2 flushed before every solve)
            tr = ncu_traffic(r["kind"])
            gbs = r["bytes"] / (r["avg_ms"] * 1e-3) / 1e9
            out = {"bound": "hbm", "kernel": f"{r['kind']} (level {r['level']}, {r['rows']} rows)",
                   "achieved": gbs, "peak": peak, "peak_source": peak_src, "unit": "GB/s", "frac": gbs / peak,
                   "traffic": tr, "algorithmic_bytes": r["bytes"],
                   "traffic_over_algorithmic": (tr / r["bytes"]) if tr else None, "avg_launch_ms": r["avg_ms"],
                   "timing": "event pair around each launch inside the solve's iteration graph (in-solve)",
                   "share_of_profiled_time": r["total_ms"] / tot_ms}
            if r["kind"] == "smooth":
                # the same kernel and launch shape back to back on the solve stream (no event between
                # launches); the level's working set stays in L2, so this is an L2-assisted figure
                bb_ms, bb_by = h.time_kernel("smooth", level=r["level"], reps=200)
                out["l2_assisted"] = {"achieved": bb_by / (bb_ms * 1e-3) / 1e9,
                                      "frac": bb_by / (bb_ms * 1e-3) / 1e9 / peak, "avg_launch_ms": bb_ms,
                                      "timing": "200 back-to-back launches between two CUDA events"}
            return out

        def alu_roof(r):
            # FP64-pipe-bound outer kernels: FP64 instructions per row (fp64_per_row) over the in-solve duration,
            # against GB300's FP64 issue rate: 2 lanes per SM per cycle (ncu: dfma peak_sustained 2/cycle/SM)
            # x 152 SMs x the maximum SM clock
            per = fp64_per_row(r["kind"], args.mode)
            sm_clk = (clk or {}).get("sm_max_mhz") or 2070.0
            pk = 2.0 * 152 * sm_clk * 1e6 / 1e9
            ach = per * r["rows"] / (r["avg_ms"] * 1e-3) / 1e9
            return {"bound": "alu", "pipe": "fp64", "kernel": f"{r['kind']} (level {r['level']}, {r['rows']} rows)",
                    "achieved": ach, "peak": pk, "peak_source": "FP64 issue rate (2 lanes/SM/cycle x 152 SMs x "
                    f"{sm_clk:.0f} MHz)", "unit": "G FP64 instructions/s", "frac": ach / pk,
                    "fp64_instructions_per_row": per, "avg_launch_ms": r["avg_ms"],
                    "traffic": ncu_traffic(r["kind"]), "algorithmic_bytes": r["bytes"],
                    "timing": "event pair around each launch inside the solve's iteration graph (in-solve)",
                    "share_of_profiled_time": r["total_ms"] / tot_ms}

        top = max(rows, key=lambda r: r["total_ms"]) if rows else None
        if top is not None:
            roof = alu_roof(top) if fp64_per_row(top["kind"], args.mode) else (hbm_roof(top) if top["bytes"] else None)
        # the dominant kernel of the FP32 V-cycle (HBM-bound), whatever the outer iteration's precision
        cyc = [r for r in rows if r["kind"] in ("smooth", "smooth0", "residual", "restrict", "prolong") and r["bytes"]]
        if cyc:
            vroof = hbm_roof(max(cyc, key=lambda r: r["total_ms"]))
    except Exception as ex:  # noqa: BLE001
        errors["profile"] = repr(ex)

    # ---- V-cycle throughput: back-to-back FP32 cycles
    vc_ms = mdofs = None
    try:
        xb = torch.zeros(n, dtype=torch.float32, device=dev)
        bb = b.float()
        for _ in range(3):
            h.vcycle(bb, xb)
        ncyc = 20
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ncyc):
            h.vcycle(bb, xb)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        vc_ms = e0.elapsed_time(e1) / ncyc
        mdofs = n / (vc_ms * 1e-3) / 1e6
    except Exception as ex:  # noqa: BLE001
        errors["vcycle"] = repr(ex)

    # ---- end to end through the public API with host buffers
    e2e = None
    try:
        b_pin = torch.as_tensor(b_host).pin_memory()
        x_pin = torch.empty(n, dtype=torch.float64).pin_memory()
        for _ in range(2):
            h.solve(b_pin, x_pin, solver="mgpcg", mode=args.mode, tol=TOL)
        barrier()
        e2e_s = 0.0
        for _ in range(args.steps):
            flush.zero_()  # L2 flush between steps, outside the clocked call
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            xh, _ = h.solve(b_pin, x_pin, solver="mgpcg", mode=args.mode, tol=TOL)  # returns with x on the host
            e2e_s += time.perf_counter() - t0
        e2e_value, e2e_s = replica_throughput(e2e_s, args.steps, world, dev)
        e2e = {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": 8 * n,
               "d2h_bytes_per_step": 8 * n,
               "note": "host wall clock around each dec_solve_host call (pinned b and x; H2D, solve, D2H); "
                       "a 256 MB L2 flush before each call, outside the clock"}
    except Exception as ex:  # noqa: BLE001
        errors["e2e"] = repr(ex)

    cfs = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            cfs = convergence_factors(torch, dev)
        except Exception as ex:  # noqa: BLE001
            errors["convergence_factors"] = repr(ex)

    others = None
    if not args.no_configs:
        try:
            others = other_configs(torch, dev, stream)
        except Exception as ex:  # noqa: BLE001
            errors["other_configs"] = repr(ex)

    batched = None
    if not args.no_batched:
        try:
            batched = batched_workload(torch, dev, flush, stream, args.steps)
        except Exception as ex:  # noqa: BLE001
            errors["batched"] = repr(ex)

    # accuracy of each result against the plain FP64 GPU result (*0 norm)
    err = None
    if x_f64 is not None:
        for m, xm in sols.items():
            d = xm - x_f64
            modes[m]["rel_err_star0_vs_f64"] = float(torch.sqrt((s0v * d * d).sum() / (s0v * x_f64 * x_f64).sum()))
        err = modes[args.mode]["rel_err_star0_vs_f64"]

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on the other workloads, beside their GPU numbers
        try:
            ocb = oracle_other_configs()
            if others is None:
                others = {}
            if batched is not None:
                batched["cpu_baseline"] = ocb.pop("batched")
            for key, val in ocb.items():
                if key in others:
                    others[key]["cpu_baseline"] = val
                else:
                    others[key] = {"cpu_baseline": val}
        except Exception as ex:  # noqa: BLE001
            errors["cpu_baseline_other_configs"] = repr(ex)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            oh, ob = oracle_setup(args.smoother)
            ts, ores = oracle_time(oh, ob, 5)
            cpu = {"value": len(ts) / sum(ts), "unit": "solves/s", "cores": cpu_cores_used(), "kind": "oracle",
                   "sample": f"5 complete FP64 oracle MG-PCG solves of the full workload ({ores.iters} iterations "
                             f"each), hierarchy build excluded"}
        except Exception as ex:  # noqa: BLE001
            errors["cpu_baseline"] = repr(ex)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"mixed_ff": "f32 cycles + float-float outer", "mixed": "f32 cycles + f64 outer",
                      "mixed_f32dot": "f32 cycles + f64 outer with f32 dot products", "f64": "f64"}[args.mode],
            "data": "synthetic",
            "config": workload_config(args, n, world),
            "e2e": e2e, "gpu_launches": launches, "roofline": roof, "roofline_vcycle": vroof, "cpu_baseline": cpu,
            "clocks": clk,
            "iters": st.iters, "rel_res": st.rel_res, "true_rel_res": modes[args.mode]["true_rel_res"],
            "modes": modes, "fp64_solves_per_s": v64,
            "speedup_vs_fp64": (value / world / v64) if v64 else None, "mode_vs_fp64_rel_err_star0": err,
            "vcycle_ms": vc_ms, "vcycle_mdof_s": mdofs, "batched": batched, "other_configs": others, "convergence_factors": cfs,
            "kernels": [{k: (round(v_, 6) if isinstance(v_, float) else v_) for k, v_ in r.items()} for r in rows],
        }
        if errors:
            line["errors"] = errors
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
