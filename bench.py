#!/usr/bin/env python
"""Benchmark: time of one fully implicit Radau IIA stage solve to a 1e-10
relative residual, and the HBM throughput of the Vanka apply and the stage
operator against the measured peak.

Workload (default): 2D Stokes, Radau IIA(3), dt = 1/64, nu = 1, manufactured
solution u = curl(sin^2(pi x) sin^2(pi y)), p = sin(2 pi x) cos(2 pi y), on the
512 x 512 two-triangle-per-square mesh reached from an 8 x 8 coarsest mesh by
6 uniform refinements (7 levels), Taylor-Hood P2-P1: 7,068,681 coupled DoFs
over 3 stages, 263,169 vertex-star patches of up to 117 DoFs.  FGMRES(30)
right-preconditioned by V(2,2) Chebyshev [2, 8] additive Vanka.

A step is one implicit RK time step through the C ABI from the interpolated
initial state (u^0, p^0) at t = 0: stage right-hand side, the FGMRES + V-cycle
solve from a zero guess to ||F - J k|| <= 1e-10 ||F||, and the update to
(u^1, p^1).  Every step repeats the same first step, so every step does the
same work (with the steady manufactured solution, stepping on would drive F
towards zero and a relative 1e-10 below rounding).  The patch inverses and the
coarse inverse are built once in set-up (dt and nu fixed) and reused every
step; set-up time is reported separately as setup_s.

--impl reference times the oracle (plain FP64 CPU restatement) on a bounded
sample of the same workload.
"""
import os
import sys

# the oracle (reference arm, CPU baseline) gets every host core for its BLAS;
# the GPU arm's own process keeps one BLAS thread (its oracle timing runs in a
# fresh subprocess)
_BLAS_THREADS = str(os.cpu_count() or 1) if "reference" in sys.argv else "1"
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, _BLAS_THREADS)

import argparse  # noqa: E402
import hashlib  # noqa: E402
import json  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "IRK stage solve time to 1e-10 resid; Vanka apply+SpMV HBM GB/s vs peak"
UNIT = "s/solve"
FALLBACK_HBM = 6800.0
# FP64 ALU peak of GB300 from the unit count and the maximum clock: 152 SMs x
# 2 FP64 FMA per clock x 2 flop x 2070 MHz.  The run measures it as well
# (irkmg_probe_peak, measure_alu_peaks) and reports against the measurement.
FP64_NOMINAL_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12

# DRAM traffic of the finest-level Vanka kernel from an ncu capture, as the
# ratio (dram__bytes_read + dram__bytes_write) / algorithmic bytes of the
# captured launch, keyed by kernel and by the hash of the kernel's source file
# at capture time; reported as ratio x algorithmic bytes per launch, null once
# the source has changed.  Captures: profiles/vanka_apply_128x128.md,
# profiles/vanka_apply_kron_fp64_256x256.md,
# profiles/vanka_apply_kron_fx_pair_128x128.md,
# profiles/vanka_apply_kron_pair32_256x256.md.
NCU_TRAFFIC = {
    ("k_vanka_apply", "8f81809572f0"): 0.97,
    ("k_vanka_apply_kron", "60c2ce575b6a"): 1.02,
    ("k_vanka_apply_kron_fx_pair", "6850cc0d8407"): 1.096,
    ("k_vanka_apply_kron_fx_pair", "4975a091f1c6"): 1.089,
    ("k_vanka_apply_kron_pair32", "8f68162f379b"): 1.110,
}
KERNEL_FILE = {"k_vanka_apply": "k_patch.cu", "k_vanka_apply_staged": "k_patch.cu",
               "k_vanka_apply_lu": "k_patch_big.cu", "k_vanka_apply_kron": "k_patch_kron.cu",
               "k_vanka_apply_kron_staged": "k_patch_kron.cu",
               "k_vanka_apply_kron_big": "k_patch_kron.cu",
               "k_vanka_apply_kron_ws": "k_patch_kron.cu",
               "k_vanka_apply_kron_pair32": "k_patch_kron.cu",
               "k_vanka_apply_kron_fx": ("k_patch_fixed.cu", "fx_patch.cuh", "fx_math.h"),
               "k_vanka_apply_kron_fx_staged": ("k_patch_fixed.cu", "fx_patch.cuh", "fx_math.h"),
               "k_vanka_apply_kron_fx_pair": ("k_patch_fixed.cu", "fx_patch.cuh", "fx_math.h")}


def kernel_source_hash(kernel="k_vanka_apply_kron"):
    files = KERNEL_FILE[kernel]
    h = hashlib.sha1()
    for f in (files,) if isinstance(files, str) else files:
        with open(os.path.join(ROOT, "paper_2202_07381_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def measure_alu_peaks(irkmg, stream):
    """FP64 and FP32 FMA rates (TFLOP/s) and the 32 x 32 -> 64-bit integer
    multiply-add rate (T/s) of this GPU, each from one timed launch of
    irkmg_probe_peak (about 10-20 ms each)."""
    h = stream.cuda_stream
    return {"fp64_tflops": irkmg.irkmg_probe_peak(0, 4000, h) / 1e12,
            "fp32_tflops": irkmg.irkmg_probe_peak(1, 200000, h) / 1e12,
            "mad_wide_s32_tops": irkmg.irkmg_probe_peak(2, 100000, h) / 1e12,
            "fp64_nominal_tflops": FP64_NOMINAL_TFLOPS,
            "how": "irkmg_probe_peak: one launch of 8 CTAs x 256 threads per SM, 8 independent "
                   "multiply-add chains per thread, CUDA events on the launch stream"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM, "fallback"


def workload(args):
    if getattr(args, "dim", 2) == 3:
        n = args.n3
        levels = int(round(np.log2(n / 4))) + 1
        if n < 8 or 4 * 2 ** (levels - 1) != n:
            raise SystemExit("--n3 must be 4 * 2^k with k >= 1")
        return dict(name=f"3D Stokes RadauIIA(2) {n}^3 cubes x 6 tets ({levels} levels from 4^3), "
                         "dt=1/16, FP32 blocked patch LU", n0=4, levels=levels, s=2, dt=1 / 16,
                    nu=1.0, n=n, dim=3, cheb=(2.0, 17.0))
    if args.small:
        return dict(name="2D Stokes RadauIIA(2) 8x8 (3 levels), dt=1/8", n0=2, levels=3, s=2,
                    dt=1 / 8, nu=1.0, n=8)
    n = args.n
    levels = int(round(np.log2(n / 8))) + 1
    if n < 16 or 8 * 2 ** (levels - 1) != n:
        raise SystemExit("--n must be 8 * 2^k with k >= 1")
    return dict(name=f"2D Stokes RadauIIA(3) {n}x{n} ({levels} levels from 8x8), dt=1/64", n0=8,
                levels=levels, s=3, dt=1 / 64, nu=1.0, n=n)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# reference arm: the oracle on a bounded sample
# ---------------------------------------------------------------------------
class _TimedOp:
    """A matrix whose products `@` add their wall time to acc[key] (timing of
    the oracle's phases; the product itself is the matrix's own)."""

    def __init__(self, A, acc, key):
        self.A, self.acc, self.key = A, acc, key

    def __matmul__(self, x):
        t = time.perf_counter()
        y = self.A @ x
        self.acc[self.key] += time.perf_counter() - t
        return y

    @property
    def T(self):
        return _TimedOp(self.A.T, self.acc, self.key)

    def __getattr__(self, name):
        return getattr(self.A, name)


def _timed_call(fn, acc, key):
    def wrapped(*a, **k):
        t = time.perf_counter()
        y = fn(*a, **k)
        acc[key] += time.perf_counter() - t
        return y
    return wrapped


def oracle_run(wl, n_sample, solves=1):
    """The oracle's set-up and FGMRES + V-cycle solve of the workload's problem
    on an n_sample x n_sample finest mesh (same tableau, dt, nu, smoother,
    coarsest mesh and tolerance), timed by phase: the stage operator products,
    the Vanka corrections, the transfers, the coarsest solves, and the rest of
    FGMRES (Gram-Schmidt, Givens, vector updates).  The phases are timed by
    wrapping the oracle's own objects; its arithmetic is untouched."""
    from oracle import fgmres, mg, problem, tableau
    A, b, c = tableau.radau_iia(wl["s"])
    levels = int(round(np.log2(n_sample / wl["n0"]))) + 1
    w0, c0 = time.perf_counter(), time.process_time()
    H = mg.Hierarchy(*synth.square_mesh(wl["n0"]), levels, A, wl["dt"], nu=wl["nu"])
    setup_s = time.perf_counter() - w0
    F, _, _ = problem.mms_rhs(H, c)
    acc = {"stage_operator": 0.0, "vanka": 0.0, "transfers": 0.0, "coarse": 0.0}
    for l, L in enumerate(H.levels):
        L.J = _TimedOp(L.J, acc, "stage_operator")
        if l > 0:
            L.P = _TimedOp(L.P, acc, "transfers")
            L.vanka.correction = _timed_call(L.vanka.correction, acc, "vanka")
    H.coarse_solve = _timed_call(H.coarse_solve, acc, "coarse")
    times, its = [], None
    for _ in range(solves):
        t0 = time.perf_counter()
        _, its, _ = fgmres.fgmres(H.finest.J, F, H.vcycle, rtol=1e-10, project=H.project_pressure)
        times.append(time.perf_counter() - t0)
    wall, cpu = time.perf_counter() - w0, time.process_time() - c0
    solve = float(np.mean(times))
    phases = {k: v / solves for k, v in acc.items()}
    phases["fgmres_rest"] = solve - sum(phases.values())
    return {"n": n_sample, "levels": levels, "N": H.finest.N, "iters": its, "setup_s": setup_s,
            "solve_s": solve, "solves": solves, "phases_s": phases,
            "cpu_time_over_wall": cpu / wall, "blas_threads": int(os.environ["OPENBLAS_NUM_THREADS"])}


def oracle_fit(runs, n_full):
    """t_solve = a N^alpha through the two largest measured sizes, evaluated at
    the workload's N: an extrapolation, labelled as such."""
    r1, r2 = sorted(runs, key=lambda r: r["N"])[-2:]
    alpha = float(np.log(r2["solve_s"] / r1["solve_s"]) / np.log(r2["N"] / r1["N"]))
    return {"law": "t_solve = a * N^alpha through the two largest measured sizes",
            "alpha": alpha, "N": n_full,
            "extrapolated_s_per_solve": r2["solve_s"] * (n_full / r2["N"]) ** alpha}


def oracle_baseline_subprocess(args, sizes=(32, 64)):
    """The oracle's per-phase timings at the given sizes, run in a fresh
    process whose BLAS may use every host core (this process keeps one)."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--oracle-sizes",
           ",".join(map(str, sizes)), "--n", str(args.n)]
    env = dict(os.environ)
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(os.cpu_count() or 1)
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, env=env)
    if r.returncode != 0:
        return None
    return json.loads(r.stdout.strip().splitlines()[-1])


def max_over_ranks(x, device):
    """Largest x over the ranks of the default process group (the slowest
    replica's time decides the job's time)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_value(ms_max, steps, world):
    """Whole-job seconds per solve: world replicas each ran `steps` solves in
    at most ms_max milliseconds."""
    return ms_max * 1e-3 / (steps * world)


def base_config(wl):
    """Workload description shared by both arms (sizes from the mesh
    formulas: (n+1)^2 vertices, (2n-1)^2 free P2 nodes in 2D)."""
    n, d = wl["n"], wl.get("dim", 2)
    nv, nf = (n + 1) ** d, (2 * n - 1) ** d
    return {"workload": wl["name"], "N": wl["s"] * (d * nf + nv), "patches_finest": nv,
            "smoother": "Chebyshev[%g,%g] V(2,2)" % wl.get("cheb", (2.0, 8.0)),
            "fgmres_restart": 30, "rtol": 1e-10}


def run_reference(args, wl, rank):
    """The oracle on the host cores.  Each step is one FGMRES solve of the
    workload's problem on a bounded sample mesh (64 x 64, 32 x 32 for long
    runs), after one set-up; the line reports the measured time of that size
    and names it in config.  --oracle-sizes: per-phase timings at several
    sizes plus the fitted extrapolation (the GPU arm's cpu_baseline)."""
    if rank != 0:
        return
    n_full = base_config(wl)["N"]
    if args.oracle_sizes:
        runs = [oracle_run(wl, int(n)) for n in args.oracle_sizes.split(",")]
        print(json.dumps({"runs": runs, "fit": oracle_fit(runs, n_full) if len(runs) > 1 else None,
                          "cores_available": os.cpu_count()}), flush=True)
        return
    n_sample = 8 if args.small else (64 if args.steps + min(args.warmup, 1) <= 30 else 32)
    a2 = argparse.Namespace(**vars(args))
    a2.n = n_sample
    swl = workload(a2)
    run = oracle_run(swl, n_sample, solves=args.steps + min(args.warmup, 1))
    v = run["solve_s"]
    line = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": base_config(swl),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"oracle FGMRES + V-cycle solve at {n_sample}x{n_sample} "
                                       f"({run['levels']} levels, N={run['N']}, {run['iters']} "
                                       f"iterations), mean of {run['solves']} solves after one "
                                       f"set-up ({run['setup_s']:.1f} s); BLAS threads "
                                       f"{run['blas_threads']}, CPU time / wall "
                                       f"{run['cpu_time_over_wall']:.2f}",
                             "phases_s": run["phases_s"]},
            "measured_size": {"n": n_sample, "N": run["N"], "iters": run["iters"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def make_context(irkmg, wl, precision, stream, apply_variant=0, patch_form=0, patch_fixed=0,
                 op_fixed=0):
    A, b, c = irkmg.irkmg_radau_iia(wl["s"])
    o = irkmg.irkmg_default_options()
    o.apply_variant = apply_variant
    o.patch_form = patch_form
    o.patch_fixed = patch_fixed
    o.op_fixed = op_fixed if wl.get("dim", 2) == 2 else 0
    if "cheb" in wl:
        o.cheb_lo, o.cheb_hi = wl["cheb"]
    o.nlevels = wl["levels"]
    o.patch_precision = precision
    o.rtol = 1e-10
    o.maxit = 300
    mesh = synth.cube_mesh(wl["n0"]) if wl.get("dim", 2) == 3 else synth.square_mesh(wl["n0"])
    t0 = time.perf_counter()
    ctx = irkmg.irkmg_setup(*mesh, A, b, c, wl["dt"], wl["nu"], o, stream=stream)
    return ctx, time.perf_counter() - t0, c


def initial_data(irkmg, ctx, wl, c):
    xy = irkmg.irkmg_p2_coords(ctx)
    free = irkmg.irkmg_free_nodes(ctx)
    nv = ctx.finest["nv"]
    if wl.get("dim", 2) == 3:
        u0 = np.concatenate(synth.mms3_velocity(*xy[free].T))
        p0 = synth.mms3_pressure(*xy[:nv].T)
        f1 = np.concatenate(synth.mms3_forcing(*xy.T, nu=wl["nu"]))
        return u0, p0 - p0.mean(), np.concatenate([f1 for _ in c])
    ux, uy = synth.mms_velocity(xy[free, 0], xy[free, 1])
    u0 = np.concatenate([ux, uy])
    p0 = synth.mms_pressure(xy[:nv, 0], xy[:nv, 1])
    p0 = p0 - p0.mean()
    fx, fy = synth.mms_forcing(xy[:, 0], xy[:, 1], nu=wl["nu"])
    f = np.concatenate([np.concatenate([fx, fy]) for _ in c])   # steady: same at every c_i
    return u0, p0, f


def run_form(irkmg, torch, wl, args, dev, stream, k_ref, precision, patch_form, patch_fixed=0,
             op_fixed=0):
    """Another form on the same workload (FP32 patches and/or decoupled patch
    solves): time per solve, iterations, the difference of its solution from
    the plain FP64 form's, and the finest-level Vanka roofline from the live
    trace (FP64 patches: FP64-pipe bound; FP32 patches: HBM bound)."""
    ctx, setup_s, c = make_context(irkmg, wl, precision, stream.cuda_stream, 0, patch_form,
                                   patch_fixed, op_fixed)
    u0, p0, f = initial_data(irkmg, ctx, wl, c)
    T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    u, p, fd = T(u0), T(p0), T(f)
    F = torch.zeros(ctx.N(), dtype=torch.float64, device=dev)
    k = torch.zeros_like(F)
    irkmg.irkmg_stage_rhs(ctx, u, p, fd, F)
    stats = []
    for i in range(args.warmup + args.steps):
        if i == args.warmup:
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        irkmg.irkmg_stage_rhs(ctx, u, p, fd, F)
        k.zero_()
        stats.append(irkmg.irkmg_solve(ctx, F, k))
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    diff = float(irkmg_rel_diff(torch, k, k_ref))
    # one traced solve for the finest-level Vanka figures
    irkmg.irkmg_trace_enable(ctx, True)
    k.zero_()
    irkmg.irkmg_solve(ctx, F, k)
    torch.cuda.synchronize()
    tr = irkmg.irkmg_trace_read(ctx)
    irkmg.irkmg_trace_enable(ctx, False)
    out = {"ms_per_step": ms, "iters": stats[-1]["iters"],
           "rel_residual": stats[-1]["rfinal"] / stats[-1]["r0"], "setup_s": setup_s,
           "rel_diff_vs_fp64_solution": diff, "patch_precision": precision,
           "patch_form": patch_form, "patch_fixed": patch_fixed, "op_fixed": op_fixed,
           "apply_kernel_per_level": [lv["apply_kernel"] for lv in ctx.levels[1:]],
           "factor_bytes_finest": ctx.finest["factor_bytes"]}
    if tr["vanka_ms"]:
        nvl = max(tr["vanka_launches"], 1)
        gbs = tr["vanka_bytes"] / (tr["vanka_ms"] * 1e-3) / 1e9
        tf = tr["vanka_flops"] / (tr["vanka_ms"] * 1e-3) / 1e12
        hbm, hbm_kind = peaks()
        out["vanka_finest"] = {"avg_launch_ms": tr["vanka_ms"] / nvl, "launches": tr["vanka_launches"],
                               "bytes_per_launch": tr["vanka_bytes"] / nvl,
                               "flops_per_launch": tr["vanka_flops"] / nvl,
                               "hbm_gbs": gbs, "hbm_frac": gbs / hbm, "tflops": tf,
                               "fp64_frac": (tf / FP64_NOMINAL_TFLOPS
                                             if precision == 64 and not patch_fixed else None),
                               "hbm_peak_source": f"{hbm_kind} hbm_gbs"}
    if patch_fixed:
        out["finest_correction_ms_per_shape"] = shape_sweep(irkmg, torch, ctx, dev, stream)
    # 2D patches are inverted in FP64 (Gauss-Jordan in shared memory) whatever
    # precision they are stored in
    out["factor"] = factor_roofline(irkmg, ctx, wl, stream, 64)
    ctx.close()
    return out


def factor_roofline(irkmg, ctx, wl, stream, prec):
    """Set-up work, after the timed regions: the finest level's patch
    factorisation (explicit inverses, 2 m^3 flops per m x m block), timed by
    the library's events while irkmg_update redoes the set-up for the same dt
    and nu; FLOP/s against the measured FMA rate of the precision the
    factorisation computes in (prec)."""
    irkmg.irkmg_trace_enable(ctx, True)
    irkmg.irkmg_update(ctx, wl["dt"], wl["nu"])
    ftr = irkmg.irkmg_trace_read(ctx)
    irkmg.irkmg_trace_enable(ctx, False)
    if not (ftr["factor_launches"] and ftr["factor_ms"] > 0):
        return None
    alu = measure_alu_peaks(irkmg, stream)
    pk = alu["fp64_tflops"] if prec == 64 else alu["fp32_tflops"]
    tf = ftr["factor_flops"] / (ftr["factor_ms"] * 1e-3) / 1e12
    return {"bound": "alu", "kernel": "patch factorisation (finest level, set-up)",
            "achieved": tf, "peak": pk, "unit": "TFLOP/s", "frac": tf / pk,
            "peak_source": "FP%d FMA rate measured by irkmg_probe_peak" % prec,
            "ms": ftr["factor_ms"], "flops": ftr["factor_flops"],
            "flops_counted": "2 m^3 per m x m block inverted (LU 2/3 m^3 + inverse 4/3 m^3)"}


def shape_sweep(irkmg, torch, ctx, dev, stream, reps=10):
    """Time of one finest-level Vanka correction (one launch over all patches
    plus the per-DoF sum) for every launch shape of the level's kernel, pinned
    with irkmg_level_set_apply; the tuned shape is restored afterwards."""
    fin = ctx.nlevels - 1
    keep = (ctx.finest["apply_shape"], ctx.finest["single_launch"])
    r = torch.rand(ctx.N(), dtype=torch.float64, device=dev)
    c = torch.zeros_like(r)
    res = {}
    for shape in range(16):
        try:
            irkmg.irkmg_level_set_apply(ctx, fin, shape, 1)
        except irkmg.IrkmgError as e:
            if "does not fit" in str(e):
                continue    # a later shape may still fit
            break           # no such launch shape: the list is exhausted
        for _ in range(2):
            irkmg.irkmg_vanka_correction(ctx, r, c)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            irkmg.irkmg_vanka_correction(ctx, r, c)
        e1.record(stream)
        torch.cuda.synchronize()
        res[f"kernel{ctx.finest['apply_kernel']}_shape{shape}"] = e0.elapsed_time(e1) / reps
    irkmg.irkmg_level_set_apply(ctx, fin, *keep)
    return res


def mesh_sweep(irkmg, torch, wl, args, dev, stream, prec, fixed, sizes=(32, 64, 128, 256)):
    """FGMRES iterations of the same stage solve (same tableau, dt, smoother,
    patch form and tolerance) on coarser finest meshes from the same 8 x 8
    coarsest mesh: the mesh-independence figure of Section 5.1, Table 1."""
    out = {}
    for n in sizes:
        w = dict(wl, n=n, levels=int(round(np.log2(n / wl["n0"]))) + 1)
        ctx, _, c = make_context(irkmg, w, prec, stream.cuda_stream, 0, args.patch_form, fixed)
        u0, p0, f = initial_data(irkmg, ctx, w, c)
        T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
        F = torch.zeros(ctx.N(), dtype=torch.float64, device=dev)
        irkmg.irkmg_stage_rhs(ctx, T(u0), T(p0), T(f), F)
        k = torch.zeros_like(F)
        st = irkmg.irkmg_solve(ctx, F, k)
        out[n] = {"iters": st["iters"], "levels": w["levels"], "N": ctx.N(),
                  "rel_residual": st["rfinal"] / st["r0"], "status": st["status"]}
        ctx.close()
    return out


def irkmg_rel_diff(torch, a, b):
    # pressure is defined up to a constant per stage: compare velocities only
    return (a - b).norm() / b.norm()


def run_batched(args, dev, stream, patch_form=1, patch_fixed=1):
    """64 independent Oseen stage systems (lid-driven cavity, seeded smooth
    wind with max |w| = 1 at the P2 nodes, Re ~ U[100, 1000], dt log-uniform in
    [1e-3, 1e-1], meshes from {32, 64, 128, 256}^2 over an 8 x 8 coarsest mesh,
    Radau IIA(2), FP64 patches in the given form, by default decoupled with
    fixed-point mat-vecs): solved one after another with irkmg_solve, then
    together with irkmg_batch_solve."""
    import torch
    from paper_2202_07381_gb300 import irkmg
    specs = synth.oseen_batch(0, args.batch)
    A, b, c = irkmg.irkmg_radau_iia(2)
    ctxs, Fs = [], []
    t0 = time.perf_counter()
    for sp in specs:
        o = irkmg.irkmg_default_options()
        o.nlevels = int(round(np.log2(sp["n"] / 8))) + 1
        o.maxit = 600
        o.patch_form = patch_form
        o.patch_fixed = patch_fixed if patch_form != 0 else 0
        ctx = irkmg.irkmg_setup(*synth.square_mesh(8), A, b, c, sp["dt"], sp["nu"], o,
                                stream=stream.cuda_stream)
        xy = irkmg.irkmg_p2_coords(ctx)
        wx, wy = synth.wind_field(xy[:, 0], xy[:, 1], synth.wind_coefficients(sp["wind_seed"]))
        sc = np.max(np.hypot(wx, wy))
        irkmg.irkmg_set_wind(ctx, np.stack([wx / sc, wy / sc], axis=1))
        lx, ly = synth.lid_velocity(xy[:, 0], xy[:, 1])
        T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
        F = torch.zeros(ctx.N(), dtype=torch.float64, device=dev)
        irkmg.irkmg_stage_rhs_full(ctx, T(np.concatenate([lx, ly])), T(np.zeros(ctx.finest["nv"])),
                                   T(np.zeros(2 * 2 * ctx.finest["np2"])), F)
        ctxs.append(ctx)
        Fs.append(F)
    setup_s = time.perf_counter() - t0
    ks_seq = [torch.zeros_like(F) for F in Fs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq = [irkmg.irkmg_solve(ctx, F, k) for ctx, F, k in zip(ctxs, Fs, ks_seq)]
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    batch = irkmg.Batch(ctxs)
    persistent = batch.persistent
    t_graph = None
    if persistent:   # the same batch with one V-cycle graph per system
        batch.persistent = False
        ks = [torch.zeros_like(F) for F in Fs]
        batch.solve(Fs, ks)          # captures the graphs
        ks = [torch.zeros_like(F) for F in Fs]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        batch.solve(Fs, ks)
        torch.cuda.synchronize()
        t_graph = time.perf_counter() - t0
        batch.persistent = True
    ks = [torch.zeros_like(F) for F in Fs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bst = batch.solve(Fs, ks)
    torch.cuda.synchronize()
    t_bat = time.perf_counter() - t0
    batch.close()
    diff = max(float((k - kr).norm() / kr.norm()) for k, kr in zip(ks, ks_seq))
    its = [s_["iters"] for s_ in bst]
    dofs = sum(c_.N() for c_ in ctxs)
    ok = all(s_["status"] == 0 for s_ in bst) and all(s_["status"] == 0 for s_ in seq)
    for c_ in ctxs:
        c_.close()
    return {"workload": f"{len(specs)} Oseen stage systems, Radau IIA(2), lid-driven cavity, "
                        "meshes from {32,64,128,256}^2, Re ~ U[100,1000], dt in [1e-3,1e-1]",
            "systems": len(specs), "dofs_total": dofs, "all_converged": ok,
            "sequential_s": t_seq, "batched_s": t_bat, "speedup": t_seq / t_bat,
            "persistent_launch": persistent, "batched_graphs_s": t_graph,
            "patch_form": patch_form, "patch_fixed": patch_fixed if patch_form != 0 else 0,
            "s_per_solve_batched": t_bat / len(specs), "iters_min_mean_max":
            [min(its), float(np.mean(its)), max(its)], "max_rel_diff_vs_sequential": diff,
            "setup_s": setup_s}


def run_ns(args, dev, stream, n=128, re=1000.0, dt=0.01, steps=2):
    """Navier-Stokes by Newton's method (Section 3.2): lid-driven cavity at
    Re = 1000 on n x n (from 8 x 8), Radau IIA(2), dt = 0.01, from rest; each
    time step solves the stage equations by inexact Newton (Eisenstat-Walker
    tolerances, V-cycle-preconditioned FGMRES), the first from k = 0 and the
    next from the previous step's stages.  Time per step includes the host
    assembly of the Newton blocks at every Newton step."""
    import torch
    from paper_2202_07381_gb300 import irkmg
    A, b, c = irkmg.irkmg_radau_iia(2)
    o = irkmg.irkmg_default_options()
    o.nlevels = int(round(np.log2(n / 8))) + 1
    o.maxit = 600
    t0 = time.perf_counter()
    ctx = irkmg.irkmg_setup(*synth.square_mesh(8), A, b, c, dt, 1.0 / re, o,
                            stream=stream.cuda_stream)
    setup_s = time.perf_counter() - t0
    L = ctx.finest
    xy = irkmg.irkmg_p2_coords(ctx)
    free = torch.tensor(irkmg.irkmg_free_nodes(ctx), device=dev)
    lx, ly = synth.lid_velocity(xy[:, 0], xy[:, 1])
    T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    un = T(np.concatenate([lx, ly]))
    pn = torch.zeros(L["nv"], dtype=torch.float64, device=dev)
    f = torch.zeros(2 * 2 * L["np2"], dtype=torch.float64, device=dev)
    k = torch.zeros(L["N"], dtype=torch.float64, device=dev)
    m, nf, np2 = L["m"], L["nf"], L["np2"]
    out = []
    for step in range(steps):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        st = irkmg.irkmg_ns_newton(ctx, un, pn, f, k, atol=1e-9, maxit=30)
        torch.cuda.synchronize()
        out.append({"s": time.perf_counter() - t1, "newton_iters": st["newton_iters"],
                    "linear_iters": st["linear_iters"], "f0": st["f0"], "ffinal": st["ffinal"]})
        for j in range(2):   # u^{n+1} = u^n + dt sum_j b_j k_j (free nodes), p likewise
            kj = k[j * m:(j + 1) * m]
            for d in range(2):
                un[d * np2 + free] += dt * b[j] * kj[d * nf:(d + 1) * nf]
            pn += dt * b[j] * kj[2 * nf:]
    ctx.close()
    return {"workload": f"Navier-Stokes lid-driven cavity Re={re:g}, {n}x{n}, Radau IIA(2), "
                        f"dt={dt:g}, Newton + Eisenstat-Walker, FP64 dense patches",
            "N": L["N"], "setup_s": setup_s, "steps": out,
            "s_per_step": float(np.mean([x["s"] for x in out]))}


def run_adjoint(args, dev, stream, n=128, s=2, dt=1 / 32, nsteps=8, every=2):
    """Gradient of J = 1/2 ||u(T) - u_target||_M^2 (u_target: the manufactured
    velocity) with respect to a per-cell P0 forcing control (seeded N(0,1)) and
    nu through nsteps implicit Radau IIA(s) steps of dt on n x n, checkpoints
    every `every` steps (irkmg_step / irkmg_adjoint_step behind
    torch.autograd): wall time of forward + backward, and the agreement of the
    directional derivatives with central differences of the forward model."""
    import torch
    from paper_2202_07381_gb300 import irkmg
    from paper_2202_07381_gb300.adjoint import TrackingProblem, tracking_objective
    A, b, c = irkmg.irkmg_radau_iia(s)
    o = irkmg.irkmg_default_options()
    o.nlevels = int(round(np.log2(n / 8))) + 1
    o.patch_form = args.patch_form
    o.patch_fixed = args.patch_fixed if args.patch_form != 0 else 0
    o.rtol, o.atol, o.maxit = 1e-12, 1e-15, 400
    t0 = time.perf_counter()
    ctx = irkmg.irkmg_setup(*synth.square_mesh(8), A, b, c, dt, 1.0, o, stream=stream.cuda_stream)
    setup_s = time.perf_counter() - t0
    xy = irkmg.irkmg_p2_coords(ctx)
    free = irkmg.irkmg_free_nodes(ctx)
    nv = ctx.finest["nv"]
    ux, uy = synth.mms_velocity(xy[free, 0], xy[free, 1])
    u0 = np.concatenate([ux, uy])
    p0 = synth.mms_pressure(xy[:nv, 0], xy[:nv, 1])
    fx, fy = synth.mms_forcing(xy[:, 0], xy[:, 1], nu=1.0)
    T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    prob = TrackingProblem(ctx, dt, T(u0), T(p0 - p0.mean()),
                           T(np.concatenate([np.concatenate([fx, fy])] * s)), T(u0), nsteps, every)
    theta = T(synth.normal(7, 2 * ctx.finest["nc"]))
    times = []
    for rep in range(2):                       # the first pass is a warm-up
        th = theta.clone().requires_grad_(True)
        nu = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        J = tracking_objective(th, nu, prob)
        J.backward()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t1)
    d = T(synth.normal(11, theta.numel()))
    with torch.no_grad():                      # J is quadratic in theta: unit step
        fd = (prob.objective(theta + d, 1.0) - prob.objective(theta - d, 1.0)) / 2.0
    ad = float((th.grad * d).sum())
    hn = 1e-6
    fdn = (prob.objective(theta, 1.0 + hn) - prob.objective(theta, 1.0 - hn)) / (2 * hn)
    its = [st_["iters"] for st_ in prob.stats]
    ctx.close()
    return {"workload": f"adjoint: Radau IIA({s}) {n}x{n}, {nsteps} steps dt={dt:g}, checkpoints "
                        f"every {every}, gradient of 1/2||u(T)-u_target||_M^2 w.r.t. a P0 forcing "
                        "field (N(0,1)) and nu",
            "forward_backward_s": times[-1], "setup_s": setup_s, "objective": float(J.detach()),
            "fd_rel_err_theta": abs(fd - ad) / abs(fd), "fd_rel_err_nu": abs(fdn - nu.grad.item()) / abs(fdn),
            "rtol": 1e-12, "fgmres_iters_min_max": [min(its), max(its)],
            "patch_form": args.patch_form, "patch_fixed": o.patch_fixed}


def run_3d(args, dev, stream, patch_form=1):
    """The 3D configuration (Kuhn tetrahedra, FP32 blocked patch LU, FP64
    FGMRES): time per stage solve, iterations, residual, roofline of the
    finest-level patch solves."""
    import torch
    from paper_2202_07381_gb300 import irkmg
    a3 = argparse.Namespace(**vars(args))
    a3.dim = 3
    wl = workload(a3)
    ctx, setup_s, c = make_context(irkmg, wl, 32, stream.cuda_stream, 0, patch_form)
    u0, p0, f = initial_data(irkmg, ctx, wl, c)
    T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    u, p, fd = T(u0), T(p0), T(f)
    F = torch.zeros(ctx.N(), dtype=torch.float64, device=dev)
    k = torch.zeros_like(F)
    irkmg.irkmg_stage_rhs(ctx, u, p, fd, F)
    stats = []
    for i in range(args.warmup + args.steps):
        if i == args.warmup:
            torch.cuda.synchronize()
            irkmg.irkmg_trace_enable(ctx, True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        irkmg.irkmg_stage_rhs(ctx, u, p, fd, F)
        k.zero_()
        stats.append(irkmg.irkmg_solve(ctx, F, k))
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    tr = irkmg.irkmg_trace_read(ctx)
    hbm, _ = peaks()
    gbs = tr["vanka_bytes"] / (tr["vanka_ms"] * 1e-3) / 1e9 if tr["vanka_ms"] else None
    out = {"workload": wl["name"], "N": ctx.N(), "patches_finest": ctx.finest["nv"],
           "patch_form": patch_form, "apply_kernel_finest": ctx.finest["apply_kernel"],
           "factor_bytes_finest": ctx.finest["factor_bytes"],
           "max_patch_dofs": ctx.finest["max_patch_dofs"], "ms_per_step": ms,
           "iters": stats[-1]["iters"], "rel_residual": stats[-1]["rfinal"] / stats[-1]["r0"],
           "setup_s": setup_s, "all_converged": all(s_["status"] == 0 for s_ in stats),
           "vanka_lu_finest": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                               "frac": gbs / hbm if gbs else None,
                               "avg_launch_ms": tr["vanka_ms"] / max(tr["vanka_launches"], 1)}}
    out["factor"] = factor_roofline(irkmg, ctx, wl, stream, 32)
    ctx.close()
    return out


def run_ours(args, wl, rank, world, local_rank):
    import torch
    from paper_2202_07381_gb300 import irkmg

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    prec = 32 if (args.form == "fp32" or wl.get("dim", 2) == 3) else 64
    fixed = args.patch_fixed if prec == 64 and args.patch_form != 0 else 0
    opfx = args.op_fixed if wl.get("dim", 2) == 2 else 0
    ctx, setup_s, c = make_context(irkmg, wl, prec, stream.cuda_stream, args.apply,
                                   args.patch_form, fixed, opfx)
    u0, p0, f = initial_data(irkmg, ctx, wl, c)
    T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    u, p, fd = T(u0), T(p0), T(f)
    u1, p1 = torch.empty_like(u), torch.empty_like(p)
    N = ctx.finest["N"]
    F = torch.zeros(N, dtype=torch.float64, device=dev)
    k = torch.zeros_like(F)
    stats = []

    def step():
        irkmg.irkmg_stage_rhs(ctx, u, p, fd, F)
        k.zero_()
        st = irkmg.irkmg_solve(ctx, F, k)
        u1.copy_(u)
        p1.copy_(p)
        irkmg.irkmg_advance(ctx, k, u1, p1)
        stats.append(st)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stats.clear()
    barrier = (lambda: torch.distributed.barrier()) if world > 1 else (lambda: None)
    # tracing off in the timed region: the library only counts its launches
    irkmg.irkmg_trace_enable(ctx, False)
    with ClockSampler(local_rank) as clk:
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # the timed region is the profiler range (a no-op unless a profiler
        # started with profiling off is attached, e.g. ncu --profile-from-start off)
        torch.cuda.profiler.start()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        barrier()
        time.sleep(0.25)
    ms = e0.elapsed_time(e1)
    launches = irkmg.irkmg_trace_read(ctx)["launches"]
    if world > 1:
        ms = max_over_ranks(ms, dev)
    iters = [s_["iters"] for s_ in stats]
    resid = [s_["rfinal"] / max(s_["r0"], 1e-300) for s_ in stats]
    assert all(s_["status"] == 0 for s_ in stats), stats

    # end to end: host state in pinned memory, copies inside the timed region
    hu = torch.tensor(u0, dtype=torch.float64).pin_memory()
    hp = torch.tensor(p0, dtype=torch.float64).pin_memory()
    hf = torch.tensor(f, dtype=torch.float64).pin_memory()
    hu1, hp1 = torch.empty_like(hu).pin_memory(), torch.empty_like(hp).pin_memory()
    h2d = (hu.numel() + hp.numel() + hf.numel()) * 8
    d2h = (hu1.numel() + hp1.numel()) * 8
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u.copy_(hu, non_blocking=True)
        p.copy_(hp, non_blocking=True)
        fd.copy_(hf, non_blocking=True)
        irkmg.irkmg_stage_rhs(ctx, u, p, fd, F)
        k.zero_()
        irkmg.irkmg_solve(ctx, F, k)
        u1.copy_(u)
        p1.copy_(p)
        irkmg.irkmg_advance(ctx, k, u1, p1)
        hu1.copy_(u1, non_blocking=True)
        hp1.copy_(p1, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    barrier()
    if world > 1:
        e2e_s = max_over_ranks(e2e_s, dev)

    assert base_config(wl)["N"] == N and base_config(wl)["patches_finest"] == ctx.finest["nv"]
    # one traced step after the timed regions: CUDA events around every
    # finest-level Vanka, operator, transfer and Gram-Schmidt launch
    irkmg.irkmg_trace_enable(ctx, True)
    stats_keep = list(stats)
    step()
    trace = irkmg.irkmg_trace_read(ctx)
    irkmg.irkmg_trace_enable(ctx, False)
    stats[:] = stats_keep
    # 2D patches are inverted in FP64; the 3D blocked LU computes in FP32
    factor = (factor_roofline(irkmg, ctx, wl, stream, 64 if wl.get("dim", 2) == 2 else 32)
              if rank == 0 and not args.small else None)
    forms = {}
    shapes_ms = None
    mesh = None
    if rank == 0 and not args.small and wl.get("dim", 2) == 2 and not args.no_mesh_sweep:
        sw = mesh_sweep(irkmg, torch, wl, args, dev, stream, prec, fixed,
                        sizes=tuple(n for n in (32, 64, 128, 256) if n < wl["n"]))
        sw[wl["n"]] = {"iters": iters[-1], "levels": wl["levels"], "N": N,
                       "rel_residual": resid[-1], "status": stats[-1]["status"]}
        its = [v["iters"] for v in sw.values()]
        mesh = {"what": "FGMRES iterations to 1e-10 per finest mesh n x n, same solver, "
                        "tableau, dt and coarsest mesh (8 x 8)",
                "per_n": {str(n): v for n, v in sw.items()},
                "iters": its, "max_minus_min": max(its) - min(its)}
    if rank == 0 and fixed and not args.small:
        # after the timed region: one finest-level correction per launch shape
        shapes_ms = shape_sweep(irkmg, torch, ctx, dev, stream)
    if rank == 0 and not args.small and prec == 64 and not args.no_forms:
        for name, fp, pf, fx, ox in (("dense_fp64", 64, 0, 0, 0), ("dense_fp32", 32, 0, 0, 0),
                                     ("kron_fp64", 64, 1, 0, 0), ("kron_fp64_fixed", 64, 1, 1, 0),
                                     ("kron_fp64_fixed_op_fixed", 64, 1, 1, 1),
                                     ("kron_fp32", 32, 1, 0, 0)):
            if pf == args.patch_form and fp == prec and fx == fixed and ox == opfx:
                continue
            forms[name] = run_form(irkmg, torch, wl, args, dev, stream, k, fp, pf, fx, ox)
            forms[name]["speedup_vs_headline"] = (ms / args.steps) / forms[name]["ms_per_step"]
        forms["batched"] = run_batched(args, dev, stream)
        forms["ns_newton"] = run_ns(args, dev, stream)
        forms["adjoint"] = run_adjoint(args, dev, stream)
        forms["3d"] = run_3d(args, dev, stream, 1)
        forms["3d_dense"] = run_3d(args, dev, stream, 0)
        forms["3d"]["speedup_vs_dense"] = forms["3d_dense"]["ms_per_step"] / forms["3d"]["ms_per_step"]
    result = None
    if rank == 0:
        hbm, hbm_kind = peaks()
        alu = measure_alu_peaks(irkmg, stream)
        fp64_peak = alu["fp64_tflops"]
        van_gbs = trace["vanka_bytes"] / (trace["vanka_ms"] * 1e-3) / 1e9 if trace["vanka_ms"] else None
        op_gbs = trace["op_bytes"] / (trace["op_ms"] * 1e-3) / 1e9 if trace["op_ms"] else None
        op_tf = trace["op_flops"] / (trace["op_ms"] * 1e-3) / 1e12 if trace["op_ms"] else None
        xfer_gbs = (trace["xfer_bytes"] / (trace["xfer_ms"] * 1e-3) / 1e9
                    if trace["xfer_ms"] else None)
        arn_gbs = (trace["arnoldi_bytes"] / (trace["arnoldi_ms"] * 1e-3) / 1e9
                   if trace["arnoldi_ms"] else None)
        red_gbs = (trace["reduce_bytes"] / (trace["reduce_ms"] * 1e-3) / 1e9
                   if trace["reduce_ms"] else None)
        nvl = max(trace["vanka_launches"], 1)
        kname = {1: "k_vanka_apply_staged", 2: "k_vanka_apply",
                 3: "k_vanka_apply_lu", 4: "k_vanka_apply_kron",
                 5: "k_vanka_apply_kron_staged",
                 6: "k_vanka_apply_kron_big", 7: "k_vanka_apply_kron_ws",
                 8: "k_vanka_apply_kron_fx", 9: "k_vanka_apply_kron_fx_staged",
                 10: "k_vanka_apply_kron_fx_pair"}[ctx.finest["apply_kernel"]]
        if kname == "k_vanka_apply_kron" and prec == 32 and wl.get("dim", 2) == 2:
            # the warp kernel's FP32 complex-layout launch on 39-DoF patches
            # runs its paired-row form
            kname = "k_vanka_apply_kron_pair32"
        h = kernel_source_hash(kname)
        ratio = NCU_TRAFFIC.get((kname, h))
        traffic = ratio * trace["vanka_bytes"] / nvl if ratio is not None else None
        value = replica_value(ms, args.steps, world)
        van_tf = trace["vanka_flops"] / (trace["vanka_ms"] * 1e-3) / 1e12 if trace["vanka_ms"] else None
        common = {"kernel": kname + " (finest level)", "traffic": traffic,
                  "launches": trace["vanka_launches"], "bytes_per_launch": trace["vanka_bytes"] / nvl,
                  "flops_per_launch": trace["vanka_flops"] / nvl,
                  "avg_launch_ms": trace["vanka_ms"] / nvl, "kernel_src": h,
                  "hbm_gbs": van_gbs, "hbm_frac": van_gbs / hbm if van_gbs else None,
                  "hbm_peak_source": f"{hbm_kind} hbm_gbs"}
        if prec == 64 and not fixed:
            # FP64 on GB300 runs at 1/62 of FP32: a dense FP64 mat-vec (2 flop per
            # 8-byte entry) is bound by the FP64 pipe, not by HBM
            roofline = {"bound": "alu", "achieved": van_tf, "peak": fp64_peak,
                        "unit": "TFLOP/s", "frac": van_tf / fp64_peak if van_tf else None,
                        "peak_source": "FP64 FMA rate measured by irkmg_probe_peak", **common}
        else:
            roofline = {"bound": "hbm", "achieved": van_gbs, "peak": hbm, "unit": "GB/s",
                        "frac": van_gbs / hbm if van_gbs else None,
                        "peak_source": f"{hbm_kind} hbm_gbs", **common}
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == 64 else "f64+f32patch", "data": "synthetic",
            "dim": wl.get("dim", 2),
            "config": {**base_config(wl),
                       "patch_precision": prec, "patch_form": args.patch_form,
                       "patch_fixed": fixed,
                       "patch_arith": ("FP64 data; patch mat-vecs as exact integer dot products of "
                                       "57-bit fixed-point matrix rows and 58-bit fixed-point "
                                       "sources, rounded once to FP64" if fixed else
                                       "FP64 FMAs" if prec == 64 else "FP32 patch entries"),
                       "op_fixed": opfx,
                       "op_arith": ("FP64 data; stage operator as exact integer dot products of "
                                    "57-bit fixed-point rows and 58-bit fixed-point iterates, "
                                    "each sum rounded once to FP64, K x + B p added and the "
                                    "stage mixing applied in FP64" if opfx else "FP64 FMAs"),
                       "apply_kernel_per_level": [lv["apply_kernel"] for lv in ctx.levels[1:]],
                       "apply_shape_per_level": [lv["apply_shape"] for lv in ctx.levels[1:]],
                       "l2": "no flush: inputs larger than L2 (finest patch inverses %.1f GB)"
                             % (ctx.finest["factor_bytes"] / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "iters_per_solve": iters, "rel_residual": max(resid), "setup_s": setup_s,
            "roofline": roofline,
            "alu_peaks": alu,
            "roofline_spmv": ({"bound": "hbm",
                               "kernel": "k_block_absmax + k_op_convert + k_residual_fx "
                                         "(finest level, one application)",
                               "achieved": op_gbs, "peak": hbm, "unit": "GB/s",
                               "frac": op_gbs / hbm if op_gbs else None,
                               "peak_source": f"{hbm_kind} hbm_gbs",
                               "bytes": "operator rows, indices and vectors of the FP64 form "
                                        "(survey formula); the conversion passes are extra"}
                              if opfx else
                              {"bound": "alu", "kernel": "k_residual_sell (finest level)",
                               "achieved": op_tf, "peak": fp64_peak, "unit": "TFLOP/s",
                               "frac": op_tf / fp64_peak if op_tf else None,
                               "peak_source": "FP64 FMA rate measured by irkmg_probe_peak",
                               "hbm_gbs": op_gbs, "hbm_frac": op_gbs / hbm if op_gbs else None})
                              | {"launches": trace["op_launches"], "tflops": op_tf,
                                 "avg_launch_ms": trace["op_ms"] / max(trace["op_launches"], 1)},
            "roofline_transfers": {"bound": "hbm", "kernel": "k_transfer (finest level)",
                                   "achieved": xfer_gbs, "peak": hbm, "unit": "GB/s",
                                   "frac": xfer_gbs / hbm if xfer_gbs else None,
                                   "launches": trace["xfer_launches"],
                                   "bytes_per_launch": trace["xfer_bytes"] / max(trace["xfer_launches"], 1),
                                   "avg_launch_ms": trace["xfer_ms"] / max(trace["xfer_launches"], 1),
                                   "bytes": "vector bytes only (weights closed-form)"},
            "roofline_arnoldi": {"bound": "hbm",
                                 "kernel": "k_multidot_part + k_multiaxpy_dot + k_multidot_final "
                                           "(classical Gram-Schmidt twice, each update fused "
                                           "with the next reduction, finest level)",
                                 "achieved": arn_gbs, "peak": hbm, "unit": "GB/s",
                                 "frac": arn_gbs / hbm if arn_gbs else None,
                                 "steps": trace["arnoldi_steps"],
                                 "avg_step_ms": trace["arnoldi_ms"] / max(trace["arnoldi_steps"], 1),
                                 "bytes_per_step": trace["arnoldi_bytes"] / max(trace["arnoldi_steps"], 1)},
            "roofline_reduce": {"bound": "hbm",
                                "kernel": "k_vanka_reduce (per-DoF sum of the one-launch patch "
                                          "results with the Chebyshev update, finest level)",
                                "achieved": red_gbs, "peak": hbm, "unit": "GB/s",
                                "frac": red_gbs / hbm if red_gbs else None,
                                "launches": trace["reduce_launches"],
                                "bytes_per_launch": trace["reduce_bytes"] / max(trace["reduce_launches"], 1),
                                "avg_launch_ms": trace["reduce_ms"] / max(trace["reduce_launches"], 1),
                                "bytes": "s (8 Q + 16 m) + 4 Q + 4 m (results, contribution "
                                         "indices and pointers, direction read and written) "
                                         "+ the iterate read and written"},
            "roofline_factor": factor,
            "traced_step": "figures from one separate traced step after the timed region",
            "gpu_launches": launches,
            "finest_correction_ms_per_shape": shapes_ms,
            "mesh_independence": mesh,
            "forms": forms,
            "clocks": clk.summary(),
            "e2e": {"value": replica_value(e2e_s * 1e3, args.steps, world), "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        }
    ctx.close()
    return result


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--small", action="store_true", help="8x8 mesh (quick check)")
    ap.add_argument("--n", type=int, default=512, help="finest mesh n x n (8 * 2^k)")
    ap.add_argument("--dim", type=int, default=2, choices=[2, 3],
                    help="3: the 3D Kuhn-tetrahedra configuration as the headline")
    ap.add_argument("--n3", type=int, default=32, help="3D finest mesh n^3 cubes (4 * 2^k)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the FP32-patch and batched forms reported beside the headline")
    ap.add_argument("--batch", type=int, default=64, help="systems in the batched form")
    ap.add_argument("--only-batched", action="store_true",
                    help="run only the batched Oseen form (64 systems by default) and print it")
    ap.add_argument("--oracle-sizes", default="",
                    help="with --impl reference: comma-separated sample sizes, per-phase timings")
    ap.add_argument("--no-mesh-sweep", action="store_true",
                    help="skip the FGMRES iteration counts on the coarser meshes")
    ap.add_argument("--patch-fixed", type=int, default=1, choices=[0, 1],
                    help="decoupled FP64 patches: 1 = exact fixed-point mat-vecs "
                         "(irkmg_options.patch_fixed)")
    ap.add_argument("--patch-form", type=int, default=1, choices=[0, 1, 2, 3],
                    help="0 dense patch systems; 1..3 Kronecker-decoupled (irkmg_options.patch_form)")
    ap.add_argument("--op-fixed", type=int, default=0, choices=[0, 1],
                    help="2D: exact fixed-point stage operator (irkmg_options.op_fixed); "
                         "measured slower than the FP64 operator on GB300, so off by default")
    ap.add_argument("--apply", type=int, default=0, choices=[0, 1, 2],
                    help="Vanka apply kernel: 0 autotuned per level, 1 TMA-staged, 2 warp-per-patch")
    args = ap.parse_args()
    wl = workload(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, wl, rank)
        return
    if args.only_batched:
        import torch
        torch.cuda.set_device(local_rank)
        dev = torch.device("cuda", local_rank)
        print(json.dumps(run_batched(args, dev, torch.cuda.current_stream(dev))), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    res = run_ours(args, wl, rank, world, local_rank)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline and wl.get("dim", 2) == 2:
            sizes = (8,) if args.small else (32, 64)
            ob = oracle_baseline_subprocess(args, sizes)
            if ob is not None:
                big = ob["runs"][-1]
                res["cpu_baseline"] = {
                    "value": big["solve_s"], "unit": UNIT, "cores": ob["cores_available"],
                    "kind": "oracle",
                    "sample": f"oracle FGMRES + V-cycle solve of the same problem at "
                              f"{big['n']}x{big['n']} ({big['levels']} levels, N={big['N']}, "
                              f"{big['iters']} iterations), measured on {ob['cores_available']} "
                              f"host cores (BLAS threads {big['blas_threads']}, CPU time / wall "
                              f"{big['cpu_time_over_wall']:.2f}); value is that size's time",
                    "runs": ob["runs"], "fit_to_workload": ob["fit"]}
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
