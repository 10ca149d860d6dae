"""Benchmark: elastic Helmholtz solves per second to relative residual 1e-6.

One step = one complete FGMRES solve (block-acoustic multigrid
preconditioner) of the 512x512 layered workload (6 layers, Vp in [1.5, 4.5],
nu in [0.25, 0.45], rho = 0.31 Vp^0.25, 10 points per shear wavelength,
20-cell absorbing layer, one point source at the top centre), inputs resident
in HBM, setup excluded.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl bah|reference]
                  [--config c2|c3|c4|c5|c5s]

--config selects another workload: c3 (1024^2 random field), c4 (1024x512
layered, 64 sources in one batch) or c5 (128^3 random field, run with the
paper's 3-D cycle: W(2,2), mixed intergrid, Jacobi 0.8/0.8/0.2); c5s is a
64^3 copy of c5, a small case for profiling the 3-D kernels.

The main arm (bah) times the mixed-precision solve (bfloat16 coefficients,
FP32 multigrid, FP64 FGMRES / operator / coarsest solve) and, beside it, the
plain FP64 solve on the same GPU; the end-to-end figure is the same solve
through the C ABI with host buffers (copies inside the timed region).  The
reference arm (--impl reference) times the CPU oracle on the host cores.
Under torchrun every rank solves its own copy of the workload (independent
right-hand sides, weak scaling, no data-path collective).
"""
from __future__ import annotations

import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse  # noqa: E402
import json  # noqa: E402
import math  # noqa: E402
import statistics  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import tempfile  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "elastic solves/s to rel-res 1e-6 (mixed vs FP64); stencil+V-cycle HBM GB/s"
UNIT = "solves/s"
WORKLOADS = {
    "c1": "2D 64x64 homogeneous medium (rho=1, Vp=2, nu=0.25), 10 points per shear wavelength, 8-cell absorbing "
          "layer, centre point source, FGMRES(20) to rel-res 1e-6",
    "c2": "2D 512x512 layered medium (6 layers, Vp U[1.5,4.5], nu U[0.25,0.45], rho=0.31 Vp^0.25), "
          "10 points per shear wavelength, 20-cell absorbing layer, one top-centre point source, "
          "FGMRES to rel-res 1e-6",
    "c3": "2D 1024x1024 smooth random medium (log Vp Gaussian random field, correlation 32 cells, std 0.2, mean "
          "log 3; nu in [0.3,0.49]), 10 points per shear wavelength, 20-cell absorbing layer, top-centre source, "
          "FGMRES to rel-res 1e-6",
    "c4": "2D 1024x512 layered medium (6 layers, seed 5), 64 point sources along row 20 solved as one batch, "
          "FGMRES to rel-res 1e-6 per source",
    "c5": "3D 128x128x128 smooth random medium (log Vp Gaussian random field, correlation 16 cells, std 0.2, mean "
          "log 3; nu in [0.3,0.49]), 8 points per shear wavelength, 10-cell absorbing layer, top-face point source, "
          "FGMRES to rel-res 1e-6",
    "c5s": "3D 64x64x64 copy of the c5 medium (correlation 8 cells, 5-cell absorbing layer), 8 points per shear "
           "wavelength, top-face point source, FGMRES to rel-res 1e-6 (a small case of the 3-D kernels, for profiles)",
}
# per-workload cycle settings where they differ from the 2-D benchmark's: the 3-D
# workload runs the paper's 3-D multigrid (Sec. 4.5: mixed intergrid, W(2,2),
# Jacobi 0.8, 0.8, 0.2) on 5 levels (coarsest 8^3) with the FP64 Krylov basis
PRESETS = {
    "2d": dict(levels=0, alpha=0.8, cycle="V", nu="1,3", jacobi="0.8,0.8,0.3", intergrid="bilinear", krylov="fp64",
               restart=10),
    # the 1024^2 random field: FGMRES(20) (FGMRES(10) needs 3172 instead of 2571 iterations)
    "c3": dict(restart=20),
    # many sources: the library's own cycle, V(1,2) with the shift by level count (1.0 at 7 levels),
    # FGMRES(20) (FGMRES(10) doubles the iteration count)
    "c4": dict(alpha=-1.0, nu="1,2", restart=20),
    "c5": dict(levels=5, alpha=0.4, cycle="W", nu="2,2", jacobi="0.8,0.8,0.2", intergrid="mixed", krylov="fp64",
               restart=20),
    "c5s": dict(levels=4, alpha=0.4, cycle="W", nu="2,2", jacobi="0.8,0.8,0.2", intergrid="mixed", krylov="fp64",
                restart=20),
}
WORKLOAD = WORKLOADS["c2"]
L2_FLUSH_BYTES = 512 << 20
FP64_PEAK_TFLOPS = 152 * 2.07e9 * 4 / 1e12   # 2 DFMA/clk/SM at the 2070 MHz maximum clock (1.26 TFLOP/s)
KERNEL_NAMES = {0: "k_elastic_apply", 1: "k_distributor", 2: "k_u_rhs", 3: "k_jacobi", 4: "k_residual",
                5: "k_restrict", 6: "k_prolong_add", 7: "k_coarse_apply", 8: "k_dot_norm_partial",
                9: "k_axpy_norm", 10: "k_norm2_partial", 11: "k_update_x", 12: "small kernels",
                14: "k_cluster_mg"}
KERNEL_NAMES_3D = {0: "k_apply3", 1: "k_distrib3", 2: "k_urhs3", 3: "k_jacobi3", 4: "k_jacobi3 (residual)",
                   5: "k_restrict3", 6: "k_prolong3", 7: "k_coarse_apply", 8: "k_dot_norm_partial",
                   9: "k_axpy_norm", 10: "k_norm2_partial", 11: "k_update_x", 12: "small kernels"}
# FP64 flops per algorithmic byte of the FP64 classes (2 flops per real FMA):
#   dot/axpy: 8 flops per complex MAC on 16 streamed bytes; operator: ~84 flops per cell on ~200 bytes
FP64_FLOP_PER_BYTE = {"dot": 0.5, "axpy": 0.5, "update": 8.0 / 8.0, "operator": 84.0 / 200.0}
# DRAM bytes (read + write) per launch of a kernel class, averaged over the class's launches in one
# FGMRES step as they occur in the solve, from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of the same build and workload; the summaries under profiles/ give the
# command and the per-kernel figures.  (workload, class) -> bytes per launch.
TRAFFIC_PER_LAUNCH = {
    # 512x512 layered: k_jacobi (level 0) and k_stencil_staged sweeps (level 1), 161 launches over
    # 10 FGMRES steps of the launch list in profiles/launches_c2_512x512_mixed.md
    ("c2", "jacobi"): 7.289e6,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="bah", choices=["bah", "reference"])
    ap.add_argument("--config", default="c2")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-iters", type=int, default=8, help="oracle FGMRES iterations per baseline sample")
    ap.add_argument("--profile-json", default="", help="write the per-kernel-class profile here")
    ap.add_argument("--levels", type=int, default=None)
    ap.add_argument("--max-coarse", type=int, default=256)
    ap.add_argument("--restart", type=int, default=None)
    ap.add_argument("--krylov", default=None, choices=["fp64", "df"])
    ap.add_argument("--rhs-block", type=int, default=0,
                    help="right-hand sides per batch (default: all sources; -1: chosen by the autotuner)")
    ap.add_argument("--gradient", action="store_true", help="also time the adjoint gradient of a receiver misfit")
    ap.add_argument("--block-krylov", action="store_true",
                    help="solve each batch by block FGMRES (one Krylov space per batch; rhs_block 2..16)")
    ap.add_argument("--tune-cycle", action="store_true",
                    help="choose the cycle, shift and restart by timing complete solves first (autotune.tune_cycle)")
    ap.add_argument("--maxit", type=int, default=20000)
    # the benchmark's tuned cycle: V(1,3) with alpha 0.8 (searched at a resolution of 0.1 on this
    # workload, as the paper searches its shifts); --alpha -1 --nu 1,2 gives the library defaults
    ap.add_argument("--alpha", type=float, default=None, help="shift alpha (-1: the library's choice)")
    ap.add_argument("--cycle", default=None, choices=["V", "W"])
    ap.add_argument("--nu", default=None, help="pre- and post-smoothing sweeps")
    ap.add_argument("--jacobi", default=None, help="Jacobi damping per level, comma separated")
    ap.add_argument("--intergrid", default=None, choices=["bilinear", "mixed"])
    ap.add_argument("--krylov-df-steps", type=int, default=2,
                    help="also time the same solve with the Krylov basis in double-FP32 (48-bit) arithmetic")
    args = ap.parse_args()
    for k, v in {**PRESETS["2d"], **PRESETS.get(args.config, {})}.items():
        if getattr(args, k) is None:
            setattr(args, k, v)
    return args


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rhs_count(buf, vector_len):
    """Right-hand sides held by a torch tensor or numpy array: its entries over
    one padded vector's (a single 3-D vector has four array dimensions, so the
    array's rank tells nothing)."""
    total = int(buf.numel()) if hasattr(buf, "numel") else int(buf.size)
    if vector_len <= 0 or total % vector_len:
        raise ValueError(f"buffer of {total} entries is not a whole number of {vector_len}-entry vectors")
    return total // vector_len


def auto_levels(n, max_coarse):
    """The level count the library picks with levels = 0: halve every axis
    while the grid has more than max_coarse cells and every axis stays even
    and at least 2 after halving."""
    n = list(n)
    L = 1
    while int(np.prod(n)) > max_coarse and all(v % 2 == 0 and v // 2 >= 2 for v in n):
        n = [v // 2 for v in n]
        L += 1
    return L


def workload_config(args, prob, levels, alpha, world):
    """The ``config`` object of the JSON line: the workload and the solver
    settings that define the measured solve, identical in both arms."""
    nsrc_all = len(prob.sources)
    return {"workload": WORKLOADS.get(args.config, args.config), "grid": [int(v) for v in prob.n],
            "unknowns": int(sum(W.compact_sizes(prob.n))), "sources": nsrc_all, "levels": int(levels),
            "cycle": f"{args.cycle}({args.nu})", "alpha": round(float(alpha), 6), "jacobi": args.jacobi,
            "intergrid": args.intergrid, "restart": args.restart, "rtol": 1e-6,
            "l2": f"GPU arm: flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)",
            "parallelism": (f"sources split over {world} GPUs, no exchange during the solves" if nsrc_all > 1
                            else f"independent replicas of the solve on {world} GPUs")}


def oracle_counts():
    path = os.path.join(ROOT, "tests", "golden", "oracle_counts.json")
    if os.path.exists(path):
        return json.load(open(path))
    return {}


# ----------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ----------------------------------------------------------------------------
def oracle_sample(prob, levels, alpha, restart, iters, reps=1, nu=(1, 2), cycle="V", weights=(0.8, 0.8, 0.3),
                  intergrid="bilinear"):
    """Oracle setup once, then ``reps`` samples of ``iters`` FGMRES iterations;
    returns (seconds per iteration list, setup seconds)."""
    from oracle import elastic, fgmres, precond
    t0 = time.perf_counter()
    S = elastic.from_problem(prob)
    H = S.H
    pc = precond.multigrid(S, levels, alpha, precision="mixed", nu_pre=nu[0], nu_post=nu[1], cycle=cycle,
                           weights=weights, intergrid=intergrid)
    setup = time.perf_counter() - t0
    b = W.padded_to_compact(W.point_source(prob), prob.n)
    per = []
    for _ in range(reps):
        t1 = time.perf_counter()
        fgmres.fgmres(lambda v: H @ v, b, pc.apply, restart=restart, rtol=1e-30, maxit=iters)
        per.append((time.perf_counter() - t1) / iters)
    return per, setup


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    prob = W.config(args.config)
    counts = oracle_counts().get(args.config)
    from oracle import precond
    levels = args.levels if args.levels else auto_levels(prob.n, args.max_coarse)
    alpha = args.alpha if args.alpha >= 0 else precond.default_alpha(levels)
    nu = tuple(int(v) for v in args.nu.split(","))
    same = (bool(counts) and counts.get("levels") == levels and abs(counts.get("alpha", -1.0) - alpha) < 1e-12
            and tuple(counts.get("nu", (1, 2))) == nu and counts.get("restart", 20) == args.restart)
    its = counts["iters"] if same else None
    per, setup = oracle_sample(prob, levels, alpha, args.restart, args.cpu_iters, reps=args.warmup + args.steps,
                               nu=nu, cycle=args.cycle, weights=tuple(float(v) for v in args.jacobi.split(",")),
                               intergrid=args.intergrid)
    per = per[args.warmup:]
    t_iter = statistics.mean(per)
    if its is None:
        value = None
        note = "no stored oracle iteration count"
    else:
        value = 1.0 / (its * t_iter)
        note = f"extrapolated: {its} oracle iterations per solve (tests/golden/oracle_counts.json) x measured s/iteration"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_iter * args.cpu_iters * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(args, prob, levels, alpha, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.cpu_iters} FGMRES iterations per step after setup ({setup:.1f} s); {note}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# clocks sampler
# ----------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        for ln in open(self.f.name):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def run_bah(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    if rank == 0:
        from paper_2411_15897_gb300 import _build
        _build.build()
    barrier()
    import paper_2411_15897_gb300 as bah

    prob = W.config(args.config)
    from paper_2411_15897_gb300 import shard
    nsrc_all = len(prob.sources)
    # many sources: each rank solves its own share (no exchange during the
    # solves); one source: every rank solves it (replicas)
    if 1 < nsrc_all < world:
        raise SystemExit(f"{world} ranks for {nsrc_all} sources: every rank needs at least one source")
    mine = shard.shard(nsrc_all, rank, world) if nsrc_all > 1 else np.array([0])
    nsrc = len(mine)
    job_units = nsrc_all if nsrc_all > 1 else world      # solves completed by the whole job per step
    rhs_block = args.rhs_block if args.rhs_block > 0 else nsrc
    tuned = None
    opts = dict(precision=bah.BAH_MIXED, levels=args.levels, max_coarse_cells=args.max_coarse, restart=args.restart,
                krylov_arith=bah.BAH_KRYLOV_DF if args.krylov == "df" else bah.BAH_KRYLOV_FP64,
                rhs_block=rhs_block, maxit=args.maxit, shift_alpha=args.alpha,
                cycle=bah.BAH_CYCLE_W if args.cycle == "W" else bah.BAH_CYCLE_V,
                nu_pre=int(args.nu.split(",")[0]), nu_post=int(args.nu.split(",")[1]),
                jacobi_w=tuple(float(v) for v in args.jacobi.split(",")),
                intergrid=bah.BAH_INTERGRID_MIXED if args.intergrid == "mixed" else bah.BAH_INTERGRID_BILINEAR,
                block_krylov=1 if args.block_krylov else 0)
    tuned_cycle = None
    if args.tune_cycle:
        # cycle, sweeps, shift and restart by timing complete solves of a sample of the
        # sources (autotune.py), before the timed context; the search grid is smaller
        # for many-source workloads, whose solves are long
        from paper_2411_15897_gb300 import autotune
        cands = (autotune.cycle_candidates() if nsrc_all == 1 else
                 autotune.cycle_candidates(alphas=(0.8, 1.0), cycles=(("V", 1, 2), ("V", 1, 3)), restarts=(10, 20)))
        tuned_cycle = autotune.tune_cycle(prob, opts, candidates=cands, sample=4)
        st_ = tuned_cycle.settings
        opts.update(st_)
        args.cycle = "W" if st_["cycle"] == 1 else "V"
        args.nu = f"{st_['nu_pre']},{st_['nu_post']}"
        args.alpha = st_["shift_alpha"]
        args.restart = st_["restart"]
    if args.rhs_block < 0:
        # batch size and launch variant by timing short solves (autotune.py), before the timed context
        from paper_2411_15897_gb300 import autotune
        tuned = autotune.tune(prob, nsrc, {k: v for k, v in opts.items() if k not in ("rhs_block", "maxit")}, iters=10)
        os.environ.update(autotune.VARIANTS[tuned.variant])
        rhs_block = opts["rhs_block"] = tuned.rhs_block
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    t_setup = time.perf_counter()
    solver = bah.Solver.from_problem(prob, **opts)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    free1, _ = torch.cuda.mem_get_info()
    context_bytes = int(free0 - free1)
    levels = solver.levels
    b_host = np.ascontiguousarray(W.all_sources(prob)[mine]) if nsrc_all > 1 else W.point_source(prob)
    b = torch.from_numpy(b_host).cuda()
    if nsrc > 1 and args.fp64_steps > 0:
        args.fp64_steps = 0          # the all-FP64 comparison is run on the single-source workloads
    x = torch.zeros_like(b)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def solve_once(s, bb, xx):
        nr = rhs_count(bb, s.vector_len)
        st, stats = bah.bah_solve(s.ctx, bb, xx, nr, 1e-6)
        if nr == 1:
            return st, stats[0]
        agg = {"iters": max(q["iters"] for q in stats), "iters_mean": statistics.mean(q["iters"] for q in stats),
               "relres_true": max(q["relres_true"] for q in stats)}
        return st, agg

    # warm-up, with every kernel class timed once to find the dominant one
    bah.bah_profile_control(solver.ctx, (1 << 16) - 1, True)
    st0, stats0 = solve_once(solver, b, x)
    prof_all = bah.bah_profile_read(solver.ctx)
    for _ in range(max(0, args.warmup - 1)):
        solve_once(solver, b, x)
    classes = prof_all["classes"]
    dom = max((k for k in classes if k != "small"), key=lambda k: classes[k]["ms"])
    dom_id = bah.BAH_K_NAMES.index(dom)

    # timed region: K solves, no instrumentation; events per step on the launching
    # stream; L2 flushed between steps (outside the events)
    bah.bah_profile_control(solver.ctx, 0, True)
    clocks = Clocks(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    step_ms, iters = [], []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, stats = solve_once(solver, b, x)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        iters.append(stats["iters"])
        assert st == bah.BAH_OK, stats
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    prof_timed = bah.bah_profile_read(solver.ctx)
    total_s = sum(step_ms) / 1e3
    if world > 1:
        t = torch.tensor([total_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    value = args.steps * job_units / total_s

    # the dominant kernel class, timed launch by launch with CUDA events recorded
    # on the launching stream, over the same number of solves right after the
    # timed region (events inside the step graphs would slow the timed solves)
    bah.bah_profile_control(solver.ctx, 1 << dom_id, True)
    for _ in range(args.steps):
        flush.zero_()
        solve_once(solver, b, x)
    prof = bah.bah_profile_read(solver.ctx)
    bah.bah_profile_control(solver.ctx, 0, True)
    dc = prof["classes"][dom]
    calls = max(dc["calls"], 1)
    dom_ms = dc["ms"] / calls
    dom_bytes = dc["bytes"] / calls

    # relative residual of the last solve, by the library's FP64 residual
    relres = stats["relres_true"]

    # FP64 mode on the same GPU
    fp64 = None
    if args.fp64_steps > 0:
        s64 = bah.Solver.from_problem(prob, **dict(opts, precision=bah.BAH_FP64))
        x64 = torch.zeros_like(b)
        solve_once(s64, b, x64)
        ms64, it64 = [], []
        for _ in range(args.fp64_steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st64, stt = solve_once(s64, b, x64)
            e1.record(stream)
            e1.synchronize()
            ms64.append(e0.elapsed_time(e1))
            it64.append(stt["iters"])
        fp64 = {"value": args.fp64_steps * job_units / (sum(ms64) / 1e3), "unit": UNIT, "iters": it64[-1],
                "ms_per_step": statistics.mean(ms64), "relres_true": stt["relres_true"]}
        s64.close()

    # the same mixed solve with the Krylov basis in double-FP32 (48-bit) instead of IEEE FP64
    kdf = None
    if args.krylov == "fp64" and args.krylov_df_steps > 0 and prob.dim == 2:
        sk = bah.Solver.from_problem(prob, **dict(opts, krylov_arith=bah.BAH_KRYLOV_DF))
        xk = torch.zeros_like(b)
        solve_once(sk, b, xk)
        msk = []
        for _ in range(args.krylov_df_steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stk, sttk = solve_once(sk, b, xk)
            e1.record(stream)
            e1.synchronize()
            msk.append(e0.elapsed_time(e1))
        kdf = {"value": args.krylov_df_steps * job_units / (sum(msk) / 1e3), "unit": UNIT, "iters": sttk["iters"],
               "ms_per_step": statistics.mean(msk), "relres_true": sttk["relres_true"],
               "dtype": "as the headline, but the Krylov basis and Gram-Schmidt in double-f32 (48-bit significand)"}
        sk.close()

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if args.e2e_steps > 0:
        bp = torch.from_numpy(b_host.copy()).pin_memory()
        xp = torch.zeros_like(bp).pin_memory()
        bnp, xnp = bp.numpy(), xp.numpy()
        solve_once(solver, bnp, xnp)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            solve_once(solver, bnp, xnp)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        barrier()
        if world > 1:
            t = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e = {"value": args.e2e_steps * job_units / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(b_host.nbytes), "d2h_bytes_per_step": int(b_host.nbytes),
               "timing": "host wall clock around the C-ABI call with pinned host buffers (copies inside)"}

    # adjoint gradient of a receiver misfit (forward solve, adjoint solve, gradient kernel)
    grad = None
    if args.gradient:
        from paper_2411_15897_gb300 import misfit as MF
        rec = torch.from_numpy(MF.receiver_indices(prob.n, prob.sources[0][1])).cuda()
        # observed data: the true medium's wavefield at the receivers; the misfit is
        # evaluated at a smoothed medium (Gaussian filter of 8 cells)
        st_true = bah.Solver.from_problem(prob, **opts)
        xt = torch.zeros_like(b)
        bah.bah_solve(st_true.ctx, b, xt, nsrc, 1e-6)
        dobs = xt.reshape(nsrc, -1)[:, rec.long()].contiguous()
        st_true.close()
        from scipy.ndimage import gaussian_filter
        sm = lambda a: torch.tensor(gaussian_filter(a, 8.0, mode="nearest"), dtype=torch.float64, requires_grad=True)
        lam_t, mu_t, rho_t = sm(prob.lam), sm(prob.mu), sm(prob.rho)
        # the context setup for the smoothed medium, timed on its own (the misfit's
        # forward pass builds the same context again before its batched solve)
        torch.cuda.synchronize()
        ts0 = time.perf_counter()
        s_sm = bah.Solver(prob.n, prob.h, lam_t.detach().numpy(), mu_t.detach().numpy(), rho_t.detach().numpy(),
                          prob.gamma, prob.omega, **opts)
        torch.cuda.synchronize()
        grad_setup_s = time.perf_counter() - ts0
        s_sm.close()
        t0 = time.perf_counter()
        J = MF.misfit(lam_t, mu_t, rho_t, prob.gamma, prob.omega, prob.n, prob.h, b, dobs, rec, opts, 1e-6)
        t1 = time.perf_counter()
        J.backward()
        # the job's gradient: the sum over ranks of each rank's sources (one collective)
        gsum = [lam_t.grad.cuda(), mu_t.grad.cuda(), rho_t.grad.cuda(), J.detach().reshape(1).cuda()]
        shard.sum_over_ranks(*gsum)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        grad = {"misfit": float(gsum[3].item()), "forward_s": t1 - t0, "setup_s": grad_setup_s,
                "forward_solve_s": (t1 - t0) - grad_setup_s, "backward_s": t2 - t1,
                "grad_norms": [float(v.norm()) for v in gsum[:3]],
                "sources": nsrc_all, "sources_per_rank": nsrc, "receivers": int(rec.numel()),
                "note": "forward = context setup for the smoothed medium (setup_s, timed separately) + the batched "
                        "solve and misfit (forward_solve_s); backward = the batched adjoint solve and the gradient "
                        "kernel"}

    # roofline of the dominant kernel class
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    achieved_gbs = dom_bytes / (dom_ms * 1e-3) / 1e9 if dom_ms > 0 else None
    kname = (KERNEL_NAMES_3D if prob.dim == 3 else KERNEL_NAMES).get(dom_id, dom)
    roof = {"kernel": kname, "bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak,
            "unit": "GB/s", "frac": (achieved_gbs / hbm_peak) if achieved_gbs else None,
            "traffic": TRAFFIC_PER_LAUNCH.get((args.config, dom)),
            "peak_source": peak_src, "avg_launch_us": dom_ms * 1e3, "algorithmic_bytes_per_launch": dom_bytes,
            "launches_timed": dc["calls"],
            "timing": f"CUDA events on the launching stream around every launch of the class, {args.steps} solves "
                      "right after the timed region"}
    if dom in FP64_FLOP_PER_BYTE and achieved_gbs:
        tfl = achieved_gbs * FP64_FLOP_PER_BYTE[dom] / 1e3
        if tfl / FP64_PEAK_TFLOPS > roof["frac"]:
            roof.update({"bound": "alu", "achieved": tfl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": tfl / FP64_PEAK_TFLOPS, "peak_source": "derived: FP64 2 FMA/clk/SM x 152 SMs x 2070 MHz",
                         "hbm_gbs": achieved_gbs})
    wc = prof_all["classes"]
    tot_ms = sum(v["ms"] for v in wc.values()) or 1.0
    shares = {k: round(v["ms"] / tot_ms, 4) for k, v in sorted(wc.items(), key=lambda kv: -kv[1]["ms"])[:6]}
    # every class in the warm-up solve: launches and device time per FGMRES step, and the
    # achieved algorithmic bandwidth as a fraction of the measured HBM peak
    nsteps = max(1, stats0["iters"] if isinstance(stats0, dict) else 1)
    classes = {k: {"launches_per_step": round(v["launches"] / nsteps, 2),
                   "us_per_step": round(1e3 * v["ms"] / nsteps, 2),
                   "us_per_launch": round(1e3 * v["ms"] / max(v["launches"], 1), 2),
                   "gbs": round(v["bytes"] / (v["ms"] * 1e6), 1) if v["ms"] > 0 else None,
                   "frac_hbm": round(v["bytes"] / (v["ms"] * 1e6) / peaks.get("hbm_gbs", 6800.0), 4) if v["ms"] > 0 else None}
               for k, v in sorted(wc.items(), key=lambda kv: -kv[1]["ms"]) if v["launches"] > 0}
    prof_path = args.profile_json
    if rank == 0 and prof_path:
        json.dump({"warmup_all_classes": prof_all, "dominant_instrumented": prof, "timed": prof_timed,
                   "dominant": dom}, open(prof_path, "w"), indent=1)

    # CPU oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        counts = oracle_counts().get(args.config)
        alpha = solver.alpha
        nu = (int(args.nu.split(",")[0]), int(args.nu.split(",")[1]))
        per, setup = oracle_sample(prob, levels, alpha, args.restart, args.cpu_iters, reps=1, nu=nu, cycle=args.cycle,
                                   weights=tuple(float(v) for v in args.jacobi.split(",")), intergrid=args.intergrid)
        same = (bool(counts) and counts.get("levels") == levels and abs(counts.get("alpha", -1.0) - alpha) < 1e-12
                and tuple(counts.get("nu", (1, 2))) == nu and counts.get("restart", 20) == args.restart)
        its = counts["iters"] if same else statistics.median(iters)
        src = "oracle's own count" if same else "the GPU run's count"
        cpu = {"value": 1.0 / (its * per[0]), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{args.cpu_iters} oracle FGMRES iterations of the same workload after a {setup:.1f} s setup, "
                         f"extrapolated to {its} iterations per solve ({src})"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(step_ms), "setup_s": setup_s, "higher_is_better": True, "scaling": "strong" if nsrc_all > 1 else "weak", "vs_baseline": None,
        "dtype": (("mixed: bf16 stencils, f32 multigrid, " if prob.dim == 3 else "mixed: bf16 coefficients, f32 multigrid, ")
                  + "f64 coarsest solve (f64 inverse applied in f64), "
                  + ("double-f32 (48-bit) Krylov basis and Gram-Schmidt" if args.krylov == "df"
                     else "f64 Krylov basis and Gram-Schmidt")
                  + (", operator w = H z on the f32 flexible basis in double-f32 arithmetic" if prob.dim == 2 else
                     ", f64 operator")
                  + ", f64 Hessenberg / Givens / true residual / solution"),
        "data": "synthetic",
        "config": workload_config(args, prob, levels, solver.alpha, world),
        "run": {"sources_per_rank": nsrc, "rhs_block": rhs_block, "autotune": tuned.as_dict() if tuned else None,
                "autotune_cycle": tuned_cycle.as_dict() if tuned_cycle else None,
                "context_bytes": context_bytes, "cluster_levels_from": solver.info["cluster_level"],
                "iters": iters[-1], "relres_true": relres},
        "fp64": fp64,
        "krylov_df": kdf,
        "mixed_over_fp64": (value / fp64["value"]) if fp64 else None,
        "e2e": e2e,
        "gpu_launches": prof_timed["launches"],
        "kernel_shares": shares,
        "classes_warmup_instrumented": classes,
        "roofline": roof,
        "clocks": clk,
        "cpu_baseline": cpu,
        "gradient": grad,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_bah(args)


if __name__ == "__main__":
    main()
