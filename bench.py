#!/usr/bin/env python
"""Bidomain time steps per second at PCG relative residual 1e-8.

Workload (one GPU): the 2D torso slice at 2049 x 2049 nodes (N = 4 198 401,
N_H = 792 653), dt = 0.1 ms, seeded stimulus disc inside the elliptic heart,
Mitchell-Schaeffer reaction term.  A step is one pass of the resolution
algorithm: fused Step 1 + Step 3 kernel, PCG on Lambda with the block-LU /
monodomain preconditioner (hierarchical Cholesky factors), normalisation.

The chosen form (eps-truncated factors stored in reduced precision) is the
headline; the plain form (exact FP64 factors) is timed on the same GPU.  The
factor and matrix working set (GBs) is far larger than the 129 MB L2, so no
flush is needed between steps.

--impl reference times the FP64 CPU oracle on the host cores instead, on a
bounded sample of the same workload (see cpu_baseline).

--workload slab3d times the 3D slab precision form instead (161 x 161 x 49
nodes with --n 161; --eps / --precision choose the reduced form, the plain
form is FP64 exact factors).

--workload learned times the learned initial guess (config of the learned
form): online training on plain steps, then held-out steps with and without
the guess.

--workload batched times the batched form instead: 64 seeded torso slices
(sides 129 ... 1025 nodes, seed 2026) advanced together, one graph launch of
the PCG loop per step for all slices, leaf sizes from the tuner; its line
also gives the same slices stepped one at a time for comparison.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "bidomain steps/s at PCG rel-res 1e-8 (chosen form); HBM GB/s of the factor solve"

# DRAM bytes per algorithmic byte of one P_1 solve, from an ncu capture of the
# same kernels on the 1025^2 slice (610.8 MB of DRAM traffic for 464.1 MB of
# algorithmic bytes at eps 1e-3, FP32, leaf 32); the traffic grows with the
# factor, so the bench's roofline reports this ratio times its own algorithmic
# bytes for the same form (other forms: null, no capture of the current kernels).
TRAFFIC_PER_ALG_BYTE = {(1e-3, "fp32", 32): 610.8 / 464.06}


def parse():
    a = argparse.ArgumentParser()
    a.add_argument("--gpus", type=int, default=1)
    a.add_argument("--steps", type=int, default=20)
    a.add_argument("--warmup", type=int, default=3)
    a.add_argument("--impl", default="ours", choices=["ours", "reference"])
    a.add_argument("--n", type=int, default=2049)
    a.add_argument("--eps", type=float, default=1e-3)
    a.add_argument("--precision", default="fp32")
    a.add_argument("--leaf", type=int, default=32)
    a.add_argument("--scheme", default="euler", choices=["euler", "cn", "strang"],
                   help="time scheme of the slice and slab workloads")
    a.add_argument("--elliptic", default="hchol", choices=["hchol", "mg"],
                   help="P_1 / P_K by hierarchical Cholesky factors or multigrid V-cycles "
                        "(mg: --precision fp64 or fp32 storage, --eps not used)")
    a.add_argument("--tol", type=float, default=1e-8)
    a.add_argument("--cpu-seconds", type=float, default=20.0)
    a.add_argument("--no-plain", action="store_true")
    a.add_argument("--gpu-build", type=int, default=1,
                   help="1: factor the large fronts on the GPU (bid_precond_opts.gpu_build); 0: host")
    a.add_argument("--no-mg", action="store_true",
                   help="skip the multigrid comparison (P_1, P_K by FP32 multigrid V-cycles)")
    a.add_argument("--no-cpu", action="store_true")
    a.add_argument("--no-cpu-full", action="store_true",
                   help="skip the whole-step oracle timings at 65^2 and 513^2")
    a.add_argument("--workload", default="slice", choices=["slice", "batched", "slab3d", "learned"])
    a.add_argument("--train-runs", type=int, default=3)
    a.add_argument("--train-steps", type=int, default=60)
    a.add_argument("--eval-runs", type=int, default=2)
    a.add_argument("--guess-dv", type=int, default=1)
    a.add_argument("--guess-policy", type=int, default=1)
    a.add_argument("--slices", type=int, default=64)
    a.add_argument("--seeds", default="",
                   help="slice workload: comma-separated stimulus seeds; the chosen form is also "
                        "timed from the resting state once per seed (mean/min/max in the line)")
    a.add_argument("--no-sequential", action="store_true")
    return a.parse_args()


def workload(n, seed, kind="slice"):
    """kind "slice": the n x n torso slice, dt 0.1 ms, seeded stimulus disc;
    kind "slab3d": the 1 x 1 x 0.3 cm slab at n x n x nz nodes, nz - 1 the
    z cells at about the x spacing (65 -> 65 x 65 x 21, 161 -> 161 x 161 x 49),
    dt 0.05 ms, centre-ball stimulus."""
    from workloads import (torso_square_2d, params_2d, stimulus_seeded_disc, slab_3d, params_3d,
                           stimulus_centre_ball)
    if kind == "slab3d":
        mesh = slab_3d(n, n, slab_nz(n))
        return mesh, params_3d(0.05), stimulus_centre_ball(mesh)
    mesh = torso_square_2d(n)
    p = params_2d(0.1)
    stim = stimulus_seeded_disc(mesh, seed=seed)
    return mesh, p, stim


def slab_nz(n):
    return (3 * (n - 1) + 9) // 10 + 1


def workload_name(args, N=None, NH=None):
    sizes = "" if N is None else f" (N={N}, N_H={NH})"
    if args.workload == "slab3d":
        n = args.n
        return (f"3D orthotropic slab {n}x{n}x{slab_nz(n)}{sizes}, fibres -60..+60 deg through "
                "the depth, isolated heart, dt 0.05 ms, centre-ball stimulus, PCG rel-res 1e-8")
    scheme = {"euler": "", "cn": ", Crank-Nicolson scheme",
              "strang": ", Strang splitting"}[getattr(args, "scheme", "euler")]
    return (f"2D torso slice {args.n}^2{sizes}, dt 0.1 ms, seeded stimulus disc{scheme}, "
            "PCG rel-res 1e-8")


class Clocks:
    """nvidia-smi sampler during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if len(r) > 5 + i and r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def cpu_baseline(n, budget_s, seed=0, kind="slice"):
    """The oracle as it stands, timed on the host cores, on a bounded sample of
    the same workload.  A whole oracle step does not fit the budget at the
    large sizes (its sparse direct solve takes minutes at 2049^2, its plain CG
    thousands of iterations), so the sample is: Step 1 and Step 3 of the first
    step, then K iterations of the oracle's plain projected CG on its Step 2,
    K sized from a short calibration run to fill the budget.  Steps/s is
    1 / (t_rhs + t_iter * K_1e-8), K_1e-8 = K log(1e-8) / log(relres_K) the
    iterations to reach the timing tolerance at the measured (linear) rate."""
    import math
    from oracle import bidomain as ob
    mesh, p, stim = workload(n, seed, kind)
    s = ob.build_system(mesh, p)
    ist = ob.heart_stimulus(s, stim)
    U, V, h = ob.initial_state(s)
    dt = p["dt"]
    g = ob.gamma_of(p, dt)
    t0 = time.perf_counter()
    Y = ob.rhs(s, V, h, ist, 0.0, dt)
    ob.gate_update(s, V, h, dt)
    t_rhs = time.perf_counter() - t0
    X0 = np.concatenate([U, V])
    t0 = time.perf_counter()
    ob.solve_cg(s, g, Y, X0, tol=1e-30, max_iter=5)
    t_cal = (time.perf_counter() - t0) / 5
    K = int(max(10, min(20000, budget_s / max(t_cal, 1e-6))))
    t0 = time.perf_counter()
    X, it = ob.solve_cg(s, g, Y, X0, tol=1e-8, max_iter=K)
    t_iter = (time.perf_counter() - t0) / max(it, 1)
    L = ob.system_matrix(s, g)
    rel = float(np.linalg.norm(L @ X - Y) / np.linalg.norm(Y))
    cores = len(os.sched_getaffinity(0))
    if it < K:      # converged inside the budget: a whole step, measured
        step_s = t_rhs + t_iter * it
        how = (f"the whole first step, measured: Step 1+3 ({t_rhs:.2f} s) and {it} iterations "
               f"of the oracle's plain projected CG to rel-res 1e-8 ({t_iter * 1e3:.2f} ms each)")
    else:
        k_need = it * math.log(1e-8) / math.log(rel) if 0 < rel < 1 else float("nan")
        step_s = t_rhs + t_iter * k_need
        how = (f"first step of the workload: Step 1+3 ({t_rhs:.2f} s) and {it} iterations of the "
               f"oracle's plain projected CG ({t_iter * 1e3:.1f} ms each, relres {rel:.2e}); "
               f"{k_need:.0f} iterations to 1e-8 extrapolated at the measured rate (optimistic: "
               "CG slows in its tail, see measured_full_steps for whole steps)")
    return {"value": 1.0 / step_s, "unit": "steps/s", "cores": cores, "kind": "oracle",
            "sample": how + f"; numpy/scipy threads on {cores} cores (its sparse products run on one)"}


_ORACLE_RUN = r"""
import json, sys, time
import numpy as np
sys.path.insert(0, sys.argv[1])
from oracle import bidomain as ob
from workloads import torso_square_2d, params_2d, stimulus_left_apex, stimulus_seeded_disc
n, steps, dt, solver = int(sys.argv[2]), int(sys.argv[3]), float(sys.argv[4]), sys.argv[5]
mesh, p = torso_square_2d(n), params_2d(dt)
s = ob.build_system(mesh, p)
stim = stimulus_left_apex(mesh) if n == 65 else stimulus_seeded_disc(mesh, seed=0)
ist = ob.heart_stimulus(s, stim)
U, V, h = ob.initial_state(s)
t0 = time.perf_counter()
for k in range(steps):
    U, V, h = ob.time_step(s, U, V, h, ist, k * dt, dt, solver=solver, tol=1e-8)
el = time.perf_counter() - t0
print(json.dumps({"seconds": el, "steps": steps}))
"""


def oracle_full_steps(n, steps, dt, solver, threads):
    """Whole oracle time steps (Step 1, Step 2 by `solver` to rel-res 1e-8 where
    it iterates, Step 3), timed in a child process whose numerical libraries use
    `threads` threads.  Returns steps/s and the seconds taken."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = str(threads)
    out = subprocess.run([sys.executable, "-c", _ORACLE_RUN, ROOT, str(n), str(steps), str(dt), solver],
                         env=env, capture_output=True, text=True, timeout=900, check=True)
    r = json.loads(out.stdout.strip().splitlines()[-1])
    return {"steps_per_s": r["steps"] / r["seconds"], "seconds": r["seconds"], "steps": r["steps"],
            "threads": threads}


def oracle_measured(cores):
    """Whole oracle steps, not extrapolated: the 65^2 slice of 20 steps of
    0.25 ms with the corner stimulus (plain CG and sparse direct Step 2, one
    thread and all cores), and one 0.1 ms step of the 513^2 slice (plain CG)."""
    return {
        "slice65_20steps_cg": [oracle_full_steps(65, 20, 0.25, "cg", t) for t in (1, cores)],
        "slice65_20steps_direct": [oracle_full_steps(65, 20, 0.25, "direct", t) for t in (1, cores)],
        "slice513_1step_cg": oracle_full_steps(513, 1, 0.1, "cg", cores),
    }


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cb = cpu_baseline(args.n, args.cpu_seconds, kind=args.workload)
    if args.workload == "slice" and not args.no_cpu_full:
        cb["measured_full_steps"] = oracle_measured(cb["cores"])
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 / cb["value"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args),
                       "solver": "oracle plain projected CG (bounded sample)"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def partition_slices(sizes, world):
    """Greedy size-balanced assignment of independent slices to ranks: largest
    first, each to the least-loaded rank (ties to the lowest rank).  Returns
    one sorted index list per rank."""
    load = [0] * world
    parts = [[] for _ in range(world)]
    for k in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(k)
        load[r] += sizes[k]
    return [sorted(p) for p in parts]


def max_over_ranks(ms, dist, device):
    """The slowest rank's time (every rank gets it); ms itself without a process group."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_batched(args):
    """The batched form: on N > 1 GPUs the slices are shared out by
    partition_slices (no collective on the data path; total work fixed)."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1711_08708_gb300 import bid
    from workloads import batched_slices, torso_square_2d, params_2d, stimulus_seeded_disc
    dev = torch.device("cuda", local)
    st = torch.cuda.current_stream()
    dt = 0.1
    p = params_2d(dt)
    specs_all = batched_slices(args.slices, 2026)
    mine = partition_slices([d["n"] ** 2 for d in specs_all], world)[rank]
    specs = [specs_all[k] for k in mine]
    meshes = [torso_square_2d(d["n"], semi_axes=d["semi_axes"], fibre_deg=d["fibre_deg"])
              for d in specs]
    systems = [bid.System(m, p) for m in meshes]
    t0 = time.perf_counter()
    leaf = bid.tune_batch_leaf(systems, dt, eps=args.eps, precision=args.precision,
                               candidates=(8, 16, 32), reps=5)
    tune_s = time.perf_counter() - t0
    B = bid.Batch(systems, dt, eps=args.eps, precision=args.precision, leaf=leaf)
    S = B.S
    n, nh = B.n, int(B.hoff[-1])
    X0 = np.zeros(n)
    h0 = np.ones(nh)
    ist = np.zeros(nh)
    for k, (m, d, sy) in enumerate(zip(meshes, specs, systems)):
        X0[B.off[k] + sy.N:B.off[k + 1]] = p["v_rest"]
        ist[B.hoff[k]:B.hoff[k + 1]] = stimulus_seeded_disc(m, seed=d["stim_seed"])[sy.perm[:sy.NH]]
    I = torch.tensor(ist, dtype=torch.float64, device=dev)

    def timed(step_fn, nsteps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0.record(st)
        out = [step_fn(k) for k in range(nsteps)]
        e1.record(st)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1), dist, dev), out

    X = torch.tensor(X0, dtype=torch.float64, device=dev)
    h = torch.tensor(h0, dtype=torch.float64, device=dev)
    tcur = [0.0]

    def bstep(_):
        its = B.step(X, h, I, tcur[0], 1, tol=args.tol)
        tcur[0] += dt
        return its[0]

    timed(bstep, args.warmup)
    l0 = bid.kernel_launches()
    with Clocks(local) as ck:
        ms, its = timed(bstep, args.steps)
    launches = bid.kernel_launches() - l0
    its = np.array(its)

    # roofline: the P_1 forest solve of all slices, timed alone
    b = torch.randn(n, dtype=torch.float64, device=dev)
    x = torch.zeros_like(b)
    for _ in range(3):
        B.apply_factor(1, b, x)
    reps = 10
    solve_ms, _ = timed(lambda k: B.apply_factor(1, b, x), reps)
    solve_ms /= reps
    pk = peaks()
    hbm = pk.get("hbm_gbs", 6780.7)
    Ntot = int(sum(sy.N for sy in systems))
    alg_bytes = B.stats["alg_bytes_p1"] + 8 * 4 * Ntot
    achieved = alg_bytes / (solve_ms * 1e-3) / 1e9

    # e2e: combined state from / to pinned host memory every step
    hX = torch.tensor(X0, dtype=torch.float64).pin_memory()
    hh = torch.tensor(h0, dtype=torch.float64).pin_memory()
    Xe = torch.empty_like(X)
    he = torch.empty_like(h)

    tcur[0] = 0.0      # the same steps as the device-timed run, from the initial state

    def estep(_):
        Xe.copy_(hX, non_blocking=True)
        he.copy_(hh, non_blocking=True)
        B.step(Xe, he, I, tcur[0], 1, tol=args.tol)
        hX.copy_(Xe, non_blocking=True)
        hh.copy_(he, non_blocking=True)
        tcur[0] += dt

    e2e_ms, _ = timed(estep, args.steps)
    io_bytes = 8 * (n + nh)

    seq = None
    if not args.no_sequential:
        # the same slices one at a time through the single-system path
        Ps = [bid.Precond(sy, dt, eps=args.eps, precision=args.precision, leaf=lf)
              for sy, lf in zip(systems, leaf)]
        Us = [torch.zeros(sy.N, dtype=torch.float64, device=dev) for sy in systems]
        Vs = [torch.full((sy.NH,), p["v_rest"], dtype=torch.float64, device=dev) for sy in systems]
        hs = [torch.ones(sy.NH, dtype=torch.float64, device=dev) for sy in systems]
        Is = [I[B.hoff[k]:B.hoff[k + 1]].contiguous() for k in range(S)]
        ts = [0.0]

        def sstep(_):
            for k in range(S):
                Ps[k].step(Us[k], Vs[k], hs[k], Is[k], ts[0], 1, tol=args.tol)
            ts[0] += dt

        timed(sstep, args.warmup)
        sms, _ = timed(sstep, args.steps)
        seq = {"steps_per_s": world * args.steps / (sms * 1e-3),
               "note": "the same slices and leaf sizes stepped one at a time (bid_step per slice)"}
        del Ps

    # every rank advances its share of the slices: one batch step of the whole
    # job per step, timed by the slowest rank
    value = args.steps / (ms * 1e-3)
    line = {
        "metric": "bidomain batch steps/s at PCG rel-res 1e-8 (batched form, every slice "
                  "advanced per step); HBM GB/s of the factor solve",
        "value": value, "unit": "batch steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {
            "workload": f"batched form: {len(specs_all)} torso slices, sides "
                        f"{min(d['n'] for d in specs_all)}..{max(d['n'] for d in specs_all)} "
                        f"(seed 2026), N total {Ntot}, N_H total {nh}, dt 0.1 ms, "
                        "seeded stimulus discs, PCG rel-res 1e-8 per slice",
            "form": {"eps": args.eps, "factor_precision": args.precision},
            "slice_steps_per_s": len(specs_all) * value,
            "slices_on_rank0": S,
            "mean_pcg_iters": float(its.mean()), "max_pcg_iters": int(its.max()),
            "leaf": {str(v): leaf.count(v) for v in sorted(set(leaf))},
            "tune_seconds": tune_s,
            "l2": "inputs larger than L2 (factors and matrices several GB)",
            "parallelism": f"slices shared by {world} GPUs" if world > 1 else "single GPU",
            "precond_stats": {k: B.stats[k] for k in (
                "factor_bytes", "alg_bytes_p1", "alg_bytes_pk", "levels1", "levelsk",
                "build_seconds")},
            "sequential": seq,
        },
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": None,
                     "kernel": "P_1 forest solve of all slices (k_permute, k_flat_fwd, k_mid_fwd, "
                               "k_wide_fwd, k_gram, k_up_fwd, k_bwd_prep, k_up_bwd, k_wide_bwd, "
                               "k_mid_bwd, k_flat_bwd over all levels)",
                     "ms": solve_ms, "algorithmic_bytes": alg_bytes,
                     "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if pk else "fallback"},
        "e2e": {"value": world / (e2e_ms / args.steps * 1e-3), "unit": "batch steps/s",
                "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes},
        "gpu_launches": launches,
        "clocks": ck.summary(),
    }
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_learned(args):
    """Learned initial guess on the 2049^2 slice (chosen form): the network is
    trained online on plain steps of training stimuli, then held-out stimuli
    are stepped with the learned guess and with the previous-step guess."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1711_08708_gb300 import bid
    from workloads import torso_square_2d, params_2d, stimulus_seeded_disc
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    st = torch.cuda.current_stream()
    n, dt = args.n, 0.1
    mesh, p = torso_square_2d(n), params_2d(dt)
    S = bid.System(mesh, p)
    P = bid.Precond(S, dt, eps=args.eps, precision=args.precision)
    crop, ncrops = 128, 16
    net = bid.Cnn(ncrops * crop * crop, seed=3)
    G = bid.Guess(S, net, n, n, max_batch_pixels=ncrops * crop * crop)

    def state(seed):
        U = torch.zeros(S.N, dtype=torch.float64, device=dev)
        V = torch.full((S.NH,), p["v_rest"], dtype=torch.float64, device=dev)
        h = torch.ones(S.NH, dtype=torch.float64, device=dev)
        I = torch.tensor(stimulus_seeded_disc(mesh, seed=seed)[S.perm[:S.NH]], dtype=torch.float64,
                         device=dev)
        return U, V, h, I

    t0 = time.perf_counter()
    train_steps = 0
    for seed in range(100, 100 + args.train_runs):
        U, V, h, I = state(seed)
        G.reset()
        G.push(U, V)
        for k in range(args.train_steps):
            P.step(U, V, h, I, k * dt, 1, tol=args.tol)
            G.push(U, V)
            if k >= 3:
                G.train(ncrops=ncrops, crop=crop, iters=8, lr=2e-3, seed=seed * 1000 + k)
            train_steps += 1
    train_s = time.perf_counter() - t0

    def run(seed, learned):
        U, V, h, I = state(seed)
        if learned:
            G.reset()
            G.push(U, V)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        l0 = bid.kernel_launches()
        with Clocks(local) as ck:
            e0.record(st)
            if learned:
                stats = G.step(P, U, V, h, I, 0.0, args.steps, tol=args.tol)
                its = stats[:, 0]
            else:
                stats = None
                its = P.step(U, V, h, I, 0.0, args.steps, tol=args.tol)
            e1.record(st)
            torch.cuda.synchronize()
        return e0.elapsed_time(e1), np.asarray(its, dtype=float), stats, \
            bid.kernel_launches() - l0, ck.summary()

    G.configure(use_dv=bool(args.guess_dv), policy=args.guess_policy)
    seeds = list(range(200, 200 + args.eval_runs))
    run(seeds[0], True)            # warm-up of both paths (graphs, buffers)
    run(seeds[0], False)
    res_l = [run(sd, True) for sd in seeds]
    res_p = [run(sd, False) for sd in seeds]
    ms_l = sum(r[0] for r in res_l)
    ms_p = sum(r[0] for r in res_p)
    nsteps = args.steps * len(seeds)
    stats = np.concatenate([r[2] for r in res_l])
    warm = stats[np.arange(len(stats)) % args.steps >= 3]
    ratio = warm[:, 2] / np.maximum(warm[:, 1], 1e-300) if args.guess_policy == 0 else np.array([np.nan])
    value = nsteps / (ms_l * 1e-3)
    line = {
        "metric": "bidomain steps/s at PCG rel-res 1e-8 with the learned initial guess (vs the "
                  "previous-step guess)",
        "value": value, "unit": "steps/s", "n_gpus": 1, "steps": nsteps, "warmup": args.steps,
        "ms_per_step": ms_l / nsteps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {
            "workload": f"learned form: 2D torso slice {n}^2 (N={S.N}, N_H={S.NH}), dt 0.1 ms; "
                        f"CNN 6->32->32->2, 3x3, BF16 inference; trained online on "
                        f"{args.train_runs} x {args.train_steps} plain steps (stimulus seeds 100..), "
                        f"evaluated on {len(seeds)} x {args.steps} held-out steps (seeds 200..)",
            "form": {"eps": args.eps, "factor_precision": args.precision},
            "guess": {"predicts_dV": bool(args.guess_dv),
                      "policy": ["smaller initial residual", "fewer iterations so far"][args.guess_policy]},
            "train_seconds": train_s, "train_steps": train_steps,
            "learned": {"steps_per_s": value, "mean_pcg_iters": float(np.mean(np.concatenate(
                [r[1] for r in res_l]))), "used_fraction": float(warm[:, 3].mean()),
                "median_initial_residual_ratio": (float(np.median(ratio)) if args.guess_policy == 0
                                                  else None)},
            "previous_step": {"steps_per_s": nsteps / (ms_p * 1e-3), "mean_pcg_iters": float(
                np.mean(np.concatenate([r[1] for r in res_p])))},
            "l2": "inputs larger than L2 (factor + matrices several GB)",
            "parallelism": "single GPU",
        },
        "gpu_launches": int(sum(r[3] for r in res_l)),
        "clocks": res_l[-1][4],
    }
    print(json.dumps(line))


def class_bytes(stats, N, NH, nnz1, nnzi):
    """Algorithmic bytes of one launch of each kernel class of bid_profile_classes
    (FP64 values, int32 columns, each matrix entry and vector entry moved once)."""
    n = N + NH
    return {
        "lambda": 12 * (nnz1 + nnzi) + 16 * N + 24 * NH,          # S_1, S_i; x read, q written, m_H
        "p1_solve": stats["alg_bytes_p1"] + 32 * N,              # factor twice; input, y, x vectors
        "p1_masked": stats["alg_bytes_p1_masked"] + 32 * N,
        "pk_solve": stats["alg_bytes_pk"] + 32 * NH,
        "si_chain": 24 * nnzi + 48 * NH + 24 * N,               # two S_i products, z_U -= P_1^-1 W
        "pcg_vectors": 96 * n,                                   # <r,z>, p update, x and r updates
        "residual": 12 * (nnz1 + nnzi) + 24 * N + 32 * NH + 16 * n,   # Y - Lambda x, projection
        "rhs_gate": 8 * N + 40 * NH,                             # Y_U = 0; V, h, m_H in, h, Y_V out
        "normalise": 32 * N,
    }


def step_bytes(cb, iters):
    """Algorithmic bytes of one time step with `iters` PCG iterations: per
    iteration a preconditioner application (two P_1 solves, one masked, a P_K
    solve, the S_i chain), a Lambda product and the vector kernels; per step the
    initial and the final residual, Step 1 + Step 3 and the normalisation."""
    it = (cb["p1_solve"] + cb["p1_masked"] + cb["pk_solve"] + cb["si_chain"] + cb["lambda"] +
          cb["pcg_vectors"])
    return iters * it + 2 * cb["residual"] + cb["rhs_gate"] + cb["normalise"]


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "learned":
        return run_learned(args)
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1711_08708_gb300 import bid

    dev = torch.device("cuda", local)
    mesh, p, stim = workload(args.n, seed=rank, kind=args.workload)
    S = bid.System(mesh, p)
    NH, N = S.NH, S.N
    ist_h = stim[S.perm[:NH]]

    def state():
        U = torch.zeros(N, dtype=torch.float64, device=dev)
        V = torch.full((NH,), p["v_rest"], dtype=torch.float64, device=dev)
        h = torch.ones(NH, dtype=torch.float64, device=dev)
        return U, V, h

    I = torch.tensor(ist_h, dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream()

    def time_form(P, I=I):
        """W warm-up steps from the initial state, then K timed steps; the state
        at the start of the timed region is kept for the end-to-end replay."""
        U, V, h = state()
        t = 0.0
        iters = []
        for _ in range(args.warmup):
            iters += list(P.step(U, V, h, I, t, 1, tol=args.tol))
            t += p["dt"]
        torch.cuda.synchronize()
        snap = (U.cpu(), V.cpu(), h.cpu(), t)
        if dist:
            dist.barrier()
        it0 = len(iters)
        l0 = bid.kernel_launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with Clocks(local) as ck:
            e0.record(st)
            for _ in range(args.steps):
                iters += list(P.step(U, V, h, I, t, 1, tol=args.tol))
                t += p["dt"]
            e1.record(st)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        launches = bid.kernel_launches() - l0
        if dist:
            tt = torch.tensor([ms], device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            ms = float(tt.item())
        return dict(ms=ms, iters=iters[it0:], launches=launches, clocks=ck.summary(), U=U, V=V, h=h,
                    snap=snap)

    # ---- chosen form
    if args.elliptic == "mg":
        args.eps = 0.0
    P = bid.Precond(S, p["dt"], eps=args.eps, precision=args.precision, leaf=args.leaf,
                    scheme=args.scheme, elliptic=args.elliptic, gpu_build=args.gpu_build)
    chosen_stats = dict(P.stats)
    chosen = time_form(P)

    # ---- e2e through the public API with host buffers: the same K steps from
    # the same state and time as the timed region, the state copied from and to
    # pinned host memory every step
    hU, hV, hh = (a.pin_memory() for a in chosen["snap"][:3])
    t = chosen["snap"][3]
    U0, V0, h0 = state()
    e2e_iters = []
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        U0.copy_(hU, non_blocking=True)
        V0.copy_(hV, non_blocking=True)
        h0.copy_(hh, non_blocking=True)
        e2e_iters += list(P.step(U0, V0, h0, I, t, 1, tol=args.tol))
        hU.copy_(U0, non_blocking=True)
        hV.copy_(V0, non_blocking=True)
        hh.copy_(h0, non_blocking=True)
        t += p["dt"]
    e1.record(st)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    io_bytes = 8 * (N + 2 * NH)
    Uc, Vc = chosen["U"].cpu().numpy(), chosen["V"].cpu().numpy()
    e2e_same = bool(np.array_equal(hU.numpy(), Uc) and np.array_equal(hV.numpy(), Vc))

    # ---- the same form from the resting state for each stimulus seed asked for
    sweep = None
    seeds = [int(x) for x in args.seeds.split(",") if x.strip()] if args.workload == "slice" else []
    if seeds:
        from workloads import stimulus_seeded_disc
        runs = []
        for sd in seeds:
            Is = torch.tensor(stimulus_seeded_disc(mesh, seed=sd)[S.perm[:NH]], dtype=torch.float64,
                              device=dev)
            r = time_form(P, Is)
            runs.append({"seed": sd, "steps_per_s": world * args.steps / (r["ms"] * 1e-3),
                         "mean_pcg_iters": float(np.mean(r["iters"])),
                         "max_pcg_iters": int(np.max(r["iters"]))})
            del r
        sps = [r["steps_per_s"] for r in runs]
        its = [r["mean_pcg_iters"] for r in runs]
        sweep = {"seeds": seeds, "runs": runs,
                 "steps_per_s": {"mean": float(np.mean(sps)), "min": float(np.min(sps)),
                                 "max": float(np.max(sps))},
                 "mean_pcg_iters": {"mean": float(np.mean(its)), "min": float(np.min(its)),
                                    "max": float(np.max(its))},
                 "note": f"the chosen form, {args.warmup} warm-up + {args.steps} timed steps from the "
                         "resting state per stimulus seed (the line's value is seed "
                         f"{rank})"}

    # ---- roofline of the dominant kernel family: the P_1 solve (forward and
    # backward passes over all tree levels), timed alone with CUDA events on the
    # stream it is launched on
    b = torch.randn(N, dtype=torch.float64, device=dev)
    x = torch.empty_like(b)
    for _ in range(3):
        P.apply_factor(1, b, x)
    reps = 10
    e0.record(st)
    for _ in range(reps):
        P.apply_factor(1, b, x)
    e1.record(st)
    torch.cuda.synchronize()
    solve_ms = e0.elapsed_time(e1) / reps
    pk = peaks()
    hbm = pk.get("hbm_gbs", 6780.7)
    # algorithmic bytes of one P_1 application: the factor read twice (stored
    # bytes_p1 already counts both passes) + input gather, y and x vectors
    alg_bytes = P.stats["alg_bytes_p1"] + 8 * 4 * N

    # ---- every kernel class of a step, each timed alone (library CUDA events on
    # this stream), and the whole step against its algorithmic bytes
    cls_ms = P.profile_classes(reps=10, stream=st.cuda_stream)
    cb = class_bytes(chosen_stats, N, NH, S.nnz_s1, S.nnz_si)
    mean_it = float(np.mean(chosen["iters"]))
    ms_step = chosen["ms"] / args.steps
    classes = {k: {"ms": cls_ms[k], "algorithmic_bytes": cb[k],
                   "achieved_gbs": cb[k] / (cls_ms[k] * 1e-3) / 1e9,
                   "frac": cb[k] / (cls_ms[k] * 1e-3) / 1e9 / hbm} for k in cb}
    sb = step_bytes(cb, mean_it)
    per_step_ms = {k: v * (mean_it if k in ("lambda", "p1_solve", "p1_masked", "pk_solve", "si_chain",
                                            "pcg_vectors") else 2 if k == "residual" else 1)
                   for k, v in cls_ms.items()}
    whole_step = {"algorithmic_bytes": sb, "ms": ms_step, "achieved_gbs": sb / (ms_step * 1e-3) / 1e9,
                  "frac": sb / (ms_step * 1e-3) / 1e9 / hbm,
                  "classes_ms_sum": sum(per_step_ms.values()),
                  "note": "bytes per step at the mean PCG iterations; classes_ms_sum adds the "
                          "classes' standalone times in the same proportions (the rest of the "
                          "step is launch gaps, host reads and the state copies of bid_step)"}
    del P
    torch.cuda.empty_cache()

    # ---- plain form on the same GPU, the same steps from the same state
    plain = None
    if not args.no_plain:
        Pp = bid.Precond(S, p["dt"], eps=0.0, precision="fp64", leaf=args.leaf, scheme=args.scheme,
                         gpu_build=args.gpu_build)
        plain = time_form(Pp)
        plain_stats = Pp.stats
        del Pp
        Up, Vp = plain["U"].cpu().numpy(), plain["V"].cpu().numpy()
        err_vs_plain = {"U": float(np.abs(Uc - Up).max() / np.abs(Up).max()),
                        "V": float(np.abs(Vc - Vp).max() / np.abs(Vp).max()),
                        "h": float(np.abs(chosen["h"].cpu().numpy() - plain["h"].cpu().numpy()).max()),
                        "note": f"after {args.warmup + args.steps} steps, max |chosen - plain| over "
                                "each block / max |plain| (h: absolute); both forms stop at rel-res "
                                f"{args.tol:g}, so this is the solve tolerance times the "
                                "conditioning, not the factor precision"}

    # ---- the multigrid alternative for P_1 and P_K on the same GPU, same steps
    mgres = None
    if not args.no_mg and args.elliptic == "hchol":
        Pm = bid.Precond(S, p["dt"], precision="fp32", scheme=args.scheme, elliptic="mg")
        mg_form = time_form(Pm)
        b = torch.randn(N, dtype=torch.float64, device=dev)
        x = torch.empty_like(b)
        for _ in range(3):
            Pm.apply_factor(1, b, x)
        e0.record(st)
        for _ in range(10):
            Pm.apply_factor(1, b, x)
        e1.record(st)
        torch.cuda.synchronize()
        vms = e0.elapsed_time(e1) / 10
        vb = Pm.stats["alg_bytes_p1"] + 16 * N      # V-cycle bytes plus the mean-sum pass
        Um, Vm = mg_form["U"].cpu().numpy(), mg_form["V"].cpu().numpy()
        mgres = {"steps_per_s": world * args.steps / (mg_form["ms"] * 1e-3),
                 "mean_pcg_iters": float(np.mean(mg_form["iters"])),
                 "build_seconds": Pm.stats["build_seconds"],
                 "levels": [Pm.stats["levels1"], Pm.stats["levelsk"]],
                 "dtype": "f64 PCG / fp32 multigrid V-cycles",
                 "p1_vcycle": {"ms": vms, "algorithmic_bytes": vb,
                               "achieved_gbs": vb / (vms * 1e-3) / 1e9,
                               "frac": vb / (vms * 1e-3) / 1e9 / hbm},
                 "error_vs_chosen": {"U": float(np.abs(Um - Uc).max() / np.abs(Uc).max()),
                                     "V": float(np.abs(Vm - Vc).max() / np.abs(Vc).max())},
                 "note": "the same block-LU preconditioner with P_1 and P_K applied by one "
                         "geometric-multigrid V-cycle each instead of the hierarchical factors"}
        del Pm

    value = world * args.steps / (chosen["ms"] * 1e-3)
    traffic_ratio = TRAFFIC_PER_ALG_BYTE.get((args.eps, args.precision, args.leaf))
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": (f"f64 PCG / {args.precision} multigrid V-cycles" if args.elliptic == "mg" else
                  f"f64 PCG / {args.precision} factors" + (f" (eps {args.eps:g})" if args.eps else "")),
        "data": "synthetic",
        "config": {
            "workload": workload_name(args, N, NH),
            "form": {"eps": args.eps, "factor_precision": args.precision, "leaf": args.leaf,
                     "scheme": args.scheme, "elliptic": args.elliptic, "gpu_build": args.gpu_build},
            "mean_pcg_iters": mean_it,
            "l2": "inputs larger than L2 (factor + matrices several GB)",
            "parallelism": f"replicas{world}" if world > 1 else "single GPU",
            "precond_stats": {k: chosen_stats[k] for k in (
                "factor_bytes", "bytes_p1", "bytes_pk", "alg_bytes_p1", "alg_bytes_p1_masked",
                "alg_bytes_pk", "levels1", "levelsk", "large_levels1", "large_levelsk",
                "masked_dead1", "masked_clusters1", "dense_entries", "lowrank_entries",
                "lowrank_blocks", "mid_clusters1", "mid_clustersk", "wide_clusters1", "wide_clustersk",
                "gram_pivots1", "gram_pivotsk", "build_seconds")},
            "plain": None if plain is None else {
                "steps_per_s": world * args.steps / (plain["ms"] * 1e-3),
                "mean_pcg_iters": float(np.mean(plain["iters"])),
                "factor_bytes": plain_stats["factor_bytes"],
                "build_seconds": plain_stats["build_seconds"],
                "dtype": "f64 PCG / fp64 factors (exact)",
            },
            "chosen_error_vs_plain": None if plain is None else err_vs_plain,
            "multigrid": mgres,
            "seed_sweep": sweep,
        },
        "roofline": {"bound": "hbm", "achieved": alg_bytes / (solve_ms * 1e-3) / 1e9, "peak": hbm,
                     "unit": "GB/s", "frac": alg_bytes / (solve_ms * 1e-3) / 1e9 / hbm,
                     "traffic": (traffic_ratio * alg_bytes if args.workload == "slice" and traffic_ratio
                                 else None),
                     "traffic_note": "ncu DRAM bytes of the same kernels on the 1025^2 slice, scaled "
                                     "by the algorithmic bytes",
                     "kernel": ("P_1 solve: k_permute, k_flat_fwd, k_mid_fwd, k_wide_fwd, k_gram, "
                                "k_up_fwd, k_bwd_prep, k_up_bwd, k_wide_bwd, k_mid_bwd, k_flat_bwd over "
                                "all tree levels" if args.elliptic == "hchol"
                                else "P_1 multigrid V-cycle: k_mg_first, k_mg_cheb, k_mg_resid, "
                                     "k_mg_apply over all levels, k_mg_dense"),
                     "ms": solve_ms, "algorithmic_bytes": alg_bytes,
                     "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if pk else "fallback",
                     "classes": classes, "whole_step": whole_step},
        "e2e": {"value": world / (e2e_ms * 1e-3), "unit": "steps/s", "h2d_bytes_per_step": io_bytes,
                "d2h_bytes_per_step": io_bytes, "mean_pcg_iters": float(np.mean(e2e_iters)),
                "same_steps_as_timed": e2e_same,
                "note": "the timed region's K steps replayed from its starting state and time, "
                        "U, V, h copied from and to pinned host memory every step"},
        "gpu_launches": chosen["launches"],
        "clocks": chosen["clocks"],
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args.n, args.cpu_seconds, kind=args.workload)
        if args.workload == "slice" and not args.no_cpu_full:
            line["cpu_baseline"]["measured_full_steps"] = oracle_measured(line["cpu_baseline"]["cores"])
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
