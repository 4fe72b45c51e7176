#!/usr/bin/env python3
"""Benchmark of the image-enhanced MFS resistance solve on one GB300 (or N replicas).

Workload (the gap sweep of Sec. 5.1 / Fig. sweep_im): two unit spheres at 18 gaps
log-spaced in [1e-3, 1], three relative motions each (squeezing, shearing, counter-rotation),
N = 800 proxy Stokeslets on R_p = 0.63, M0 = 1600 basic collocation nodes, images and caps by
the n_im rule (<= 20 per contact, <= 60 image sources), one-body truncation 5e-12, GMRES
tolerance 1e-6.  One step = the 54 resistance solves (steps 1-3 of the preconditioned apply
inside GMRES, the refinement residual with the double-float operator at this tolerance,
lambda = B^+ mu, forces and torques), all 54 in one lockstep batch
in which the three motions of a geometry share its factor reads; the 18 discretisations and
their one-body SVDs are built once before timing (reported as setup_s).

metric   Stokeslet pair-interactions/s: (target node, vector source) pairs evaluated by the
         pair kernel over the timed steps / device time (an S+R+D image triple counts 3).
e2e      the same through the host-buffer C-ABI calls (velocities in, forces/torques out).
--impl reference   the FP64 CPU oracle (tests' reference) on a bounded sample of the workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

N_PROXY, R_PROXY, M_BASIC = 800, 0.63, 1600
MOTIONS = ("squeeze", "shear", "rotate")
SWEEP_TOL = 1e-6          # GMRES tolerance of the timed solves (Sec. 3, Sec. 5)
SWEEP_RESTART = 300
GOLDEN = os.path.join(ROOT, "tests", "golden", "gap_sweep_oracle.json")
# Algorithmic work per pair (FMA = 2 flops, rsqrt = 1): 28 flops per Stokeslet pair and 63 per
# S+R+D image triple at one node (shared distance and 1/r).  This is what `frac` is measured in.
FLOPS_ALG = (28.0, 63.0)
# FP32-pipe operations the double-float (compensated) kernel issues for the same pair math,
# counted from its source: 248 per Stokeslet pair (204 instructions, 44 of them FMAs) and 544
# per image triple (436, 108 FMAs).  Their rate against the FP32 peak is `issue_frac`, a
# measure of how busy the pipes are, not of algorithmic throughput.
FLOPS_ISSUED_DW = (248.0, 544.0)
# dram__bytes_read.sum + dram__bytes_write.sum of one pairs_dw_multi_kernel<3> launch over three
# gap-sweep geometries with their three motions each (ncu --set full on
# `bench.py --profile-case gemv_rhs`; 0.94 MB read, 0 written): the kernel is FP32-issue-bound
# and its operands stay in L2 (the single-problem kernel: 5.05 MB for an 18-problem launch)
PAIR_DW_TRAFFIC_BYTES = 0.940e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 sweep and FP32 kernel side runs")
    ap.add_argument("--restart", type=int, default=SWEEP_RESTART, help="GMRES restart length of the timed solves")
    ap.add_argument("--tol", type=float, default=SWEEP_TOL, help="GMRES tolerance of the timed solves")
    ap.add_argument("--kernel-case", type=int, default=0,
                    help="profiling case: build the sweep, run this many batched GMRES iterations, exit")
    ap.add_argument("--profile-case", default="", choices=["", "far", "tensor", "gemv_rhs"],
                    help="profiling case: 'far' = pass-operator applies on a 343-sphere lattice with the far field, "
                         "'tensor' = the same on 60 contact-free spheres with the tensor-core step 1; then exit")
    ap.add_argument("--suspension", type=int, default=200,
                    help="spheres of the far-field suspension solve among the extras (0 = skip)")
    ap.add_argument("--cluster-example", type=int, default=0,
                    help="run only the fixed-cluster example (Sec. 4, Ex. 2) with this many spheres and the far "
                         "field, print its JSON and exit")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def workload_config(args):
    from paper_2407_03343_gb300 import workloads
    return {"workload": "gap sweep: 2 unit spheres x 18 gaps in [1e-3, 1] x 3 motions (54 resistance solves)",
            "n_proxy": N_PROXY, "r_proxy": R_PROXY, "m_basic": M_BASIC, "n_im": "rule, <= 20",
            "eps_trunc": 5e-12, "gmres_tol": args.tol, "gmres_restart": args.restart, "precision": args.precision,
            "gaps": [float(g) for g in workloads.gap_sweep_gaps()],
            "l2": "256 MB write between timed steps; resident factors ~5 GB exceed L2"}


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle baseline
def host_cores():
    """Threads numpy's BLAS may use: the environment's setting if any, else every host core."""
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(v, "").isdigit():
            return int(os.environ[v])
    return os.cpu_count() or 1


def oracle_sample(seconds_budget=20.0):
    """Step 2 of the oracle's preconditioned apply (off-diagonal target-from-source blocks built
    and applied, as the oracle does it) for the delta = 1e-3 problem of the sweep, numpy FP64
    with its BLAS on all host cores."""
    from oracle import geometry, solve
    from paper_2407_03343_gb300 import workloads
    delta = workloads.gap_sweep_gaps()[0]
    d = geometry.build(workloads.two_spheres(delta), 1.0,
                       geometry.Params(n_proxy=N_PROXY, r_proxy=R_PROXY, m_basic=M_BASIC))
    rng = np.random.default_rng(0)
    lam = [rng.normal(size=solve.n_unknowns(d, k)) for k in range(2)]
    pairs = 0
    for k in range(2):
        kp = 1 - k
        sp = d.spheres[kp]
        pairs += d.spheres[k].colloc.shape[0] * (sp.proxy.shape[0] + 3 * sp.image.shape[0])
    reps, t0 = 0, time.perf_counter()
    while True:
        for k in range(2):
            _ = solve.scaled_block(d, k, 1 - k) @ lam[1 - k]
        reps += 1
        el = time.perf_counter() - t0
        if el > seconds_budget or reps >= 50:
            break
    return {"value": pairs * reps / el, "unit": "pair-interactions/s", "cores": host_cores(), "kind": "oracle",
            "sample": f"oracle step-2 apply (off-diagonal blocks built in numpy FP64 and applied) of the "
                      f"delta=1e-3 two-sphere problem, {pairs} pairs per apply, {reps} applies in {el:.1f} s"}


def oracle_solve_sample():
    """One full oracle solve of a sweep problem (matrix-free GMRES on eq. resistance with the
    three-step apply, O3) at the benchmark's tolerance, timed on the host: the hardest problem of
    the sweep, squeezing at delta = 1e-3 (20 image points per sphere).  Set-up (the two one-body
    SVDs) timed separately."""
    from oracle import geometry, solve
    from paper_2407_03343_gb300 import workloads
    gap = workloads.gap_sweep_gaps()[0]
    t0 = time.perf_counter()
    d = geometry.build(workloads.two_spheres(gap), 1.0, geometry.Params(n_proxy=N_PROXY, r_proxy=R_PROXY,
                                                                        m_basic=M_BASIC))
    op = solve.Operator(d)
    t1 = time.perf_counter()
    v, w = workloads.motion("squeeze")
    sol = solve.solve_o3(d, v, w, op=op, tol=SWEEP_TOL)
    t2 = time.perf_counter()
    return {"problem": f"gap {gap:.4g}, squeeze", "setup_s": t1 - t0, "solve_s": t2 - t1, "iters": sol.iters,
            "cores": host_cores()}


def reduce_over_ranks(total_ms, pairs, device):
    """(max over ranks of the timed milliseconds, sum over ranks of the pairs); identity on one
    rank.  device: the tensor device of the process group's backend (CUDA for NCCL, None = CPU)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(total_ms), float(pairs)
    import torch
    tt = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    pt = torch.tensor([float(pairs)], dtype=torch.float64, device=device)
    dist.all_reduce(pt)
    return float(tt.item()), float(pt.item())


def suspension_kernel_rates(device, fp32_peak):
    """Device time of one pair-kernel launch per precision on the 200-sphere suspension
    (volume fraction 0.2, ~300 near contacts, N = 800, M0 = 1600; ~1e11 pairs per launch,
    4 target nodes per thread), discretised without the one-body factors."""
    from paper_2407_03343_gb300 import mfs, workloads
    ctx = mfs.Context(device)
    ctx.set_spheres(workloads.suspension(200, 0.2, seed=3))
    ctx.build(n_proxy=N_PROXY, r_proxy=R_PROXY, m_basic=M_BASIC, build_factors=0)
    s = ctx.sizes()
    lam = np.random.default_rng(0).normal(size=s.n_unknowns)
    mu = np.zeros(3 * s.n_colloc)
    ctx.set_profiling(True)
    out = {"pairs_per_launch": s.pairs_fp, "contacts": s.n_contacts, "nodes": s.n_colloc}
    for name, prec in (("fp32", mfs.FP32), ("double_float", mfs.MIXED), ("fp64", mfs.FP64)):
        fl = FLOPS_ALG
        ctx.apply_pairs(lam, mu, prec)   # warm-up
        ctx.timing(reset=True)
        reps = 3 if prec != mfs.FP64 else 1
        for _ in range(reps):
            ctx.apply_pairs(lam, mu, prec)
        t = ctx.timing(reset=True)
        sec = t.pair_ms / 1000.0 / t.pair_launches
        flops = (t.pair_proxy * fl[0] + t.pair_image_nodes * fl[1]) / t.pair_launches
        out[name] = {"ms_per_launch": 1000 * sec, "pairs_per_s": s.pairs_fp / sec, "tflops": flops / sec / 1e12,
                     "frac_of_fp32_peak": flops / sec / 1e12 / fp32_peak if prec != mfs.FP64 else None,
                     "frac_of_fp64_peak": flops / sec / 1e12 / 1.0 if prec == mfs.FP64 else None}
        if prec == mfs.MIXED:
            issued = (t.pair_proxy * FLOPS_ISSUED_DW[0] + t.pair_image_nodes * FLOPS_ISSUED_DW[1]) / t.pair_launches
            out[name]["issue_frac"] = issued / sec / 1e12 / fp32_peak
    ctx.close()
    return out


FAR = dict(far_dist=3.5, far_n_eq=300, far_r_eq=1.0, far_r_chk=2.0, far_eps=1e-6)


def suspension_solve(device, P=200, tol=SWEEP_TOL):
    """The random suspension (P unit spheres at volume fraction 0.2, near contacts at gaps
    log-uniform in [1e-3, 1e-1], N = 800, M0 = 1600, random rigid motions) solved in MIXED
    precision with the far field in the GMRES passes (spheres more than 3.5 radii apart through 300
    equivalent Stokeslets) and the exact double-float operator in the refinement residual.  The
    solve is timed with CUDA events on the context's stream; the operator applies of the passes,
    of the exact double-float operator and of the plain FP64 operator are timed per launch."""
    import torch
    from paper_2407_03343_gb300 import mfs, workloads
    st = torch.cuda.Stream()
    ctx = mfs.Context(device, stream=st.cuda_stream)
    centres = workloads.suspension(P, 0.2, seed=3)
    ctx.set_spheres(centres)
    t0 = time.perf_counter()
    ctx.build(n_proxy=N_PROXY, r_proxy=R_PROXY, m_basic=M_BASIC, **FAR)
    setup = time.perf_counter() - t0
    s = ctx.sizes()
    t0 = time.perf_counter()
    sh = ctx.tune_pairs()
    tune_s = time.perf_counter() - t0
    shapes = {f: getattr(sh, f) for f, _ in sh._fields_}
    v, w = workloads.rigid_velocities(P, seed=1)
    ctx.set_rigid_velocities(v, w)
    ctx.set_profiling(True)
    mu = ctx.rhs()
    applies = {}
    for name, prec, reps in (("pass_far_field", mfs.MIXED_PASS, 3), ("exact_double_float", mfs.MIXED, 2),
                             ("exact_fp64", mfs.FP64, 1)):
        ctx.apply_operator(mu, prec)
        ctx.timing(reset=True)
        for _ in range(reps):
            ctx.apply_operator(mu, prec)
        t = ctx.timing(reset=True)
        applies[name] = {"pair_ms": t.pair_ms / reps, "far_ms": t.far_ms / reps, "gemv_ms": t.gemv_ms / reps,
                         "near_pairs": t.pair_interactions / reps, "far_equivalent_pairs": t.far_pairs / reps}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    info = ctx.solve(precision="mixed", tol=tol, max_iter=4000, allow_not_converged=True)
    e1.record(st)
    e1.synchronize()
    t = ctx.timing(reset=True)
    F, T = ctx.forces_torques()
    solve_s = e0.elapsed_time(e1) / 1000.0
    out = {"spheres": P, "contacts": s.n_contacts, "nodes": s.n_colloc, "setup_s": setup,
           "pairs_exact_per_apply": s.pairs_fp, "pairs_near_per_apply": s.pairs_near_fp,
           "equivalent_pairs_per_apply": s.pairs_far_eq, "device_GB": ctx.memory_in_use() / 1e9,
           "tuned_shapes": shapes, "tune_s": tune_s, "applies_ms": applies, "solve_s": solve_s, "iters": info.iters, "refinements": info.refinements,
           "rel_residual_exact_operator": info.rel_residual, "converged": info.converged, "tol": tol,
           "near_pairs_per_s": t.pair_interactions / (t.pair_ms / 1000.0) if t.pair_ms else None,
           "equivalent_pairs_per_s": t.far_pairs / (t.far_ms / 1000.0) if t.far_ms else None,
           "near_ms": t.pair_ms, "far_ms": t.far_ms, "gemv_ms": t.gemv_ms,
           "ft_finite": bool(np.all(np.isfinite(F)) and np.all(np.isfinite(T))),
           "timing": "solve: CUDA events on the context stream, one solve; applies: per-launch CUDA events"}
    ctx.close()
    return out


def cluster_example(device, P=100, delta=1e-2, r_proxy=0.75, far=False):
    """Sec. 4, Ex. 2: a cluster grown so that every sphere has a neighbour delta away, held fixed
    in the shear flow u_inf = (5 y, 0, 0); basic method (no images, as the paper runs it), N = 686,
    M0 = 823, GMRES tolerance 1e-6.  Every sphere shares the basic factor (one SVD), so step 1 of
    the passes runs on the tensor cores; with far=True the passes use the far field as well.
    Reports the solve (CUDA events), its iterations against Table cluster_table, the largest
    relative surface residual (eq. residual) on the check grids of up to 20 spheres, and
    max |lambda|."""
    import torch
    from paper_2407_03343_gb300 import mfs, workloads
    centres = workloads.cluster(P, delta, seed=1)
    st = torch.cuda.Stream()
    ctx = mfs.Context(device, stream=st.cuda_stream)
    ctx.set_spheres(centres)
    kw = dict(n_proxy=686, r_proxy=r_proxy, m_basic=823, nim_fixed=0)
    if far:
        kw.update(FAR)
    t0 = time.perf_counter()
    ctx.build(**kw)
    setup = time.perf_counter() - t0
    U, E, Om = workloads.shear_flow(5.0)
    ctx.set_background_flow(U=U, E=E, Omega=Om)
    ctx.set_rigid_velocities(np.zeros((P, 3)), np.zeros((P, 3)))
    ctx.set_profiling(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    info = ctx.solve(precision="mixed", tol=1e-6, allow_not_converged=True)
    e1.record(st)
    e1.synchronize()
    t = ctx.timing(reset=True)
    # check grid: the 500-point Fibonacci grid of the spheres, axes permuted (y, z, x)
    n = 500
    j = np.arange(1, n + 1)
    ct = 1.0 - (2.0 * j - 1.0) / n
    ph = np.mod(2.0 * np.pi * j / ((1.0 + 5.0 ** 0.5) / 2.0), 2.0 * np.pi)
    st_ = np.sqrt(1.0 - ct * ct)
    chk = np.stack([st_ * np.cos(ph), st_ * np.sin(ph), ct], axis=1)[:, [1, 2, 0]]
    ks = np.linspace(0, P - 1, min(P, 20)).astype(int)
    x = np.concatenate([centres[k] + chk for k in ks])
    u = ctx.eval_velocity(x)
    ubc = -(U[None, :] + x @ E.T + np.cross(Om[None, :], x))
    # pointwise ratio where |u_bc| is at least 1e-2 of its largest value on the sphere (the shear
    # flow vanishes on the plane y = 0, through the cluster); the plain maximum is reported too
    nb = np.linalg.norm(ubc, axis=1).reshape(len(ks), -1)
    err = np.linalg.norm(u - ubc, axis=1).reshape(len(ks), -1)
    keep = nb >= 1e-2 * nb.max(axis=1, keepdims=True)
    eres = float((err[keep] / nb[keep]).max())
    eres_all = float((err / nb).max())
    lam = ctx.strengths()
    s = ctx.sizes()
    out = {"spheres": P, "delta": delta, "r_proxy": r_proxy, "far_field": far, "setup_s": setup,
           "solve_s": e0.elapsed_time(e1) / 1000.0, "iters": info.iters, "converged": info.converged,
           "rel_residual": info.rel_residual, "eps_res_max_sampled": eres, "eps_res_max_sampled_all_points": eres_all,
           "spheres_checked": int(len(ks)),
           "lambda_max": float(np.abs(lam).max()), "dof": 3 * s.n_colloc, "factors": s.n_factors,
           "near_ms": t.pair_ms, "far_ms": t.far_ms, "gemv_ms": t.gemv_ms,
           "paper_P100_iters": {"1e-2,0.75": 92, "1e-3,0.75": 122, "1e-3,0.65": 116},
           "paper_P2000_iters": {"1e-2,0.75": 144, "1e-3,0.75": 176, "1e-3,0.65": 156},
           "paper_cpu_time_h": {"P100": 0.51, "P2000": 12.8}}
    ctx.close()
    return out


def profile_case(kind, device):
    """Small cases for ncu captures: the far-field and tensor-core kernels (two pass applies), and
    the step-1 GEMVs of three right-hand sides per geometry (three gap-sweep geometries with the
    three motions each, four lockstep iterations; ~2 GB of factors)."""
    from paper_2407_03343_gb300 import mfs, workloads
    if kind == "gemv_rhs":
        ctxs = []
        for gap in (1e-3, 1e-2, 1e-1):
            c = mfs.Context(device)
            c.set_spheres(workloads.two_spheres(gap))
            c.build(n_proxy=N_PROXY, r_proxy=R_PROXY, m_basic=M_BASIC)
            ctxs.append(c)
        probs = [c for _ in MOTIONS for c in ctxs]
        vel = [workloads.motion(m) for m in MOTIONS for _ in ctxs]
        mfs.batch_solve_rhs(probs, vel, mfs.default_solve_opts(precision="mixed", tol=1e-12, max_iter=4, max_refine=1),
                            allow_not_converged=True)
        for c in ctxs:
            c.close()
        print(json.dumps({"profile_case": kind}))
        return
    ctx = mfs.Context(device)
    if kind == "far":
        # 343 spheres on a 7 x 7 x 7 lattice 3 radii apart (no contacts: one shared factor, little
        # device memory), 480 nodes each: 343 tiles of 512 nodes, 4 per thread, as in the
        # 200-sphere suspension; 6 near neighbours, 336 far spheres
        g = np.arange(7) * 3.0
        ctx.set_spheres(np.array([[x, y, z] for x in g for y in g for z in g]))
        ctx.build(n_proxy=160, r_proxy=R_PROXY, m_basic=480, **FAR)
    else:
        g = np.arange(4) * 3.0
        c = np.array([[x, y, z] for x in g for y in g for z in g])[:60]
        ctx.set_spheres(c)
        ctx.build(n_proxy=N_PROXY, r_proxy=R_PROXY, m_basic=M_BASIC, tensor_step1=2)
    mu = ctx.rhs()
    for _ in range(2):
        ctx.apply_operator(mu, mfs.MIXED_PASS)
    ctx.close()
    print(json.dumps({"profile_case": kind}))


def batched_suspensions(device, n_problems=16, p_hi=8):
    """Many small independent suspensions (P_i log-uniform in [2, p_hi], volume fraction
    U(0.05, 0.3), gaps of attached spheres log-uniform in [1e-3, 1e-1]; N = 400, M0 = 800,
    R_p = 0.63): one lockstep MIXED batch against the same problems solved one after another in
    plain FP64, both at tol 1e-6, wall time including host synchronisation."""
    import threading as th
    from paper_2407_03343_gb300 import mfs, workloads
    cents = workloads.batch(n_problems=n_problems, seed=5, p_lo=2, p_hi=p_hi)
    ctxs = [mfs.Context(device) for _ in cents]
    errs = []

    def build(i):
        try:
            ctxs[i].set_spheres(cents[i])
            ctxs[i].build(n_proxy=400, r_proxy=0.63, m_basic=800)
        except Exception as e:  # surfaced below
            errs.append(e)
    t0 = time.perf_counter()
    thr = [th.Thread(target=build, args=(i,)) for i in range(len(ctxs))]
    [t.start() for t in thr]
    [t.join() for t in thr]
    if errs:
        raise errs[0]
    setup = time.perf_counter() - t0
    for i, c in enumerate(ctxs):
        v, w = workloads.rigid_velocities(cents[i].shape[0], seed=100 + i)
        c.set_rigid_velocities(v, w)
        c.set_profiling(True)
        c.timing(reset=True)
    t0 = time.perf_counter()
    infos = mfs.batch_solve(ctxs, precision="mixed", tol=1e-6, allow_not_converged=True)
    t_mixed = time.perf_counter() - t0
    ft_mixed = [np.concatenate([a.ravel() for a in c.forces_torques()]) for c in ctxs]
    pairs = sum(c.timing(reset=True).pair_interactions for c in ctxs)
    t0 = time.perf_counter()
    for c in ctxs:
        c.solve(precision="fp64", tol=1e-6, allow_not_converged=True)
    t_fp64 = time.perf_counter() - t0
    ft_err = max(float(np.abs(a - np.concatenate([x.ravel() for x in c.forces_torques()])).max()
                       / max(1e-300, np.abs(a).max())) for a, c in zip(ft_mixed, ctxs))
    out = {"problems": len(ctxs), "spheres": int(sum(c.shape[0] for c in cents)),
           "contacts": int(sum(workloads.count_near_contacts(c)[0] for c in cents)), "setup_s": setup,
           "mixed_batch_s": t_mixed, "fp64_sequential_s": t_fp64, "speedup": t_fp64 / t_mixed,
           "mixed_pairs_per_s": pairs / t_mixed, "converged": int(sum(i.converged for i in infos)),
           "max_ft_diff_mixed_vs_fp64": ft_err}
    for c in ctxs:
        c.close()
    return out


def sweep_accuracy(ctxs, d_F, d_T, probs):
    """Errors of the last solved sweep against the oracle's solutions stored by
    tests/golden/make_gap_sweep_oracle.py (O3 to 1e-9): the force/torque error of every one of
    the 54 problems, max |F - F_o|, |T - T_o| over the problem's 12 components relative to the
    largest of them, and the surface-velocity error at the stored check points of the problems
    each context still holds (its last right-hand side), max |u - u_o| relative to max |u_o|.
    Computed outside the timed region."""
    import torch
    if not os.path.exists(GOLDEN):
        return {"error": "oracle values missing: " + os.path.relpath(GOLDEN, ROOT)}
    gold = json.load(open(GOLDEN))
    ng = len(ctxs)
    ft_err, u_err = [], []
    torch.cuda.synchronize()
    for i, c in enumerate(probs):
        g = gold["geometries"][i % ng]["problems"][i // ng]
        F, T = d_F[i].cpu().numpy(), d_T[i].cpu().numpy()
        Fo, To = np.array(g["F"]), np.array(g["T"])
        ref = max(np.abs(Fo).max(), np.abs(To).max())
        ft_err.append(max(np.abs(F - Fo).max(), np.abs(T - To).max()) / ref)
    last = len(MOTIONS) - 1
    for gi, c in enumerate(ctxs):
        geo = gold["geometries"][gi]
        x = np.array(geo["check_points"])
        uo = np.array(geo["problems"][last]["u"])
        u = c.eval_velocity(x)
        u_err.append(float(np.abs(u - uo).max() / np.abs(uo).max()))
    return {"ft_rel_err_max": float(max(ft_err)), "ft_rel_err_median": float(statistics.median(ft_err)),
            "ft_problems": len(ft_err), "u_rel_err_max": float(max(u_err)), "u_problems": len(u_err),
            "u_points_per_problem": int(np.array(gold["geometries"][0]["check_points"]).shape[0]),
            "targets": {"u": 1e-3, "ft": 1e-5},
            "oracle": "O3 matrix-free GMRES on eq. resistance to 1e-9 (tests/golden/gap_sweep_oracle.json)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    cfg = workload_config(args)
    for _ in range(args.warmup):
        oracle_sample(2.0)
    vals, t0 = [], time.perf_counter()
    for _ in range(args.steps):
        vals.append(oracle_sample(8.0))
    el = time.perf_counter() - t0
    v = sum(x["value"] for x in vals) / len(vals)
    line = {"impl": "reference", "metric": "Stokeslet pair-interactions/s", "value": v,
            "unit": "pair-interactions/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": dict(vals[-1], value=v),
            "e2e": {"value": v, "unit": "pair-interactions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    rank, world, local = dist_env()
    import torch
    from paper_2407_03343_gb300 import mfs, workloads

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    mfs.lib()
    if args.profile_case:
        profile_case(args.profile_case, local)
        return 0
    if args.cluster_example:
        print(json.dumps({"cluster_example": cluster_example(local, args.cluster_example, far=True)}))
        return 0

    gaps = workloads.gap_sweep_gaps()
    streams = [torch.cuda.Stream() for _ in gaps]
    ctxs = [mfs.Context(local, stream=s.cuda_stream) for s in streams]

    # ---- setup (discretisation + one-body SVDs), concurrently across gaps
    t_setup = time.perf_counter()
    errs = []

    def build(i):
        try:
            ctxs[i].set_spheres(workloads.two_spheres(gaps[i]))
            ctxs[i].build(n_proxy=N_PROXY, r_proxy=R_PROXY, m_basic=M_BASIC)
        except Exception as e:  # surfaced below
            errs.append(e)
    th = [threading.Thread(target=build, args=(i,)) for i in range(len(gaps))]
    [t.start() for t in th]
    [t.join() for t in th]
    if errs:
        raise errs[0]
    setup_s = time.perf_counter() - t_setup
    sizes = [c.sizes() for c in ctxs]

    prec = args.precision
    opts = mfs.default_solve_opts(precision=prec, tol=args.tol, restart=args.restart)
    vel = {m: workloads.motion(m) for m in MOTIONS}
    if args.kernel_case:
        # the benchmark's 54-problem batch, cut off after this many GMRES iterations
        kprobs = [c for _ in MOTIONS for c in ctxs]
        kvel = [vel[m] for m in MOTIONS for _ in ctxs]
        mfs.batch_solve_rhs(kprobs, kvel, mfs.default_solve_opts(precision=prec, tol=1e-12, max_iter=args.kernel_case,
                                                                 max_refine=1), allow_not_converged=True)
        torch.cuda.synchronize()
        print(json.dumps({"kernel_case": args.kernel_case, "setup_s": setup_s}))
        return 0
    dev = torch.device("cuda", local)
    d_vel = {m: (torch.tensor(v, dtype=torch.float64, device=dev), torch.tensor(w, dtype=torch.float64, device=dev))
             for m, (v, w) in vel.items()}
    # the 54 problems: every geometry with each of the three motions, one lockstep batch in which
    # the three right-hand sides of a geometry share its factor reads
    probs = [c for _ in MOTIONS for c in ctxs]
    vel_host = [vel[m] for m in MOTIONS for _ in ctxs]
    d_F = [torch.zeros((2, 3), dtype=torch.float64, device=dev) for _ in probs]
    d_T = [torch.zeros((2, 3), dtype=torch.float64, device=dev) for _ in probs]
    v_ptrs = [d_vel[m][0].data_ptr() for m in MOTIONS for _ in ctxs]
    w_ptrs = [d_vel[m][1].data_ptr() for m in MOTIONS for _ in ctxs]
    F_ptrs = [t.data_ptr() for t in d_F]
    T_ptrs = [t.data_ptr() for t in d_T]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    main_stream = torch.cuda.current_stream()

    def device_step():
        return mfs.batch_solve_rhs_device(probs, v_ptrs, w_ptrs, F_ptrs, T_ptrs, opts)

    def timed_step(fn):
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(main_stream)
        for s in streams:
            s.wait_event(start)
        out = fn()
        for s in streams:
            e = torch.cuda.Event()
            e.record(s)
            main_stream.wait_event(e)
        end.record(main_stream)
        end.synchronize()
        return start.elapsed_time(end), out

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for c in ctxs:
        c.set_profiling(True)
    for _ in range(args.warmup):
        timed_step(device_step)
        flush.fill_(1.0)
    for c in ctxs:
        c.timing(reset=True)

    clk = ClockSampler(local)
    barrier()
    clk.start()
    ms = []
    iters = []
    for _ in range(args.steps):
        t, infos = timed_step(device_step)
        ms.append(t)
        iters.append(sum(i.iters for i in infos))
        flush.fill_(1.0)
    barrier()
    clocks = clk.stop()
    tms = [c.timing(reset=True) for c in ctxs]
    total_ms = sum(ms)
    pairs = sum(t.pair_interactions for t in tms)
    launches = sum(t.kernel_launches for t in tms)
    pair_ms = sum(t.pair_ms for t in tms)
    pair_launches = sum(t.pair_launches for t in tms)
    gemv_ms = sum(t.gemv_ms for t in tms)
    gemv_bytes = sum(t.gemv_bytes for t in tms)
    gemv_launches = sum(t.gemv_launches for t in tms)
    krylov_ms = sum(t.krylov_ms for t in tms)
    krylov_bytes = sum(t.krylov_bytes for t in tms)

    # max over ranks of the timed region, pairs summed over ranks (weak scaling: every rank
    # solves its own sweep, no data-path collective)
    total_ms_max, pairs_all = reduce_over_ranks(total_ms, pairs, dev if world > 1 else None)
    value = pairs_all / (total_ms_max / 1000.0)

    # ---- roofline of the dominant kernel (pair kernel), from its own launch events:
    # algorithmic flops = proxy pairs x 28 + image node-pairs x 63, counted by the library for
    # every pair launch in the timed steps, over the device time of those launches
    kind = 1 if prec == "mixed" else 0   # MFS_MIXED or MFS_FP64 pair kernel
    k_ms = sum(t.by_kind_ms[kind] for t in tms)
    k_launch = sum(t.by_kind_launches[kind] for t in tms)
    k_proxy = sum(t.by_kind_proxy[kind] for t in tms)
    k_image = sum(t.by_kind_image_nodes[kind] for t in tms)
    alg_flops = k_proxy * FLOPS_ALG[0] + k_image * FLOPS_ALG[1]
    # FP32-pipe flops the double-float evaluation issued, counted by the library (a pair geometry
    # shared by several right-hand sides on one geometry is evaluated once)
    issued_flops = sum(t.pair_issued_flops for t in tms)
    shared_rhs = sum(t.pair_shared_rhs for t in tms)
    achieved_tflops = alg_flops / (k_ms / 1000.0) / 1e12 if k_ms > 0 else 0.0
    fp64_refine = {"launches": sum(t.by_kind_launches[0] for t in tms), "ms": sum(t.by_kind_ms[0] for t in tms)}
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    sm_mhz = clocks["sm_mhz"] or sm_max
    # FP32 FMA lanes x 2 flops x the median SM clock sampled under load (152 SMs x 128 lanes)
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    probe = {}
    try:
        p32, ms32p = mfs.probe_alu_peak(local, "fp32")
        p64, ms64p = mfs.probe_alu_peak(local, "fp64")
        probe = {"fp32_ffma_tflops": p32, "fp64_dfma_tflops": p64, "launch_ms": [ms32p, ms64p]}
    except Exception as e:  # measured peak is context only; the roofline uses the derived one
        probe = {"error": str(e)}
    fp64_peak = probe.get("fp64_dfma_tflops") or 1.0
    peak = fp32_peak if prec == "mixed" else fp64_peak
    roofline = {"bound": "alu", "kernel": "pairs_dw_batch_kernel" if prec == "mixed" else "pairs_batch_kernel<double>",
                "achieved": achieved_tflops, "peak": peak, "unit": "TFLOP/s", "frac": achieved_tflops / peak,
                "flops_per_unit": {"stokeslet_pair": FLOPS_ALG[0], "image_triple": FLOPS_ALG[1]},
                "units_per_launch": {"proxy_pairs": k_proxy / max(k_launch, 1),
                                     "image_node_pairs": k_image / max(k_launch, 1)},
                # dram read + write of one captured launch (ncu, 18 gap-sweep problems, see profiles/)
                "traffic": PAIR_DW_TRAFFIC_BYTES if prec == "mixed" else None,
                "traffic_launch": "pairs_dw_multi_kernel<3>, 9-problem launch of --profile-case gemv_rhs"
                if prec == "mixed" else None,
                "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 flops x median SM clock under load"
                if prec == "mixed" else "FP64 DFMA probe (mfs_probe_alu_peak)",
                "peak_probe": probe,
                "avg_launch_us": 1000.0 * k_ms / max(k_launch, 1),
                "share_of_step": k_ms / total_ms if total_ms > 0 else None,
                "fp64_refinement_pair_launches": fp64_refine}
    if prec == "mixed":
        # FP32-pipe operations actually issued by the compensated double-float evaluation
        roofline["issue_frac"] = issued_flops / (k_ms / 1000.0) / 1e12 / fp32_peak if k_ms > 0 else None
        # pair interactions (per right-hand side, the metric's unit) evaluated in items where the
        # three motions of a gap share each pair's geometry; frac counts 28 / 63 flops for each
        roofline["shared_rhs_frac"] = shared_rhs / max(1, k_proxy + 3 * k_image)
        roofline["kernel"] = "pairs_dw_multi_kernel + pairs_dw_batch_kernel"
    gemv = {"GBps": gemv_bytes / (gemv_ms / 1000.0) / 1e9 if gemv_ms > 0 else None,
            "frac_of_hbm": gemv_bytes / (gemv_ms / 1000.0) / 1e9 / hbm_peak if gemv_ms > 0 else None,
            "share_of_step": gemv_ms / total_ms if total_ms > 0 else None, "launches": gemv_launches,
            "bytes": "factor bytes read: Sigma^+ U^T (FP32 in the passes, hi/lo pairs in residuals) and V (hi/lo)"}
    krylov = {"GBps": krylov_bytes / (krylov_ms / 1000.0) / 1e9 if krylov_ms > 0 else None,
              "frac_of_hbm": krylov_bytes / (krylov_ms / 1000.0) / 1e9 / hbm_peak if krylov_ms > 0 else None,
              "share_of_step": krylov_ms / total_ms if total_ms > 0 else None,
              "bytes": "(4j + 10) n doubles per Arnoldi step j: two dot-product and two update launches of CGS2"}
    accuracy = sweep_accuracy(ctxs, d_F, d_T, probs) if rank == 0 else None

    # ---- end to end through host buffers
    e2e_ms = []
    h2d = d2h = 0
    barrier()
    for _ in range(max(1, min(args.steps, 3))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mfs.batch_solve_rhs(probs, vel_host, opts)   # host velocities in, host forces/torques out
        e2e_ms.append(1000.0 * (time.perf_counter() - t0))
    h2d = len(MOTIONS) * len(ctxs) * 2 * 6 * 8
    d2h = len(MOTIONS) * len(ctxs) * 2 * 6 * 8
    pairs_per_step = pairs / args.steps
    e2e_value = pairs_per_step / (statistics.mean(e2e_ms) / 1000.0)

    extras = {}
    if not args.no_extras and rank == 0:
        # plain FP64 GPU solve of the same sweep against the mixed one (the metric's second part),
        # each timed with CUDA events over repeats, both checked against the oracle
        o64 = mfs.default_solve_opts(precision="fp64", tol=args.tol, restart=args.restart)
        solve_ms = {}
        for name, o, reps in (("fp64", o64, 2), ("mixed", opts, 5)):
            ts = []
            for _ in range(reps):
                flush.fill_(1.0)
                t, _ = timed_step(lambda: mfs.batch_solve_rhs_device(probs, v_ptrs, w_ptrs, F_ptrs, T_ptrs, o))
                ts.append(t)
            solve_ms[name] = ts
            if name == "fp64":
                acc64 = sweep_accuracy(ctxs, d_F, d_T, probs)
        for c in ctxs:
            c.timing(reset=True)
        m64, mmix = statistics.median(solve_ms["fp64"]), statistics.median(solve_ms["mixed"])
        extras["sweep_solve_s"] = {"fp64": m64 / 1000.0, "mixed": mmix / 1000.0, "speedup": m64 / mmix,
                                   "tol": args.tol, "repeats": {k: len(v) for k, v in solve_ms.items()},
                                   "timing": "CUDA events on the launching stream, median of the repeats",
                                   "accuracy_fp64": acc64}
        # FP32 pair kernel on the same problems (inner solves of the FP32 mode, 30 iterations each)
        o32 = mfs.default_solve_opts(precision="fp32", tol=1e-6, max_iter=30, max_refine=1)
        for c in ctxs:
            c.set_rigid_velocities(*vel["squeeze"])
        mfs.batch_solve(ctxs, o32, allow_not_converged=True)
        t32 = [c.timing(reset=True) for c in ctxs]
        p32 = sum(t.pair_interactions for t in t32)
        ms32 = sum(t.pair_ms for t in t32)
        fl32 = sum(t.pair_proxy * 28.0 + t.pair_image_nodes * 63.0 for t in t32)
        extras["fp32_pair_kernel"] = {"pairs_per_s": p32 / (ms32 / 1000.0) if ms32 else None,
                                      "tflops": fl32 / (ms32 / 1000.0) / 1e12 if ms32 else None,
                                      "frac_of_fp32_peak": (fl32 / (ms32 / 1000.0) / 1e12) / fp32_peak if ms32 else None,
                                      "avg_launch_us": 1000.0 * ms32 / max(1, sum(t.pair_launches for t in t32))}
        extras["cpu_baseline"] = oracle_sample(15.0)
        extras["oracle_solve"] = oracle_solve_sample()
        extras["pair_kernels_200_spheres"] = suspension_kernel_rates(local, fp32_peak)
        extras["batched_suspensions"] = batched_suspensions(local)
        extras["cluster_shear_P100"] = cluster_example(local, 100)
        if args.suspension > 0:
            extras["suspension_far_field_solve"] = suspension_solve(local, args.suspension, args.tol)

    if rank == 0:
        line = {"metric": "Stokeslet pair-interactions/s", "value": value, "unit": "pair-interactions/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64 (pair sums double-float on FP32 pipes)" if prec == "mixed" else "f64",
                "data": "synthetic", "config": workload_config(args),
                "roofline": roofline, "gemv": gemv, "krylov": krylov, "accuracy": accuracy, "clocks": clocks,
                "e2e": {"value": e2e_value, "unit": "pair-interactions/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "ms_per_step": statistics.mean(e2e_ms)},
                "gpu_launches": launches, "setup_s": setup_s,
                "gmres_iters_per_step": statistics.mean(iters) if iters else None}
        if "cpu_baseline" in extras:
            line["cpu_baseline"] = extras.pop("cpu_baseline")
        line.update(extras)
        print(json.dumps(line))
    for c in ctxs:
        c.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
