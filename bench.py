"""Benchmark: batched parametric slab solves to a 1e-6 relative flux change.

Workload: 4096 independent single-group slabs (10 cm), cells ~ U{64..2048},
Gauss-Legendre S_N with N even ~ U{8..64}, sinusoidal or piecewise
coefficients and clipped Fourier sources from per-instance seeds (the
batched parametric workload).  One step solves the whole batch: the warm
start when a trained operator is available, then the FP32 source iterations
with FP64 norms, all through the C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank solves its own batch
(rank-seeded): weak scaling, no collective on the data path.
"""
import argparse
import collections
import json
import multiprocessing as mp
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "solves/s to 1e-6 residual (batched slab S_N solve), neural-operator warm start"
UNIT = "solves/s"
TOL = 1e-6
RECAST_TOL = 1e-3
RECAST_ITMAX = 10
# DRAM bytes (read + write) of one warm-step sweep launch on this workload,
# from the ncu capture summarised in profiles/sn1d_kernel_4096slab.txt; None
# once the sweep kernel changes until it is captured again.
SWEEP_TRAFFIC_BYTES = 70_240_000 + 31_363_584
WORKLOAD = ("4096 slabs, cells U{64..2048}, GL S_N N even U{8..64}, sinusoidal or "
            "piecewise coefficients, Fourier sources, vacuum, tol 1e-6 rel. L2 flux change")


# ------------------------------------------------------------ multi-rank
def rank_instances(rank, limit=0):
    """The rank's own batch: the 4096-slab recipe seeded by the rank (weak
    scaling; ranks share no instances and exchange no data)."""
    return W.slab_batch(seed=5 + rank, n_inst=limit if limit > 0 else 4096)


def max_over_ranks(x, world, device):
    """Largest value of x over the ranks (the job's elapsed time)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, steps, seconds):
    """Units all ranks processed divided by the slowest rank's time."""
    return world * units_per_rank * steps / seconds


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# --------------------------------------------------------------- oracle leg
def _oracle_one(args):
    I, N, L, sigt, sigs, Q = args
    from oracle import quadrature as Qd
    from oracle import transport as T
    P = T.uniform_slab(I, L, sigt, sigs, Q=Q)
    T.source_iteration(P, Qd.gauss_legendre(N), tol=TOL, itmax=200000)
    return I * N


def oracle_rate(insts, seconds, seed=0, pool=None):
    """Solve a random sample of the batch with the FP64 oracle on all host
    cores for about `seconds`; returns (solves/s, cores, n_solved, elapsed).
    At most two jobs per core are in flight: once the time is up nothing new
    is submitted, the jobs in flight are waited for and counted, and no work
    is left queued in the pool for a later call."""
    cores = os.cpu_count() or 1
    own = pool is None
    if own:
        pool = mp.get_context("spawn").Pool(cores)
    order = np.random.default_rng(seed).permutation(len(insts))
    jobs = [(insts[b].I, insts[b].N, insts[b].L, insts[b].sigt, insts[b].sigs, insts[b].Q)
            for b in order]
    t0 = time.perf_counter()
    done, nxt = 0, 0
    pending = collections.deque()
    while True:
        while (nxt < len(jobs) and len(pending) < 2 * cores and
               time.perf_counter() - t0 < seconds):
            pending.append(pool.apply_async(_oracle_one, (jobs[nxt],)))
            nxt += 1
        if not pending:
            break
        pending.popleft().get()
        done += 1
    el = time.perf_counter() - t0
    if own:
        pool.terminate()
        pool.join()
    return done / el if el > 0 else 0.0, cores, done, el


# ----------------------------------------------------- per-config lines
def _events_ms(torch, stream, fn, reps=3):
    """Median CUDA-event time (ms) of fn() on `stream` over reps runs after one warm-up."""
    fn()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts)), out


def run_configs(s, stream, deeponet_params, local):
    """The four single-problem workloads on the GPU: plain guess and neural-
    operator warm start, time to tolerance (CUDA events), iterations.  Each
    operator is the workload's own, trained untimed at p* on solutions the
    solver produces.  Returns (results, raw answers for the oracle leg)."""
    import torch
    from paper_2509_01416_gb300 import NOP_NO_FNO1D, NOP_NO_FNO2D, NOP_NO_DEEPONET, no_config
    from paper_2509_01416_gb300 import train as TR
    res, raw = {}, {}
    clk = Clocks(local, os.path.join(ROOT, ".bench_clocks_configs.csv"))
    clk.__enter__()
    # ---- 1: uniform slab, S16, plain method, FP64 to a 1e-8 change
    c = W.uniform_slab_s16()
    s.set_slabs([c.I], [c.L], [c.N], c.sigt, c.sigs, source=c.Q)
    clk.mark(True)
    ms, (phi, info) = _events_ms(torch, stream, lambda: s.solve_fixed_source(
        tol=1e-8, itmax=100000, precision=1))
    res["1_uniform_slab_s16"] = {"plain": {"ms": ms, "iterations": int(info["iterations"][0])},
                                 "precision": "f64", "tol": 1e-8}
    raw["1"] = phi
    # ---- 2: heterogeneous slab, S32, DeepONet warm start (the batch's operator)
    c = W.hetero_slab_s32()
    cfg2 = no_config(NOP_NO_DEEPONET, sensors=128, width=128, basis=128, depth=4,
                     sigma_t_star=W.P_STAR[0], sigma_s_star=W.P_STAR[1], length=W.L_SLAB)
    s.no_set(cfg2, deeponet_params)
    s.set_slabs([c.I], [c.L], [c.N], c.sigt, c.sigs, source=c.Q)
    kw = dict(tol=1e-6, itmax=100000, precision=0)
    mp_, (pp, ip) = _events_ms(torch, stream, lambda: s.solve_fixed_source(**kw))
    mw, (pw, iw) = _events_ms(torch, stream, lambda: s.solve_fixed_source(
        warm_start=1, recast_tol=RECAST_TOL, recast_itmax=RECAST_ITMAX, **kw))
    res["2_hetero_slab_s32"] = {
        "plain": {"ms": mp_, "iterations": int(ip["iterations"][0])},
        "warm": {"ms": mw, "iterations": int(iw["iterations"][0]),
                 "recast_iterations": int(iw["recast_iterations"])},
        "operator": "DeepONet 128 sensors, 4x128, p=128 (the batch's, trained above)",
        "precision": "f32 sweeps, f64 norms", "tol": 1e-6}
    raw["2"] = (pp, pw)
    # ---- 3: three-region eigen slab, S32, FNO-1D (width 64, 32 modes) warm start
    c = W.eigen_slab_s32()
    nsf = c.nusigf.copy()
    s.set_slabs([c.I], [c.L], [c.N], c.sigt, c.sigs, nu_sigma_f=nsf, chi=[1.0])
    k0, _, _ = s.solve_eigen(tol=1e-7, tol_k=1e-9, tol_inner=1e-7, itmax=5000, precision=0,
                             allow_noconv=True)
    nsf = nsf * (c.k_target / k0[0])      # production scaled so that k is the recipe's target
    cfg3 = no_config(NOP_NO_FNO1D, width=64, modes=32, depth=4, proj=128, length=W.L_SLAB)
    s.no_set(cfg3, W.fno1d_init(31, width=64, modes=32, proj=128))
    t0 = time.perf_counter()
    S3, Y3, _ = TR.fno1d_training_set(s, cfg3, W.training_sources(32, 400, c.I))
    h3 = TR.train_fno(s, S3, Y3, steps=800, batch=20, seed=33, lr=2e-3)
    tr3 = time.perf_counter() - t0
    s.set_slabs([c.I], [c.L], [c.N], c.sigt, c.sigs, nu_sigma_f=nsf, chi=[1.0])
    kw = dict(tol=1e-6, tol_k=1e-7, tol_inner=1e-6, itmax=5000, itmax_inner=5000, precision=0)
    mp_, (kp, pp, ip) = _events_ms(torch, stream, lambda: s.solve_eigen(**kw))
    mw, (kwv, pw, iw) = _events_ms(torch, stream, lambda: s.solve_eigen(
        warm_start=1, recast_tol=1e-3, recast_itmax=50, **kw))
    res["3_eigen_slab_s32"] = {
        "plain": {"ms": mp_, "inner": int(ip["inner"][0]), "outer": int(ip["outer"]),
                  "k": float(kp[0])},
        "warm": {"ms": mw, "inner": int(iw["inner"][0]), "outer": int(iw["outer"]),
                 "k": float(kwv[0]), "recast_iterations": int(iw["recast_iterations"])},
        "operator": "FNO-1D width 64, 32 modes, 4 layers (simple preconditioning, App. A2)",
        "training": {"samples": 400, "steps": 800, "seconds": tr3,
                     "loss_first": float(h3[0]), "loss_last": float(np.mean(h3[-20:]))},
        "k_target": c.k_target, "precision": "f32 sweeps, f64 norms and k",
        "tol": {"flux": 1e-6, "k": 1e-7}}
    raw["3"] = (nsf, kp[0], pp, kwv[0], pw)
    # ---- 4: 256x256 8-group checkerboard, LS S8, FNO-2D warm start
    c = W.checkerboard_xy_8g()
    bc = tuple(c.bc[f] for f in ("x0", "xL", "y0", "yL"))
    cfg4 = no_config(NOP_NO_FNO2D, width=32, modes=16, depth=4, proj=128, length=c.Lx)
    s.no_set(cfg4, W.fno2d_init(4, width=32, modes=16, proj=128))
    t0 = time.perf_counter()
    S4, Y4 = TR.fno2d_training_set(s, cfg4, W.training_sources_2d(6, 8, c.nx), bc=bc)
    h4 = TR.train_fno(s, S4, Y4, steps=60, batch=2, seed=2, lr=2e-3)
    tr4 = time.perf_counter() - t0
    s.set_xy(c.nx, c.ny, c.Lx, c.Ly, c.sigt.reshape(-1), c.sigs.reshape(-1),
             nu_sigma_f=c.nusigf.reshape(-1), chi=c.chi, bc=bc)
    # |dk|/k below about 1e-9 is under the noise of k from FP32 fluxes: the
    # outer loop then stops only when the noise happens to fall below it
    kw = dict(tol=1e-7, tol_k=1e-8, tol_inner=1e-7, itmax=2000, itmax_inner=120, precision=0,
              allow_noconv=True)
    mp_, (kp, pp, ip) = _events_ms(torch, stream, lambda: s.solve_eigen(**kw), reps=2)
    mw, (kwv, pw, iw) = _events_ms(torch, stream, lambda: s.solve_eigen(
        warm_start=1, recast_tol=1e-2, recast_itmax=10, **kw), reps=2)
    clk.mark(False)
    clk.__exit__()
    res["4_checkerboard_xy_8g"] = {
        "plain": {"ms": mp_, "inner": int(ip["inner"][0]), "outer": int(ip["outer"]),
                  "k": float(kp[0])},
        "warm": {"ms": mw, "inner": int(iw["inner"][0]), "outer": int(iw["outer"]),
                 "k": float(kwv[0]), "recast_iterations": int(iw["recast_iterations"])},
        "operator": "FNO-2D width 32, 16x16 modes, 4 layers (simple preconditioning)",
        "training": {"samples": 8, "steps": 60, "seconds": tr4,
                     "loss_first": float(h4[0]), "loss_last": float(np.mean(h4[-10:]))},
        "precision": "f32 sweeps, f64 norms and k", "iteration": "Jacobi in energy (default)",
        "tol": {"flux": 1e-7, "k": 1e-8}}
    raw["4"] = (kp[0], pp, kwv[0], pw)
    return res, raw, clk.summary()


def _oracle_config(job):
    """One config's FP64 oracle, single thread: (seconds, result)."""
    from oracle import quadrature as Qd
    from oracle import transport as T
    kind = job[0]
    t0 = time.perf_counter()
    if kind == "fixed":
        _, I, L, N, sigt, sigs, Q, tol = job
        r = T.source_iteration(T.uniform_slab(I, L, sigt, sigs, Q=Q), Qd.gauss_legendre(N),
                               tol=tol, itmax=1000000)
        out = (r.phi[0], r.iterations)
    elif kind == "eigen":
        _, I, L, N, sigt, sigs, nsf, tk, tp, ti = job
        e = T.power_iteration(T.uniform_slab(I, L, sigt, sigs, nusigf=nsf), Qd.gauss_legendre(N),
                              tol_k=tk, tol_phi=tp, tol_inner=ti)
        out = (e.phi[0], e.k, e.outer, e.inner_total)
    else:   # a bounded sample of the x-y oracle: two source iterations of config 4
        c = W.checkerboard_xy_8g()
        bcm = {k: (T.REFLECTIVE if v else T.VACUUM) for k, v in c.bc.items()}
        P = T.XY(dx=c.Lx / c.nx, dy=c.Ly / c.ny, sigt=c.sigt, sigs=c.sigs, nusigf=c.nusigf,
                 chi=c.chi, bc=bcm)
        T.source_iteration(P, Qd.level_symmetric_s8(), src=np.zeros_like(c.sigt),
                           phi0=np.ones_like(c.sigt), tol=0.0, itmax=2)
        out = None
    return time.perf_counter() - t0, out


def oracle_configs(res, raw, pool):
    """The oracle beside every config (single thread each, in parallel over
    configs): its time and iterations, and the GPU answers' errors against it."""
    from tests.helpers import rel_l2, xy_golden
    c1, c2, c3 = W.uniform_slab_s16(), W.hetero_slab_s32(), W.eigen_slab_s32()
    nsf3 = raw["3"][0]
    jobs = {
        "1": ("fixed", c1.I, c1.L, c1.N, c1.sigt, c1.sigs, c1.Q, 1e-8),
        "2": ("fixed", c2.I, c2.L, c2.N, c2.sigt, c2.sigs, c2.Q, 1e-6),
        "2c": ("fixed", c2.I, c2.L, c2.N, c2.sigt, c2.sigs, c2.Q, 1e-12),
        "3": ("eigen", c3.I, c3.L, c3.N, c3.sigt, c3.sigs, nsf3, 1e-7, 1e-6, 1e-6),
        "3c": ("eigen", c3.I, c3.L, c3.N, c3.sigt, c3.sigs, nsf3, 1e-12, 1e-10, 1e-12),
        "4": ("xy_sample",),
    }
    fut = {k: pool.apply_async(_oracle_config, (j,)) for k, j in jobs.items()}
    out = {k: f.get() for k, f in fut.items()}
    t1, (o1, it1) = out["1"]
    res["1_uniform_slab_s16"]["oracle"] = {"seconds": t1, "iterations": it1, "threads": 1}
    res["1_uniform_slab_s16"]["error_vs_oracle"] = {"flux_rel_l2_same_rule": rel_l2(raw["1"], o1)}
    t2, (o2, it2) = out["2"]
    _, (o2c, _) = out["2c"]
    pp, pw = raw["2"]
    res["2_hetero_slab_s32"]["oracle"] = {"seconds": t2, "iterations": it2, "threads": 1}
    res["2_hetero_slab_s32"]["error_vs_oracle"] = {
        "plain_flux_rel_l2_same_rule": rel_l2(pp, o2), "warm_flux_rel_l2_same_rule": rel_l2(pw, o2),
        "warm_flux_rel_l2_vs_converged": rel_l2(pw, o2c)}
    t3, (o3, k3, n3, in3) = out["3"]
    _, (o3c, k3c, _, _) = out["3c"]
    _, kp, pp, kw_, pw = raw["3"]
    res["3_eigen_slab_s32"]["oracle"] = {"seconds": t3, "outer": n3, "inner": in3, "k": k3,
                                         "threads": 1}
    res["3_eigen_slab_s32"]["error_vs_oracle"] = {
        "plain_dk_same_rule": abs(kp - k3), "warm_dk_same_rule": abs(kw_ - k3),
        "plain_flux_rel_l2_same_rule": rel_l2(pp, o3), "warm_flux_rel_l2_same_rule": rel_l2(pw, o3),
        "warm_dk_vs_converged": abs(kw_ - k3c), "warm_flux_rel_l2_vs_converged": rel_l2(pw, o3c)}
    t4, _ = out["4"]
    k0, g, j, i, ref, _ = xy_golden()
    c4 = W.checkerboard_xy_8g()
    kp, pp, kw_, pw = raw["4"]
    res["4_checkerboard_xy_8g"]["oracle"] = {
        "seconds_per_source_iteration": t4 / 2, "threads": 1,
        "seconds_to_converge_estimate": t4 / 2 * 918,
        "note": "a timed sample of 2 source iterations; the converged oracle solve "
                "(tests/golden/make_xy_golden.py) takes 918 inner iterations"}
    res["4_checkerboard_xy_8g"]["error_vs_oracle"] = {
        "plain_dk": abs(kp - k0), "warm_dk": abs(kw_ - k0),
        "plain_flux_rel_l2_sampled": rel_l2(pp.reshape(c4.sigt.shape)[g, j, i], ref),
        "warm_flux_rel_l2_sampled": rel_l2(pw.reshape(c4.sigt.shape)[g, j, i], ref),
        "against": "converged FP64 oracle (tests/golden/xy_checkerboard_8g.txt)"}
    return res


# ---------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampler (every 50 ms).  It starts before the plain-guess
    runs, so it is sampling by the time the warm-start region is timed;
    mark() brackets that region and summary() keeps the samples inside it
    (all samples if their timestamps cannot be read)."""

    def __init__(self, idx, path):
        self.idx, self.path, self.p = idx, path, None
        self.t0 = self.t1 = None

    def __enter__(self):
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + q,
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def mark(self, start):
        if start:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        import datetime
        try:
            rows = [[c.strip() for c in r.split(",")]
                    for r in open(self.path).read().strip().splitlines()]
        except Exception:
            return None
        def numeric(r):
            try:
                float(r[2])
                float(r[3])
                return True
            except ValueError:
                return False
        rows = [r for r in rows if len(r) > 9 and numeric(r)]
        if not rows:
            return None
        inside = []
        if self.t0 is not None and self.t1 is not None:
            for r in rows:
                try:
                    ts = datetime.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                except ValueError:
                    inside = []
                    break
                if self.t0 - 0.05 <= ts <= self.t1 + 0.05:
                    inside.append(r)
        used = inside or rows
        sm = [float(r[2]) for r in used]
        mx = [float(r[3]) for r in used]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in used:
            for k, v in zip(names, r[6:10]):
                if v.lower() in ("active", "0x1", "1"):
                    reasons.add(k)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm),
                "window": "timed warm-start region" if inside else "plain and warm-start runs"}


# ------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--train-steps", type=int, default=10000,
                    help="Adam steps of the operator's training (0: untrained operator, "
                         "no training set; for profiling runs)")
    ap.add_argument("--recast-tol", type=float, default=RECAST_TOL)
    ap.add_argument("--recast-itmax", type=int, default=RECAST_ITMAX)
    ap.add_argument("--xy-sweep", action="store_true",
                    help="profiling aid: time a fixed amount of x-y sweep work instead")
    ap.add_argument("--slab-sweep", type=int, default=0, metavar="N",
                    help="profiling aid: time the plain solve of the first N instances "
                         "of the batch instead (cold, tuned schedule)")
    ap.add_argument("--no-dsa", action="store_true",
                    help="skip the diffusion-synthetic-acceleration comparison runs")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the four single-problem workloads (per-config lines)")
    ap.add_argument("--instances", type=int, default=0,
                    help="solve only the first N instances of the batch (profiling aid)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    insts = rank_instances(rank, args.instances)
    cores = os.cpu_count() or 1

    if args.impl == "reference":
        if rank != 0:
            return
        run_reference(args, insts, world)
        return
    if args.xy_sweep:
        run_xy_sweep(local)
        return
    if args.slab_sweep > 0:
        run_slab_sweep(local, args.slab_sweep)
        return

    # the oracle's process pool starts before the first GPU call
    pool = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool = mp.get_context("spawn").Pool(cores)

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2509_01416_gb300 import Solver
    n, wdt, order, sigt, sigs, src, _ = W.slab_batch_arrays(insts)
    B, Ctot = len(insts), int(n.sum())
    stream = torch.cuda.Stream()
    s = Solver(local)
    s.set_stream(stream.cuda_stream)

    # ---- neural operator, trained once at p* on solver-generated solutions
    # (not timed): 2000 GRF sources on 512 cells, S32, Adam
    from paper_2509_01416_gb300 import NOP_NO_DEEPONET, no_config
    from paper_2509_01416_gb300 import train as TR
    cfg = no_config(NOP_NO_DEEPONET, sensors=128, width=128, basis=128, depth=4,
                    sigma_t_star=W.P_STAR[0], sigma_s_star=W.P_STAR[1], length=W.L_SLAB)
    torch.cuda.synchronize()
    t_tr = time.perf_counter()
    s.no_set(cfg, W.deeponet_init(1000 + rank))
    hist = None
    if args.train_steps > 0:
        U, Xc, Y, _ = TR.deeponet_training_set(s, cfg,
                                               W.training_sources(2000 + rank, 2000, 512))
        hist = TR.train(s, U, Xc, Y, steps=args.train_steps, batch=100, seed=3000 + rank)
    train_s = time.perf_counter() - t_tr

    s.set_slabs(n, wdt, order, sigt, sigs, source=src)
    phi_dev = torch.empty(Ctot, dtype=torch.float64, device="cuda")

    def step(warm=True, dsa=False, cold=False, schedule=0):
        return s.solve_fixed_source_dev(phi_dev.data_ptr(), tol=TOL, itmax=200000,
                                        precision=0, warm_start=1 if warm else 0,
                                        recast_tol=args.recast_tol,
                                        recast_itmax=args.recast_itmax, dsa=dsa, cold=cold,
                                        schedule=schedule)

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(warm, steps, clk=None, dsa=False, cold=False, schedule=0):
        for _ in range(max(3, args.warmup)):
            info = step(warm, dsa, cold, schedule)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.set_timing(True)
        barrier()
        torch.cuda.synchronize()
        if clk:
            clk.mark(True)
            # the timed warm-start region is the one a profiler started with
            # --profile-from-start off records
            torch.cuda.profiler.start()
        ev0.record(stream)
        for _ in range(steps):
            info = step(warm, dsa, cold, schedule)
        ev1.record(stream)
        torch.cuda.synchronize()
        if clk:
            torch.cuda.profiler.stop()
            clk.mark(False)
        barrier()
        tm = s.timing()
        s.set_timing(False)
        return max_over_ranks(ev0.elapsed_time(ev1), world, "cuda"), tm, info

    # the sweep's arithmetic ceilings, measured on this device (untimed)
    rcp_peak, fma_peak = s.measure_alu_peaks()
    # the first solve on this context measures the slab layouts' costs (the
    # autotuner); it is untimed like the training
    s.set_timing(True)
    step(False)
    tune_ms = s.timing()["last_tune_ms"]
    s.set_timing(False)
    clk = Clocks(local, os.path.join(ROOT, ".bench_clocks_rank%d.csv" % rank))
    clk.__enter__()
    half = max(1, args.steps // 2)
    # plain guess and the analytic-model schedule, both cold like the headline
    plain_ms, plain_tm, plain_info = timed(False, half, cold=True)
    model_ms, model_tm, _ = timed(False, half, cold=True, schedule=3)
    # headline: the warm start with a cold schedule (no iteration counts of
    # earlier solves of this batch), as for a batch seen for the first time
    ms_max, tm, info = timed(True, args.steps, clk, cold=True)
    clk.__exit__()
    cached_ms, cached_tm, cached_info = timed(True, args.steps)
    value = whole_job_rate(world, B, args.steps, ms_max / 1e3)
    plain_value = whole_job_rate(world, B, half, plain_ms / 1e3)
    # the classical accelerator of the iteration itself on the same batch, alone
    # and behind the warm start (not part of the headline metric)
    accel = {}
    if not args.no_dsa:
        for key, warm in (("dsa", False), ("warm_start_and_dsa", True)):
            k = max(1, args.steps // 2)
            ms_a, _, info_a = timed(warm, k, dsa=True)
            it_a = info_a["iterations"].astype(np.float64)
            accel[key] = {"value": whole_job_rate(world, B, k, ms_a / 1e3), "unit": UNIT,
                          "ms_per_step": ms_a / k, "iterations_mean": float(np.mean(it_a)),
                          "iterations_max": int(np.max(it_a))}

    # ---- end to end through the C ABI with host buffers (warm start): the
    # step's inputs go from pinned host memory to the device and the flux
    # comes back into a pinned buffer
    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.from_numpy(a[:0].copy()).dtype, pin_memory=True)
        v = t.numpy()
        v[...] = a
        return t, v
    host = [pinned(np.ascontiguousarray(a)) for a in (n, wdt, order, sigt, sigs, src)]
    hn, hw, ho, hst, hss, hsrc = [v for _, v in host]
    phi_pin = torch.empty(Ctot, dtype=torch.float64, pin_memory=True)
    phi_h = phi_pin.numpy()
    h2d = sum(v.nbytes for v in (hn, hw, ho, hst, hss, hsrc))
    d2h = 8 * Ctot + 8 * B
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.set_slabs(hn, hw, ho, hst, hss, source=hsrc)
        s.solve_fixed_source(tol=TOL, itmax=200000, precision=0, warm_start=1,
                             recast_tol=args.recast_tol, recast_itmax=args.recast_itmax,
                             out=phi_h, cold=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = whole_job_rate(world, B, args.steps, max_over_ranks(e2e_s, world, "cuda"))

    # ---- the four single-problem workloads beside the batch (rank 0, N=1)
    configs = cfg_raw = cfg_clk = None
    if rank == 0 and world == 1 and not args.no_configs:
        configs, cfg_raw, cfg_clk = run_configs(s, stream, s.no_get(), local)

    if rank != 0:
        s.close()
        if world > 1:
            dist.destroy_process_group()
        return

    peaks, src_peak = _peaks()
    ck = clk.summary() or {}
    smx = float(peaks.get("sm_max_mhz", 2070.0))
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    # one reciprocal per cell-angle update: the measured reciprocal rate is
    # the sweep's arithmetic ceiling
    mufu_peak = rcp_peak
    sweep_s = tm["sweep_ms"] / 1e3
    upd = tm["cell_angle_updates"]
    achieved = upd / sweep_s if sweep_s > 0 else 0.0
    cells_iter = float(np.sum(info["iterations"].astype(np.float64) * n))
    alg_bytes = 20.0 * cells_iter * args.steps        # 20 B per cell per iteration
    sweep_gbs = alg_bytes / sweep_s / 1e9 if sweep_s > 0 else 0.0
    warm_iters = info["iterations"].astype(np.float64)
    plain_iters = plain_info["iterations"].astype(np.float64)

    cpu = None
    if pool is not None:
        if configs is not None:
            configs = oracle_configs(configs, cfg_raw, pool)
        rate, cores_used, nsol, el = oracle_rate(insts, args.cpu_seconds, pool=pool)
        pool.terminate()
        pool.join()
        cpu = {"value": rate, "unit": UNIT, "cores": cores_used, "kind": "oracle",
               "sample": "%d instances of a random permutation of the batch solved by the "
                         "FP64 oracle (zero guess, tol 1e-6) in %.1f s on %d processes"
                         % (nsol, el, cores_used)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "precision": {"sweep": "f32", "norms": "f64"},
        "data": "synthetic (seeded; paper's samples unpublished)",
        "config": {"workload": WORKLOAD if B == 4096 else
                               "first %d of: %s" % (B, WORKLOAD),
                   "instances_per_gpu": B, "cells_per_gpu": Ctot,
                   "l2": "inputs larger than L2: %.0f MB resident per GPU" %
                         ((Ctot * (3 * 8 + 24)) / 1e6),
                   "warm_start": "DeepONet (128 sensors, 4x128, p=128, BF16) recast, "
                                 "tol %g, itmax %d" % (args.recast_tol, args.recast_itmax)},
        "schedule": "cold: iteration counts estimated from the coefficients, none "
                    "carried over from earlier solves of this batch",
        "warm_start_layout_cached": {
            "value": whole_job_rate(world, B, args.steps, cached_ms / 1e3), "unit": UNIT,
            "ms_per_step": cached_ms / args.steps,
            "note": "the same batch re-solved: the scheduler orders instances by the "
                    "iteration counts of the previous solve of this layout"},
        "autotuner": {"calibration_ms": tune_ms,
                      "plain_sweep_ms_model": model_tm["sweep_ms"] / half,
                      "plain_sweep_ms_tuned": plain_tm["sweep_ms"] / half,
                      "gain_over_model": (model_tm["sweep_ms"] / plain_tm["sweep_ms"]
                                          if plain_tm["sweep_ms"] > 0 else None),
                      "direct_lane_instances": int(tm["last_direct_instances"]),
                      "team_instances": int(tm["last_block_instances"])},
        "plain_guess": {"value": plain_value, "unit": UNIT,
                        "ms_per_step": plain_ms / max(1, args.steps // 2),
                        "iterations_mean": float(np.mean(plain_iters)),
                        "iterations_max": int(np.max(plain_iters))},
        "warm_start": {"iterations_mean": float(np.mean(warm_iters)),
                       "iterations_max": int(np.max(warm_iters)),
                       "recast_iterations": int(info["recast_iterations"]),
                       "operator_ms_per_step": tm["operator_ms"] / args.steps,
                       "sweep_ms_per_step": tm["sweep_ms"] / args.steps,
                       "speedup_vs_plain": value / plain_value if plain_value else None},
        "iteration_accelerators": accel or None,
        "training": None if hist is None else
                    {"samples": 2000, "steps": args.train_steps, "batch": 100,
                     "seconds": train_s, "loss_first": float(hist[0]),
                     "loss_last": float(np.mean(hist[-20:]))},
        "clocks": ck,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(tm["launches"]),
        "roofline": {"bound": "alu", "kernel": "sn1d_kernel<float>", "achieved": achieved,
                     "peak": mufu_peak, "unit": "cell-angle updates/s",
                     "frac": achieved / mufu_peak if mufu_peak else None,
                     "traffic": SWEEP_TRAFFIC_BYTES if B == 4096 else None,
                     "traffic_unit": "bytes per launch (ncu dram read + write)",
                     "peak_source": "measured on this GB300 by nop_measure_alu_peaks: "
                                    "rcp.approx.ftz.f32 rate (one per update); FP32 FMA "
                                    "%.3g/s; %d SMs, nominal 16 rcp/clk/SM x %.0f MHz = %.3g/s"
                                    % (fma_peak, n_sm, smx, n_sm * 16 * smx * 1e6),
                     "sweep_ms_per_step": tm["sweep_ms"] / args.steps,
                     "last_step_trace": {"span_ms": tm["last_span_ms"],
                                         "longest_instance_ms": tm["last_inst_max_ms"],
                                         "mean_instance_ms": tm["last_inst_mean_ms"],
                                         "block_instances": tm["last_block_instances"]},
                     "sweep_algorithmic_gbs": sweep_gbs,
                     "sweep_algorithmic_frac_of_hbm": sweep_gbs / float(peaks.get("hbm_gbs", 6800.0))},
        "cpu_baseline": cpu,
        "configs": None if configs is None else dict(configs, clocks=cfg_clk),
    }
    print(json.dumps(line))
    s.close()
    if world > 1:
        dist.destroy_process_group()


def run_xy_sweep(local):
    """Profiling aid, not the headline: a fixed amount of x-y work (the 256x256
    8-group checkerboard eigenproblem, 2 outer x 5 inner source iterations)
    timed with CUDA events after a warm-up solve; the timed solve is bracketed
    with cudaProfilerStart/Stop.  Prints one JSON line."""
    import torch
    from paper_2509_01416_gb300 import Solver
    torch.cuda.set_device(local)
    c = W.checkerboard_xy_8g()
    bc = tuple(c.bc[f] for f in ("x0", "xL", "y0", "yL"))
    stream = torch.cuda.Stream()
    s = Solver(local)
    s.set_stream(stream.cuda_stream)
    s.set_xy(c.nx, c.ny, c.Lx, c.Ly, c.sigt.reshape(-1), c.sigs.reshape(-1),
             nu_sigma_f=c.nusigf.reshape(-1), chi=c.chi, bc=bc)
    kw = dict(tol=1e-12, tol_k=1e-12, tol_inner=1e-12, itmax=2, itmax_inner=5, check=False)
    s.solve_eigen(**kw)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.set_timing(True)
    torch.cuda.profiler.start()
    ev0.record(stream)
    _, _, info = s.solve_eigen(**kw)
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    tm = s.timing()
    s.set_timing(False)
    ms = ev0.elapsed_time(ev1)
    inner = int(np.max(info["inner"]))
    upd = c.nx * c.ny * 40 * c.sigt.shape[0] * inner
    print(json.dumps({"metric": "x-y sweep cell-direction-group updates per second",
                      "value": upd / (ms / 1e3), "unit": "updates/s", "ms": ms,
                      "sweep_phase_ms": tm["sweep_ms"], "inner_iterations": inner,
                      "outer_iterations": int(info["outer"]), "launches": int(tm["launches"]),
                      "config": {"workload": "checkerboard_xy_8g: 256x256, 8 groups, LS S8"}}))
    s.close()


def run_slab_sweep(local, n):
    """Profiling aid, not the headline: the plain FP32 solve (tol 1e-6, cold
    schedule) of the first n instances of the batch, twice; the first solve
    calibrates the measured schedule (four candidate sweep launches, then the
    solve's own), so the sixth sn1d_kernel launch is the second solve's sweep,
    timed here with CUDA events.  Prints one JSON line."""
    import torch
    from paper_2509_01416_gb300 import Solver
    torch.cuda.set_device(local)
    n_, wdt, order, sigt, sigs, src, _ = W.slab_batch_arrays(rank_instances(0, n))
    stream = torch.cuda.Stream()
    s = Solver(local)
    s.set_stream(stream.cuda_stream)
    s.set_slabs(n_, wdt, order, sigt, sigs, source=src)
    phi = torch.empty(int(n_.sum()), dtype=torch.float64, device="cuda")
    kw = dict(tol=TOL, itmax=200000, precision=0, cold=True)
    s.solve_fixed_source_dev(phi.data_ptr(), **kw)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.set_timing(True)
    ev0.record(stream)
    info = s.solve_fixed_source_dev(phi.data_ptr(), **kw)
    ev1.record(stream)
    torch.cuda.synchronize()
    tm = s.timing()
    s.set_timing(False)
    print(json.dumps({"metric": "slab cell-angle updates per second", "unit": "updates/s",
                      "value": tm["cell_angle_updates"] / (tm["sweep_ms"] / 1e3),
                      "solve_ms": ev0.elapsed_time(ev1), "sweep_ms": tm["sweep_ms"],
                      "iterations": int(np.sum(info["iterations"])),
                      "config": {"workload": "first %d instances of the 4096-slab batch" % n}}))
    s.close()


def run_reference(args, insts, world):
    """The oracle as it stands, on the host cores: each step a bounded sample."""
    cores = os.cpu_count() or 1
    pool = mp.get_context("spawn").Pool(cores)
    per = max(1.0, args.cpu_seconds / 3.0)
    for _ in range(args.warmup):
        oracle_rate(insts, min(per, 2.0), seed=1, pool=pool)
    tot_s, tot_n = 0.0, 0
    for k in range(args.steps):
        rate, _, nsol, el = oracle_rate(insts, per, seed=100 + k, pool=pool)
        tot_s += el
        tot_n += nsol
    pool.terminate()
    pool.join()
    value = tot_n / tot_s if tot_s > 0 else 0.0
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_s / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)",
            "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "per step: instances of a random permutation of the "
                                       "batch solved for %.1f s by the FP64 oracle (zero guess, "
                                       "tol 1e-6; jobs in flight at the deadline finish and "
                                       "count); %d instances over %d steps"
                                       % (per, tot_n, args.steps)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
