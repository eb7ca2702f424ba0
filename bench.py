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
SWEEP_TRAFFIC_BYTES = None
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
    ap.add_argument("--no-dsa", action="store_true",
                    help="skip the diffusion-synthetic-acceleration comparison runs")
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
