"""The bench's multi-rank path on CPU: two gloo ranks on 127.0.0.1.

Instances are independent, so ranks shard the work (each its own seeded
batch) and exchange nothing but the MAX of their elapsed times.  This checks
the sharding (no shared instances), the max-over-ranks reduction that the
bench's timing uses and the whole-job rate built from it.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as tmp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        insts = bench.rank_instances(rank, limit=6)
        sig = [(s.I, s.N, float(s.sigt[0]), float(s.Q.sum())) for s in insts]
        elapsed = 0.5 + rank            # rank 1 is the slow one
        t = bench.max_over_ranks(elapsed, world, "cpu")
        rate = bench.whole_job_rate(world, len(insts), 3, t)
        out[rank] = (sig, t, rate)
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_ranks_shard_and_reduce():
    world = 2
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    s0, t0, r0 = out[0]
    s1, t1, r1 = out[1]
    # every rank sees the slowest rank's time
    assert t0 == t1 == 1.5
    # whole-job rate: all ranks' units over the slowest time
    assert r0 == pytest.approx(world * 6 * 3 / 1.5)
    # the two shards are different batches
    assert not set(s0) & set(s1)


def test_rank_batches_are_prefix_stable():
    import bench
    a = bench.rank_instances(0, limit=5)
    b = bench.rank_instances(0, limit=9)
    for x, y in zip(a, b):
        assert x.I == y.I and x.N == y.N
        assert np.array_equal(x.sigt, y.sigt) and np.array_equal(x.Q, y.Q)


@pytest.mark.timeout(300)
def test_oracle_sample_leaves_no_work_queued():
    # a timed oracle sample must not leave jobs in the pool for the next one
    import multiprocessing as mp
    import time
    import bench
    import workloads as W
    insts = [W.slab_instance(np.random.default_rng(b), 200, 16) for b in range(600)]
    pool = mp.get_context("spawn").Pool(2)
    try:
        bench.oracle_rate(insts[:4], 5.0, pool=pool)       # start the workers
        # a short sample over the whole list (many seconds of work)...
        bench.oracle_rate(insts, 0.05, seed=1, pool=pool)
        # ...must not delay the next sample: it solves instances at once
        t0 = time.perf_counter()
        _, _, n2, el = bench.oracle_rate(insts, 1.0, seed=2, pool=pool)
        assert n2 > 0 and el < 1.0 + 5.0
        assert time.perf_counter() - t0 < 10.0
    finally:
        pool.terminate()
        pool.join()


def test_clock_summary_keeps_the_timed_window(tmp_path):
    import datetime
    import bench
    base = datetime.datetime(2026, 1, 2, 3, 4, 5)
    rows = []
    for k, (mhz, slow) in enumerate([(1200, "Not Active"), (2070, "Not Active"),
                                     (2055, "Active"), (2070, "Not Active"), (990, "Not Active")]):
        ts = (base + datetime.timedelta(milliseconds=100 * k)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        rows.append("%s, 0, %d, 2070, 900.00, 0x0000000000000000, Not Active, Not Active, "
                    "%s, Not Active" % (ts, mhz, slow))
    f = tmp_path / "clocks.csv"
    f.write_text("\n".join(rows) + "\n")
    c = bench.Clocks(0, str(f))
    c.t0 = (base + datetime.timedelta(milliseconds=100)).timestamp()
    c.t1 = (base + datetime.timedelta(milliseconds=300)).timestamp()
    s = c.summary()
    assert s["samples"] == 3 and s["window"] == "timed warm-start region"
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_thermal_slowdown"]
    # without a window every sample counts
    c.t0 = c.t1 = None
    s = c.summary()
    assert s["samples"] == 5 and s["sm_mhz"] == 2055.0
