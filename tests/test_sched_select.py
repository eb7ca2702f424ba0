"""The slab batch scheduler's team selection (host arithmetic, no GPU):
nop_sched_select_teams decides which instances run on a 12-warp team from
their one-warp and team latencies."""
import ctypes as C

import numpy as np

from paper_2509_01416_gb300 import build as B
from paper_2509_01416_gb300 import capi


def _select(lw, lt, warps, width=12, mode=0, margin=1.0):
    B.build()
    L = capi.lib()
    lw = np.ascontiguousarray(lw, dtype=np.float64)
    lt = np.ascontiguousarray(lt, dtype=np.float64)
    team = np.zeros(len(lw), dtype=np.int32)
    span = C.c_double()
    rc = L.nop_sched_select_teams(len(lw), capi._ptr(lw), capi._ptr(lt), warps, width, mode,
                                  margin, capi._ptr(team, capi._ip), C.byref(span))
    assert rc == 0
    return team.astype(bool), span.value


def test_uniform_batch_needs_no_team():
    # equal instances: every warp latency equals the mean load over the warps
    team, span = _select(np.full(96, 10.0), np.full(96, 2.0), warps=96)
    assert not team.any() and abs(span - 10.0) < 1e-12


def test_one_long_instance_gets_a_team_and_the_span_accounts_for_it():
    lw = np.full(200, 1.0)
    lw[7] = 50.0
    lt = lw / 5.0                       # a team runs 5x faster at 12x the SM time
    team, span = _select(lw, lt, warps=100)
    assert list(np.flatnonzero(team)) == [7]
    # S = (sum of the other warp latencies + 12 x team latency) / warps
    assert abs(span - (199 * 1.0 + 12 * 10.0) / 100) < 1e-12
    assert lw[7] > span                 # the condition that put it on a team holds at S


def test_instances_without_a_team_layout_stay_on_warps():
    lw = np.array([100.0, 100.0, 1.0, 1.0])
    lt = np.array([-1.0, 10.0, 0.1, 0.1])
    team, _ = _select(lw, lt, warps=4)
    assert list(team) == [False, True, False, False]


def test_forced_modes():
    lw, lt = np.array([1.0, 2.0, 3.0]), np.array([0.5, -1.0, 1.0])
    assert list(_select(lw, lt, warps=3, mode=1)[0]) == [True, False, True]
    assert not _select(lw, lt, warps=3, mode=2)[0].any()


def test_no_warp_instance_outlasts_the_span_and_teams_are_the_longest():
    # random batches: no instance left on a warp outlasts the final span, and
    # every team instance is longer on a warp than every warp instance
    rng = np.random.default_rng(5)
    for _ in range(20):
        lw = rng.lognormal(0.0, 1.0, 500)
        lt = lw / rng.uniform(3, 8, 500)
        team, span = _select(lw, lt, warps=150)
        assert np.all(lw[~team] <= span * (1 + 1e-12))
        if team.any():
            assert lw[team].min() >= lw[~team].max()


def test_margin_leaves_no_warp_instance_near_the_span():
    # with margin m, an instance stays on a warp only while m x its latency is
    # within the span, so every warp instance ends by span / m
    rng = np.random.default_rng(7)
    for _ in range(10):
        lw = rng.lognormal(0.0, 1.0, 500)
        lt = lw / rng.uniform(3, 8, 500)
        t1, s1 = _select(lw, lt, warps=150, margin=1.0)
        t2, s2 = _select(lw, lt, warps=150, margin=1.25)
        assert np.all(1.25 * lw[~t2] <= s2 * (1 + 1e-12))
        assert t2.sum() >= t1.sum() and np.all(t2[t1])


def test_margin_below_one_is_rejected():
    B.build()
    L = capi.lib()
    lw = np.ones(3)
    team = np.zeros(3, dtype=np.int32)
    rc = L.nop_sched_select_teams(3, capi._ptr(lw), capi._ptr(lw), 3, 12, 0, 0.9,
                                  capi._ptr(team, capi._ip), None)
    assert rc != 0
