"""The column-grouping planner behind PR_GROUP_AUTO (host logic, no GPU):
its minimum is checked against brute force over every set partition of the
columns, and its choices against cases whose answer is plain."""
import itertools
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def B():
    from paper_2108_02997_gb300 import binding
    binding.lib()
    return binding


def _width(m, us):
    for k in range(6):
        if (1 << k) >= m and us[k] > 0:
            return k
    return None


def _set_partitions(items):
    if not items:
        yield []
        return
    first, rest = items[0], items[1:]
    for part in _set_partitions(rest):
        for i in range(len(part)):
            yield part[:i] + [[first] + part[i]] + part[i + 1:]
        yield [[first]] + part


def _brute_force(iters, us):
    best = math.inf
    for part in _set_partitions(list(range(len(iters)))):
        cost = 0.0
        for grp in part:
            k = _width(len(grp), us)
            if k is None:
                cost = math.inf
                break
            cost += max(iters[c] for c in grp) * us[k]
        best = min(best, cost)
    return best


def _plan_cost(iters, us, job, wid):
    cost = 0.0
    for j in set(job.tolist()):
        members = [c for c in range(len(iters)) if job[c] == j]
        w = {int(wid[c]) for c in members}
        assert len(w) == 1 and len(members) <= w.pop() <= 32
        k = _width(len(members), us)
        assert wid[members[0]] >= 1 << k and us[int(math.log2(wid[members[0]]))] > 0
        cost += max(iters[c] for c in members) * us[int(math.log2(wid[members[0]]))]
    return cost


def test_minimum_equals_brute_force(B):
    rng = np.random.default_rng(7)
    for trial in range(40):
        n = int(rng.integers(1, 8))
        iters = rng.integers(1, 400, size=n).astype(float)
        us = np.sort(rng.uniform(1.0, 100.0, size=6))
        if trial % 3 == 1:
            us[rng.integers(1, 6)] = -1.0      # a width that could not be timed
        job, wid, cost = B.plan_columns(iters, us)
        want = _brute_force(list(iters), list(us))
        assert cost == pytest.approx(want, rel=1e-12), (iters, us)
        assert _plan_cost(list(iters), list(us), job, wid) == pytest.approx(cost, rel=1e-12)


def test_flat_launch_times_pack_everything(B):
    # launch time independent of width (a small graph): one job holds all
    iters = [30, 200, 45, 500, 12, 90, 90, 7, 33, 61]
    job, wid, cost = B.plan_columns(iters, [10.0] * 6)
    assert len(set(job.tolist())) == 1 and set(wid.tolist()) == {16}
    assert cost == pytest.approx(500 * 10.0)


def test_launch_time_proportional_to_width_keeps_columns_apart(B):
    # no saving from sharing the index stream: every column alone
    iters = [30, 200, 45, 500, 12]
    job, wid, cost = B.plan_columns(iters, [5.0 * (1 << k) for k in range(6)])
    assert len(set(job.tolist())) == 5 and set(wid.tolist()) == {1}
    assert cost == pytest.approx(5.0 * sum(iters))


def test_jobs_follow_iteration_order(B):
    # equal iteration counts belong together; jobs are numbered from the longest
    iters = [100, 10, 100, 10, 100, 10, 100, 10]
    us = [10.0, 11.0, 12.0, 30.0, 60.0, 120.0]
    job, wid, cost = B.plan_columns(iters, us)
    assert cost == pytest.approx(100 * 12.0 + 10 * 12.0)
    assert {int(job[c]) for c in (0, 2, 4, 6)} == {0} and {int(job[c]) for c in (1, 3, 5, 7)} == {1}
    assert set(wid.tolist()) == {4}


def test_more_than_32_columns(B):
    iters = [50.0] * 70
    job, wid, cost = B.plan_columns(iters, [10.0] * 6)
    sizes = sorted(np.bincount(job).tolist())
    assert sum(sizes) == 70 and max(sizes) <= 32 and len(sizes) == 3
    assert cost == pytest.approx(3 * 50 * 10.0)


def test_rejects_bad_arguments(B):
    with pytest.raises(B.PageRankError):
        B.plan_columns([10.0, 0.0], [1.0] * 6)
    with pytest.raises(B.PageRankError):
        B.plan_columns([10.0], [0.0, 1.0, 1.0, 1.0, 1.0, 1.0])
    with pytest.raises(B.PageRankError):
        B.plan_columns([float("nan")], [1.0] * 6)
    job, wid, cost = B.plan_columns([], [1.0] * 6)
    assert job.size == 0 and cost == 0.0


# ---- shared launch latency (jobs of one width share each launch)

def _shared_cost(iters, us, lat, job, wid):
    """Independent restatement of the model: every width used pays the latency
    once for its longest job; every job pays its iterations times its width's
    launch time less the latency (at least 5 % of the launch time)."""
    by_job = {}
    for c, j in enumerate(job.tolist()):
        by_job.setdefault(j, []).append(c)
    width_max = {}
    cost = 0.0
    for j, members in by_job.items():
        w = int(wid[members[0]])
        k = int(math.log2(w))
        m = max(iters[c] for c in members)
        cost += m * max(us[k] - lat, 0.05 * us[k])
        width_max[k] = max(width_max.get(k, 0.0), m)
    return cost + lat * sum(width_max.values())


def _singles(n):
    return np.arange(n, dtype=np.int32), np.ones(n, np.int32)


@pytest.mark.parametrize("seed", range(6))
def test_shared_plan_is_cheapest_candidate(B, seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 12))
    iters = rng.integers(5, 80, size=n).astype(np.float64)
    base = float(rng.uniform(10, 300))
    us = np.array([base * (1 + g) for g in np.cumsum(rng.uniform(0.05, 1.0, size=6)) - rng.uniform(0.05, 1.0)])
    us = np.maximum(us, base)
    lat = float(rng.uniform(0.0, 0.9)) * us[0]
    job, wid, cost = B.plan_columns_shared(iters, us, lat)
    assert math.isclose(cost, _shared_cost(iters, us, lat, job, wid), rel_tol=1e-12)
    # never worse than the whole-launch-time plan or one job per column
    j0, w0, _ = B.plan_columns(iters, us)
    assert cost <= _shared_cost(iters, us, lat, j0, w0) * (1 + 1e-12)
    js, ws = _singles(n)
    assert cost <= _shared_cost(iters, us, lat, js, ws) * (1 + 1e-12)
    # every job fits its width
    for j in set(job.tolist()):
        members = [c for c in range(n) if job[c] == j]
        assert len(members) <= int(wid[members[0]]) <= 32


def test_shared_plan_latency_bound_small_graph(B):
    """Eleven equal columns on a small graph: a launch is almost all latency,
    so eleven single-column jobs sharing one launch beat packing them."""
    iters = np.full(11, 20.0)
    us = np.array([30.0, 45.0, 70.0, 120.0, 220.0, 420.0])
    job, wid, cost = B.plan_columns_shared(iters, us, 28.0)
    assert (wid == 1).all() and len(set(job.tolist())) == 11
    assert math.isclose(cost, 20.0 * 28.0 + 11 * 20.0 * 2.0)
    # the whole-launch-time plan packs them
    j0, w0, _ = B.plan_columns(iters, us)
    assert (w0 > 1).any()


def test_shared_plan_without_latency_is_the_plain_plan(B):
    iters = np.array([40.0, 39.0, 12.0, 11.0, 10.0])
    us = np.array([100.0, 150.0, 260.0, 500.0, 990.0, 1990.0])
    j1, w1, _ = B.plan_columns_shared(iters, us, 0.0)
    j0, w0, _ = B.plan_columns(iters, us)
    assert (j1 == j0).all() and (w1 == w0).all()
    with pytest.raises(Exception):
        B.plan_columns_shared(iters, us, -1.0)
