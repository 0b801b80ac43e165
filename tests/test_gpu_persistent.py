"""Persistent passes (PR_LOOP_PERSISTENT): Section 2's iteration run inside one
cooperative launch, every CTA of a job waiting on the job's device counter for
the others and taking the job's stopping decisions itself. The passes do the
same arithmetic in the same order as the CUDA-graph loop, so every result is
bit-identical to it (and so to the oracle within the FP64 parity bound);
solves whose passes are split fall back to the graph loop; a wait that never
ends ends the solve with PR_ETIMEOUT instead of hanging, and the context stays
usable."""
import numpy as np
import pytest

from tests.parity import assert_fp64_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2108_02997_gb300 import binding
    binding.lib()
    return binding


@pytest.fixture(scope="module")
def er(gg):
    return gg.erdos_renyi_10k(seed=1)


@pytest.fixture(scope="module")
def er_dev(B, er):
    return B.Graph.from_csr(er)


def _loops(B):
    return B.pr_last_solve_stats()["loop_phases"]


def _same(a, b, what):
    """Two prepared batches solved over the same instances: equal bit for bit."""
    assert np.array_equal(a["iters"], b["iters"]), what
    assert np.array_equal(a["err"], b["err"]), what
    assert np.array_equal(a["err_l1"], b["err_l1"]), what
    assert np.array_equal(a["converged"], b["converged"]), what
    for k, (x, y) in enumerate(zip(a["out"], b["out"])):
        assert np.array_equal(x, y), f"{what}: instance {k} ranks differ"


def _run(B, insts, **kw):
    pb = B.PreparedBatch(insts)
    pb.solve(**kw)
    return {"iters": pb.iters.copy(), "err": pb.err.copy(), "err_l1": pb.err_l1.copy(),
            "converged": pb.converged.copy(), "out": [x.out.copy() for x in insts]}, _loops(B)


def test_single_solve_equals_graph_and_host_loops(B, orc, er, er_dev):
    res = {}
    for loop in ("persistent", "graph", "host"):
        res[loop] = B.pr_solve(er_dev, 0.85, 1e-10, 1, 500, loop=loop, kernels="fused")
        lp = _loops(B)
        assert lp[loop] == 1 and sum(lp.values()) == 1, (loop, lp)
    p, g, h = res["persistent"], res["graph"], res["host"]
    assert p.iters == g.iters == h.iters and p.err == g.err == h.err
    assert np.array_equal(p.ranks, g.ranks) and np.array_equal(p.ranks, h.ranks)
    st = B.pr_solve(er_dev, 0.85, 1e-10, 1, 500, loop="persistent", kernels="fused")
    stats = B.pr_last_solve_stats()
    assert stats["launches"] == 2 and stats["passes"] == p.iters + 1   # init + one cooperative launch
    ref = orc.pagerank(er, 0.85, 1e-10, 1, 500, history=True)
    assert_fp64_parity(st.ranks, st.iters, st.err, ref, 1e-10, 1, "persistent")


def test_default_loop_is_persistent_where_it_applies(B, er_dev):
    B.pr_solve(er_dev, 0.85, 1e-8, 1, 500)
    assert _loops(B) == {"graph": 0, "host": 0, "persistent": 1}
    # split passes (a gather and an update kernel) keep the graph loop
    B.pr_solve(er_dev, 0.85, 1e-8, 1, 500, loop="persistent", kernels="split")
    assert _loops(B) == {"graph": 1, "host": 0, "persistent": 0}


@pytest.mark.parametrize("group", ["single", "pack"])
@pytest.mark.parametrize("precision", ["df64", "fp64", "fp32", "mixed"])
def test_sweep_equals_graph_loop(B, er_dev, precision, group):
    """The alpha x tau x norm sweep on shared trajectories (stopping rules
    firing at different passes, answers copied out while the other columns go
    on), as eleven one-column jobs or as one job of all eleven columns (seven
    taus: 231 rules, within the 256 a job may hold): persistent and graph loops
    with the same jobs give the same bits; mixed precision runs both of its
    phases persistent."""
    alphas = [round(0.5 + 0.05 * i, 2) for i in range(11)]
    nt = 10 if group == "single" else 7
    taus = [10.0 ** -k for k in range(1, nt + 1)] if precision != "fp32" else [10.0 ** -k for k in range(1, 6)]

    def insts():
        return [B.Instance(er_dev, a, t, nm, 500) for a in alphas for t in taus for nm in (1, 2, 3)]
    p, lp = _run(B, insts(), loop="persistent", precision=precision, group=group)
    assert lp["persistent"] == (2 if precision == "mixed" else 1) and lp["graph"] == 0, lp
    g, lg = _run(B, insts(), loop="graph", precision=precision, group=group)
    assert lg["persistent"] == 0 and lg["graph"] >= 1, lg
    _same(p, g, f"sweep {precision} {group}")
    assert p["converged"].all()


def test_planner_takes_one_column_jobs_for_small_persistent_sweeps(B, er_dev):
    """With persistent passes, the planner gives each column of a small
    graph a job of its own (PR_GROUP_AUTO): the same bits as explicit
    one-column jobs."""
    alphas = [round(0.5 + 0.05 * i, 2) for i in range(11)]

    def insts():
        return [B.Instance(er_dev, a, t, nm, 500) for a in alphas for t in (1e-4, 1e-10) for nm in (1, 3)]
    a, la = _run(B, insts(), group="auto")
    s, _ = _run(B, insts(), group="single", loop="persistent")
    assert la["persistent"] == 1
    _same(a, s, "auto vs single")


@pytest.mark.parametrize("precision", ["df64", "fp32"])
def test_many_graphs_and_adversarial_rows(B, gg, precision):
    """Several graphs in one launch (one job each, finishing at different
    passes: a finished job's CTAs leave while the others go on) with rows of every
    tile kind, including rows cut into chunks whose partial sums meet through
    counters that every pass resets; edgeless and single-vertex graphs."""
    from tests.test_gpu_parity import adversarial
    gs = adversarial(gg)
    dgs = [B.Graph.from_csr(g) for g in gs.values()]
    try:
        tau = 1e-10 if precision != "fp32" else 1e-5

        def insts():
            return [B.Instance(dg, a, tau, nm, 500) for dg in dgs for a in (0.6, 0.85, 0.99) for nm in (1, 3)]
        p, lp = _run(B, insts(), loop="persistent", precision=precision, kernels="fused", group="pack")
        assert lp["persistent"] >= 1 and lp["graph"] == 0, lp
        g, _ = _run(B, insts(), loop="graph", precision=precision, kernels="fused", group="pack")
        _same(p, g, f"adversarial {precision}")
    finally:
        for dg in dgs:
            dg.close()


def test_pass_cap_ends_a_persistent_solve(B, orc, er, er_dev):
    """The watchdog's pass budget stops persistent passes like the other loops
    (PR_ETIMEOUT, the context stays usable)."""
    x = B.Instance(er_dev, 0.99, 1e-14, 1, 500)
    st = B.pr_solve_batch([x], loop="persistent", max_passes=5, check=False)
    assert st == B.PR_ETIMEOUT and x.status == B.PR_ETIMEOUT
    assert b"pass cap" in B.lib().pr_last_error()
    ref = orc.pagerank(er, 0.85, 1e-10, 1, 500, history=True)
    res = B.pr_solve(er_dev, 0.85, 1e-10, 1, 500, loop="persistent")
    assert_fp64_parity(res.ranks, res.iters, res.err, ref, 1e-10, 1, "after the pass cap")


def test_a_wait_that_runs_out_ends_the_solve(B, orc, er, er_dev):
    """With the arrivals held back (the test hook), every CTA's wait runs out
    after persist_wait_us of device time: the solve returns PR_ETIMEOUT, and
    the next solve on the same context is correct."""
    x = B.Instance(er_dev, 0.85, 1e-10, 1, 500)
    B.hold_decisions(True)
    try:
        st = B.pr_solve_batch([x], loop="persistent", persist_wait_us=20000, check=False)
    finally:
        B.hold_decisions(False)
    assert st == B.PR_ETIMEOUT and x.status == B.PR_ETIMEOUT
    assert b"waited too long" in B.lib().pr_last_error()
    ref = orc.pagerank(er, 0.85, 1e-10, 1, 500, history=True)
    res = B.pr_solve(er_dev, 0.85, 1e-10, 1, 500, loop="persistent")
    assert_fp64_parity(res.ranks, res.iters, res.err, ref, 1e-10, 1, "after a wait ran out")
