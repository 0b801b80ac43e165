"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by
element, on seeded inputs spanning several work units and ragged tails, plus
the degenerate graphs of the method."""
import numpy as np
import pytest

from tests.parity import assert_fp64_parity, rel_l1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2108_02997_gb300 import binding
    binding.lib()
    return binding


@pytest.fixture(scope="module")
def er10k(gg):
    return gg.erdos_renyi_10k(seed=1)


@pytest.fixture(scope="module")
def er10k_dev(B, er10k):
    return B.Graph.from_csr(er10k)


def adversarial(gg):
    n = 3000
    out = {}
    # one hub with in-degree n-1 (split across CTAs) and dangling leaves
    out["hub"] = gg.from_edges(n, list(range(1, n)), [0] * (n - 1))
    # everything dangling (no edges)
    out["edgeless"] = gg.from_edges(n, [], [])
    out["single"] = gg.from_edges(1, [], [])
    out["pair"] = gg.from_edges(2, [0], [1])
    # isolated vertices + rows straddling each lane-group threshold (in-degrees 1..70, 500..520, 2040..2060)
    src, dst = [], []
    rng = np.random.default_rng(3)
    v = 0
    for d in list(range(1, 71)) + list(range(500, 521)) + list(range(2040, 2061)) + [5000, 9000]:
        s = rng.choice(np.arange(20000), size=d, replace=False)
        src += list(s)
        dst += [20000 + v] * d
        v += 1
    out["thresholds"] = gg.from_edges(20000 + v + 500, src, dst)
    out["cycle"] = gg.from_edges(1000, list(range(1000)), [(i + 1) % 1000 for i in range(1000)])
    return out


@pytest.mark.parametrize("kernels", ["fused", "split"])
@pytest.mark.parametrize("precision", ["df64", "fp64"])
def test_er10k_plain_matches_oracle(B, orc, er10k, er10k_dev, precision, kernels):
    ref = orc.pagerank(er10k, 0.85, 1e-10, 1, 500, history=True)
    res = B.pr_solve(er10k_dev, 0.85, 1e-10, 1, 500, precision=precision, history=True, kernels=kernels)
    assert_fp64_parity(res.ranks, res.iters, res.err, ref, 1e-10, 1, f"er10k {precision}")
    assert res.converged == ref.converged
    # per-iteration norms follow the oracle's within the bound that the rank
    # tolerance implies (see tests/parity.py)
    h = res.err_history
    k = min(len(h), len(ref.err_hist))
    assert np.abs(h[:k] - ref.err_hist[:k]).max() <= 2e-12


@pytest.mark.parametrize("norm", [1, 2, 3])
@pytest.mark.parametrize("tau", [1e-3, 1e-6, 1e-9])
def test_er10k_norms_and_tolerances(B, orc, er10k, er10k_dev, norm, tau):
    ref = orc.pagerank(er10k, 0.85, tau, norm, 500, history=True)
    res = B.pr_solve(er10k_dev, 0.85, tau, norm, 500)
    assert_fp64_parity(res.ranks, res.iters, res.err, ref, tau, norm, f"norm {norm} tau {tau}")


@pytest.mark.parametrize("alpha", [0.0, 0.5, 0.95, 1.0])
def test_er10k_alpha_extremes(B, orc, er10k, er10k_dev, alpha):
    ref = orc.pagerank(er10k, alpha, 1e-9, 1, 500, history=True)
    res = B.pr_solve(er10k_dev, alpha, 1e-9, 1, 500)
    assert_fp64_parity(res.ranks, res.iters, res.err, ref, 1e-9, 1, f"alpha {alpha}")


@pytest.mark.parametrize("kernels", ["fused", "split"])
def test_adversarial_graphs(B, orc, gg, kernels):
    for name, g in adversarial(gg).items():
        dg = B.Graph.from_csr(g)
        for norm in (1, 3):
            for prec in ("df64", "fp64"):
                ref = orc.pagerank(g, 0.85, 1e-10, norm, 500, history=True)
                res = B.pr_solve(dg, 0.85, 1e-10, norm, 500, precision=prec, kernels=kernels)
                assert_fp64_parity(res.ranks, res.iters, res.err, ref, 1e-10, norm,
                                   f"{name} {prec} norm {norm} {kernels}")
        dg.close()


def test_cap_reached(B, orc, er10k, er10k_dev):
    ref = orc.pagerank(er10k, 0.99, 1e-14, 1, 25, history=True)
    res = B.pr_solve(er10k_dev, 0.99, 1e-14, 1, 25)
    assert res.iters == 25 and not res.converged and not ref.converged
    assert rel_l1(res.ranks, ref.ranks) <= 1e-12


def test_host_loop_equals_graph_loop(B, er10k_dev):
    a = B.pr_solve(er10k_dev, 0.85, 1e-10, 2, 500, loop="graph")
    b = B.pr_solve(er10k_dev, 0.85, 1e-10, 2, 500, loop="host")
    assert a.iters == b.iters and np.array_equal(a.ranks, b.ranks) and a.err == b.err
    st = B.pr_last_solve_stats()
    # init + one pass per update + the pass that copies the answer out; a pass
    # is one kernel, or two (gather + update) for one column
    assert st["passes"] == b.iters + 1 and st["kernel_ms"] > 0
    assert st["launches"] in (1 + st["passes"], 1 + 2 * st["passes"])


def test_user_start_vector(B, orc, er10k, er10k_dev):
    rng = np.random.default_rng(5)
    r0 = rng.random(er10k.n)
    r0 /= r0.sum()
    ref = orc.pagerank(er10k, 0.85, 1e-10, 1, 500, init=r0, history=True)
    res = B.pr_solve(er10k_dev, 0.85, 1e-10, 1, 500, init=r0)
    assert_fp64_parity(res.ranks, res.iters, res.err, ref, 1e-10, 1, "user start")


def test_device_buffers(B, orc, er10k, er10k_dev):
    import torch
    out = torch.empty(er10k.n, dtype=torch.float64, device="cuda")
    r0 = torch.full((er10k.n,), 1.0 / er10k.n, dtype=torch.float64, device="cuda")
    res = B.pr_solve(er10k_dev, 0.85, 1e-10, 1, 500, out=out, init=r0)
    ref = orc.pagerank(er10k, 0.85, 1e-10, 1, 500, history=True)
    assert_fp64_parity(out.cpu().numpy(), res.iters, res.err, ref, 1e-10, 1, "device buffers")


@pytest.mark.parametrize("kernels", ["fused", "split"])
@pytest.mark.parametrize("scale", [14, 17])
def test_rmat_matches_oracle(B, orc, gg, scale, kernels):
    g = gg.rmat(scale, 16, seed=scale)
    dg = B.Graph.from_csr(g)
    for norm, tau in ((1, 1e-10), (2, 1e-8), (3, 1e-10)):
        ref = orc.pagerank(g, 0.85, tau, norm, 500, history=True, threads=orc.default_threads())
        res = B.pr_solve(dg, 0.85, tau, norm, 500, kernels=kernels)
        assert_fp64_parity(res.ranks, res.iters, res.err, ref, tau, norm, f"rmat{scale} norm {norm} {kernels}")
    dg.close()


def test_device_side_graph_validation(B):
    """Per-edge checks of pr_graph_create run on the device: an out-of-range
    source and out-degrees that disagree with the sources (same total) are
    rejected with PR_EINVAL and no handle."""
    with pytest.raises(B.PageRankError) as ei:
        B.Graph([0, 1, 2], [0, 5], [2, 0])
    assert ei.value.status == B.PR_EINVAL and "out of range" in str(ei.value)
    with pytest.raises(B.PageRankError) as ei:
        B.Graph([0, 1, 2], [0, 0], [1, 1])
    assert ei.value.status == B.PR_EINVAL and "does not match" in str(ei.value)
    g = B.Graph([0, 1, 2], [1, 0], [1, 1])   # the valid 2-cycle still works afterwards
    assert g.info() == (2, 2, 0)
    g.close()


@pytest.mark.parametrize("loop", ["graph", "host"])
def test_watchdog_ends_the_device_loop(B, orc, er10k, er10k_dev, loop):
    """A device loop that outlives its pass budget stops itself and reports
    PR_ETIMEOUT; the context stays usable (no GPU fault is involved)."""
    x = B.Instance(er10k_dev, 0.99, 1e-14, 1, 500)
    st = B.pr_solve_batch([x], loop=loop, max_passes=5, check=False)
    assert st == B.PR_ETIMEOUT and x.status == B.PR_ETIMEOUT
    assert b"pass cap" in B.lib().pr_last_error()
    ref = orc.pagerank(er10k, 0.85, 1e-10, 1, 500, history=True)
    res = B.pr_solve(er10k_dev, 0.85, 1e-10, 1, 500, loop=loop)
    assert_fp64_parity(res.ranks, res.iters, res.err, ref, 1e-10, 1, f"after watchdog ({loop})")


def test_road_grid_matches_oracle(B, orc, gg):
    """A road-like lattice (in-degrees 0..4, many dangling-free short rows):
    every row is in a small-degree class."""
    g = gg.road_grid(300, 400, seed=11)
    with B.Graph.from_csr(g) as dg:
        for norm, tau in ((1, 1e-10), (2, 1e-9), (3, 1e-7)):
            ref = orc.pagerank(g, 0.85, tau, norm, 500, history=True, threads=orc.default_threads())
            res = B.pr_solve(dg, 0.85, tau, norm, 500)
            assert_fp64_parity(res.ranks, res.iters, res.err, ref, tau, norm, f"road norm {norm}")


def test_kernel_occupancy_and_split_times(B, er10k_dev):
    """pr_kernel_occupancy reports resident CTAs for every width; a split
    host-loop solve reports its gather and update kernel times, which add up
    to the pass time."""
    for prec in ("df64", "fp64", "fp32"):
        for w in (1, 2, 4, 8, 16, 32):
            assert 1 <= B.kernel_occupancy(prec, w) <= 8
    with pytest.raises(B.PageRankError):
        B.kernel_occupancy("df64", 3)
    with pytest.raises(B.PageRankError):
        B.kernel_occupancy("mixed", 1)
    B.pr_solve(er10k_dev, 0.85, 1e-10, 1, 500, loop="host", kernels="split")
    st = B.pr_last_solve_stats()
    assert st["gather_ms"] > 0 and st["update_ms"] > 0
    assert abs(st["gather_ms"] + st["update_ms"] - st["kernel_ms"]) <= 1e-6 * max(1.0, st["kernel_ms"])
    B.pr_solve(er10k_dev, 0.85, 1e-10, 1, 500, loop="host", kernels="fused")
    st = B.pr_last_solve_stats()
    assert st["gather_ms"] == 0 and st["update_ms"] == 0 and st["kernel_ms"] > 0
