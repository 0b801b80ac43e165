"""GPU parity of the batched paths: the alpha x tau x norm sweep (Sections 2-4)
as one batch, with and without shared trajectories; many graphs in one batch;
mixed precision and FP32 against the error bound of the L1 contraction."""
import numpy as np
import pytest

from tests.parity import assert_bound_parity, assert_fp64_parity, previous_iterates, rel_l1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2108_02997_gb300 import binding
    binding.lib()
    return binding


@pytest.fixture(scope="module")
def er(gg):
    return gg.erdos_renyi_10k(seed=1)


def _sweep_specs(alphas, taus):
    return [(a, t, nm) for a in alphas for t in taus for nm in (1, 2, 3)]


def _oracle_sweep(orc, g, specs, max_iter=500):
    out = {}
    for a in sorted({s[0] for s in specs}):
        mine = [s for s in specs if s[0] == a]
        res = orc.pagerank_taps(g, a, [(t, nm, max_iter) for _, t, nm in mine])
        for s, r in zip(mine, res):
            out[s] = r
    return out


@pytest.mark.parametrize("share", [True, False])
def test_sweep_matches_oracle(B, orc, er, share):
    specs = _sweep_specs([0.5, 0.85, 1.0], [1e-2, 1e-6, 1e-10])
    ref = _oracle_sweep(orc, er, specs)
    with B.Graph.from_csr(er) as dg:
        insts = [B.Instance(dg, a, t, nm, 500) for a, t, nm in specs]
        B.pr_solve_batch(insts, share=share)
        for (a, t, nm), x in zip(specs, insts):
            assert x.status == 0
            assert_fp64_parity(x.out, x.iters, x.err, ref[(a, t, nm)], t, nm, f"alpha {a} tau {t} norm {nm} share {share}")


def test_sweep_device_outputs_with_aliases(B, orc, er):
    """Outputs in device memory: rules that fire on the same iterate as an
    earlier one (equal tau, or a loose tau in every norm) receive their answer
    by the batched alias copy; every output is checked."""
    import torch
    specs = _sweep_specs([0.6, 0.85], [1e-1, 1e-2, 1e-8]) + [(0.85, 1e-8, 1), (0.85, 1e-8, 3)]
    ref = _oracle_sweep(orc, er, specs)
    with B.Graph.from_csr(er) as dg:
        outs = [torch.full((er.n,), -1.0, dtype=torch.float64, device="cuda") for _ in specs]
        insts = [B.Instance(dg, a, t, nm, 500, out=o) for (a, t, nm), o in zip(specs, outs)]
        B.pr_solve_batch(insts, outputs_on_device=True)
        torch.cuda.synchronize()
        for (a, t, nm), x, o in zip(specs, insts, outs):
            assert x.status == 0
            assert_fp64_parity(o.cpu().numpy(), x.iters, x.err, ref[(a, t, nm)], t, nm, f"alpha {a} tau {t} norm {nm}")


def test_full_330_sweep(B, orc, er):
    """The paper's alpha sweep (0.50..1.00 step .05) x tau 1e-1..1e-10 x three
    norms: 330 instances in one call, cap 500."""
    alphas = [round(0.5 + 0.05 * i, 2) for i in range(11)]
    specs = _sweep_specs(alphas, [10.0 ** -k for k in range(1, 11)])
    ref = _oracle_sweep(orc, er, specs)
    with B.Graph.from_csr(er) as dg:
        insts = [B.Instance(dg, a, t, nm, 500) for a, t, nm in specs]
        B.pr_solve_batch(insts)
        for (a, t, nm), x in zip(specs, insts):
            assert_fp64_parity(x.out, x.iters, x.err, ref[(a, t, nm)], t, nm, f"alpha {a} tau {t} norm {nm}")
        # the paper's trends (Sections 2-4) hold on this graph
        it = {s: x.iters for s, x in zip(specs, insts)}
        for a in alphas:
            for t in [10.0 ** -k for k in range(1, 11)]:
                assert it[(a, t, 3)] <= it[(a, t, 2)] <= it[(a, t, 1)]


def test_many_graphs_one_batch(B, orc, gg):
    graphs = [gg.rmat(9 + (i % 5), 16, seed=500 + i) for i in range(10)]
    dgs = [B.Graph.from_csr(g) for g in graphs]
    insts = [B.Instance(d, 0.85, 1e-10, 1, 500) for d in dgs]
    B.pr_solve_batch(insts)
    for g, x in zip(graphs, insts):
        ref = orc.pagerank(g, 0.85, 1e-10, 1, 500, history=True)
        assert_fp64_parity(x.out, x.iters, x.err, ref, 1e-10, 1, g.name)
    for d in dgs:
        d.close()


def test_mixed_graphs_and_columns(B, orc, gg):
    g1 = gg.rmat(12, 16, seed=31)
    g2 = gg.erdos_renyi(3000, 20000, 100, 32)
    d1, d2 = B.Graph.from_csr(g1), B.Graph.from_csr(g2)
    specs = [(d1, g1, 0.7, 1e-8, 2), (d2, g2, 0.9, 1e-9, 1), (d1, g1, 0.85, 1e-7, 3), (d2, g2, 0.6, 1e-6, 3)]
    insts = [B.Instance(d, a, t, nm, 500) for d, _, a, t, nm in specs]
    B.pr_solve_batch(insts)
    for (d, g, a, t, nm), x in zip(specs, insts):
        ref = orc.pagerank(g, a, t, nm, 500, history=True)
        assert_fp64_parity(x.out, x.iters, x.err, ref, t, nm, f"{g.name} alpha {a}")
    d1.close(); d2.close()


@pytest.mark.parametrize("alpha", [0.85, 0.95])
def test_mixed_precision_error_bound(B, orc, gg, alpha):
    g = gg.rmat(16, 16, seed=24)
    ref = orc.pagerank(g, alpha, 1e-13, 1, 10000, threads=orc.default_threads())
    with B.Graph.from_csr(g) as dg:
        specs = [(t, nm) for t in (1e-4, 1e-8, 1e-10) for nm in (1, 2, 3)]

        def solve(caps):
            xs = [B.Instance(dg, alpha, t, nm, c) for (t, nm), c in zip(specs, caps)]
            B.pr_solve_batch(xs, precision="mixed")
            return xs
        insts = solve([500] * len(specs))
        prev = previous_iterates(solve, insts)
        for x, rp in zip(insts, prev):
            assert x.converged
            assert_bound_parity(orc, g, alpha, x.tol, x.norm, 500, x.out, x.iters, x.converged, ref.ranks,
                                r_prev=rp, err=x.err, err_l1=x.err_l1, what=f"tau {x.tol} norm {x.norm}")
        # a tight tau is reached by the refinement phase: close to the FP64 answer
        tight = [x for x in insts if x.tol == 1e-10 and x.norm == 1][0]
        assert rel_l1(tight.out, ref.ranks) < 1e-8


def test_fp32_error_bound(B, orc, er):
    """FP32 throughout: an L1 stop (bound from tau alone) and an Linf stop
    (bound from the host-recomputed last step)."""
    ref = orc.pagerank(er, 0.85, 1e-13, 1, 10000)
    with B.Graph.from_csr(er) as dg:
        x = B.Instance(dg, 0.85, 1e-5, 1, 500)
        B.pr_solve_batch([x], precision="fp32")
        assert x.converged
        assert_bound_parity(orc, er, 0.85, 1e-5, 1, 500, x.out, x.iters, x.converged, ref.ranks, what="fp32 L1")

        def solve(caps):
            xs = [B.Instance(dg, 0.85, 1e-8, 3, caps[0])]
            B.pr_solve_batch(xs, precision="fp32")
            return xs
        y = solve([500])
        rp = previous_iterates(solve, y)
        assert_bound_parity(orc, er, 0.85, 1e-8, 3, 500, y[0].out, y[0].iters, y[0].converged, ref.ranks,
                            r_prev=rp[0], err=y[0].err, err_l1=y[0].err_l1, what="fp32 Linf")


def test_invalid_instance_reports_its_status(B, er):
    with B.Graph.from_csr(er) as dg:
        good = B.Instance(dg, 0.85, 1e-6, 1, 500)
        bad = B.Instance(dg, 1.5, 1e-6, 1, 500)
        st = B.pr_solve_batch([good, bad], check=False)
        assert st == B.PR_EINVAL and bad.status == B.PR_EINVAL
        assert good.status == 0 and good.converged


@pytest.mark.parametrize("group", ["auto", "pack", "single"])
def test_grouping_modes_match_oracle(B, orc, gg, group):
    """Every grouping of a 12-column alpha x tau batch on two graphs (jobs of
    several widths, run as separate sub-solves under "auto") meets parity."""
    g1 = gg.rmat(15, 16, seed=41)
    g2 = gg.erdos_renyi(20000, 160000, 900, 42)
    specs = [(gi, a, t, nm) for gi in (0, 1) for a, t, nm in
             ((0.5, 1e-9, 1), (0.7, 1e-10, 2), (0.85, 1e-10, 1), (0.9, 1e-8, 3), (0.95, 1e-10, 1), (0.99, 1e-7, 2))]
    graphs = [g1, g2]
    dgs = [B.Graph.from_csr(g) for g in graphs]
    insts = [B.Instance(dgs[gi], a, t, nm, 500) for gi, a, t, nm in specs]
    B.pr_solve_batch(insts, group=group)
    for (gi, a, t, nm), x in zip(specs, insts):
        ref = orc.pagerank(graphs[gi], a, t, nm, 500, history=True, threads=orc.default_threads())
        assert_fp64_parity(x.out, x.iters, x.err, ref, t, nm, f"{group} graph {gi} alpha {a}")
    for d in dgs:
        d.close()


@pytest.mark.parametrize("group", ["auto", "pack", "single"])
def test_grouping_modes_mixed_precision(B, orc, gg, group):
    g = gg.rmat(14, 16, seed=43)
    alphas = (0.6, 0.8, 0.85, 0.9, 0.95)
    refs = {a: orc.pagerank(g, a, 1e-13, 1, 10000) for a in alphas}
    with B.Graph.from_csr(g) as dg:
        insts = [B.Instance(dg, a, 1e-10, 1, 500) for a in alphas]
        B.pr_solve_batch(insts, precision="mixed", group=group)
        for a, x in zip(alphas, insts):
            assert x.converged
            assert_bound_parity(orc, g, a, 1e-10, 1, 500, x.out, x.iters, x.converged, refs[a].ranks,
                                what=f"{group} alpha {a}")


def test_graph_tune_measures_and_caches(B, gg):
    g = gg.rmat(14, 16, seed=44)
    with B.Graph.from_csr(g) as dg:
        t1 = B.pr_graph_tune(dg, "df64", 8)
        assert all(t > 0 for t in t1[:4]) and t1[4] == 0 and t1[5] == 0
        t2 = B.pr_graph_tune(dg, "df64", 8)
        assert t2 == t1                                   # cached, not timed again
        with B.Graph.from_csr(g) as dg2:                  # same signature: same entry
            assert B.pr_graph_tune(dg2, "df64", 4)[:3] == t1[:3]
        with pytest.raises(B.PageRankError):
            B.pr_graph_tune(dg, "df64", 3)


@pytest.mark.parametrize("kernels", ["fused", "split"])
@pytest.mark.parametrize("width", [2, 4, 8, 16])
def test_multi_column_kernels_match_oracle(B, orc, gg, kernels, width):
    """One job of `width` columns (distinct alphas, PR_GROUP_PACK) with one
    fused kernel per pass or split passes, df64 and fp64."""
    g = gg.rmat(15, 16, seed=47)
    alphas = [0.5 + 0.45 * k / max(width - 1, 1) for k in range(width)]
    refs = {a: orc.pagerank(g, a, 1e-10, 1, 500, history=True, threads=orc.default_threads()) for a in alphas}
    with B.Graph.from_csr(g) as dg:
        for prec in ("df64", "fp64"):
            insts = [B.Instance(dg, a, 1e-10, 1, 500) for a in alphas]
            B.pr_solve_batch(insts, group="pack", kernels=kernels, precision=prec)
            for a, x in zip(alphas, insts):
                assert_fp64_parity(x.out, x.iters, x.err, refs[a], 1e-10, 1, f"W {width} {kernels} {prec} alpha {a}")


def test_alpha_continuation_matches_oracle_from_the_same_starts(B, orc, gg):
    """PR_INIT_CHAIN (the alpha sweep of Section 2 in its order): on each
    graph the first alpha starts from 1/N and every later one from the
    previous alpha's final answer. Each column is compared with the oracle run
    from the start the chain gave it (the previous column's answer as returned),
    and two graphs run their chains side by side."""
    g1 = gg.rmat(14, 16, seed=61)
    g2 = gg.erdos_renyi(5000, 40000, 200, 62)
    alphas = [0.95, 0.5, 0.7, 0.85, 0.6]          # given out of order: the chain sorts them
    graphs = [g1, g2]
    dgs = [B.Graph.from_csr(g) for g in graphs]
    # two taps on every (graph, alpha): the chain continues from the later one
    specs = [(gi, a, t, 1) for gi in (0, 1) for a in alphas for t in (1e-6, 1e-10)]
    insts = [B.Instance(dgs[gi], a, t, nm, 500) for gi, a, t, nm in specs]
    B.pr_solve_batch(insts, init="chain")
    for gi, g in enumerate(graphs):
        prev = None
        for a in sorted(alphas):
            xs = [(t, x) for (gj, a2, t, nm), x in zip(specs, insts) if gj == gi and a2 == a]
            taps = [(t, 1, 500) for t, _ in xs]
            refs = orc.pagerank_taps(g, a, taps, init=prev, threads=orc.default_threads())
            for (t, x), r in zip(xs, refs):
                assert_fp64_parity(x.out, x.iters, x.err, r, t, 1, f"graph {gi} alpha {a} tau {t}")
            prev = [x for t, x in xs if t == 1e-10][0].out
    # the chain saves updates over the uniform start on the later alphas
    uni = [B.Instance(dgs[gi], a, t, nm, 500) for gi, a, t, nm in specs]
    B.pr_solve_batch(uni)
    assert sum(x.iters for x in insts) < sum(x.iters for x in uni)
    for d in dgs:
        d.close()


def test_sweep_outputs_match_oracle(B, orc, er):
    """The alpha sweep's outputs (Section 2): per alpha, the L1 distance of its
    ranks to the alpha = 0.85 ranks and its iterations relative to alpha = 0.85,
    from the batched sweep and from the oracle."""
    alphas = [0.5, 0.6, 0.7, 0.8, 0.85, 0.9, 0.95]
    with B.Graph.from_csr(er) as dg:
        xs = [B.Instance(dg, a, 1e-10, 1, 500) for a in alphas]
        B.pr_solve_batch(xs)
    refs = [orc.pagerank(er, a, 1e-10, 1, 500, history=True) for a in alphas]
    k85 = alphas.index(0.85)
    for a, x, r in zip(alphas, xs, refs):
        d_gpu = float(np.abs(x.out - xs[k85].out).sum())
        d_orc = float(np.abs(r.ranks - refs[k85].ranks).sum())
        # each answer is within 1e-12 (relative L1) of the oracle's
        assert abs(d_gpu - d_orc) <= 4e-12, (a, d_gpu, d_orc)
        assert x.iters * refs[k85].iters == r.iters * xs[k85].iters, (a, x.iters, r.iters)


def test_fp32_stalls_in_the_papers_order(B, gg):
    """The sensitivity stalls of Section 4 reproduced with FP32 arithmetic on a
    slow-mixing road-like lattice (300 x 400, seed 7), alpha 0.85: below some
    tau the FP32 iteration cannot reduce its step and runs into the 500 cap,
    first for L1, then L2, then Linf (the paper: L1 from 1e-8, L2/Linf from
    1e-9 on web-BerkStan), while DF64 converges at every tau."""
    g = gg.road_grid(300, 400, seed=7)
    taus = [10.0 ** -k for k in range(4, 13)]
    onset = {}
    with B.Graph.from_csr(g) as dg:
        for prec in ("fp32", "df64"):
            xs = [B.Instance(dg, 0.85, t, nm, 500) for t in taus for nm in (1, 2, 3)]
            B.pr_solve_batch(xs, precision=prec)
            for nm in (1, 2, 3):
                hit = [x.tol for x in xs if x.norm == nm and x.iters >= 500]
                # once a norm stalls, every smaller tau stalls too
                assert all(not x.converged for x in xs if x.norm == nm and hit and x.tol <= max(hit))
                onset[(prec, nm)] = max(hit) if hit else 0.0
    assert onset[("df64", 1)] == onset[("df64", 2)] == onset[("df64", 3)] == 0.0
    assert onset[("fp32", 1)] > 0.0
    assert onset[("fp32", 1)] > onset[("fp32", 2)] > onset[("fp32", 3)] > 0.0


def test_planner_precision_choice(B, orc, gg):
    """PR_PREC_AUTO: per graph the planner runs DF64 or mixed precision,
    whichever its cost model predicts cheaper; every answer meets the bound of
    the precision used (FP64 parity when no column ran mixed)."""
    g = gg.rmat(15, 16, seed=71)
    alphas = (0.5, 0.7, 0.85, 0.9, 0.95)
    with B.Graph.from_csr(g) as dg:
        xs = [B.Instance(dg, a, 1e-10, 1, 500) for a in alphas]
        B.pr_solve_batch(xs, precision="auto")
        st = B.pr_last_solve_stats()
        assert st["columns"] == len(alphas) and 0 <= st["mixed_columns"] <= len(alphas)
        for a, x in zip(alphas, xs):
            if st["mixed_columns"] == 0:
                ref = orc.pagerank(g, a, 1e-10, 1, 500, history=True, threads=orc.default_threads())
                assert_fp64_parity(x.out, x.iters, x.err, ref, 1e-10, 1, f"auto alpha {a}")
            else:
                star = orc.pagerank(g, a, 1e-13, 1, 10000, threads=orc.default_threads())
                assert_bound_parity(orc, g, a, 1e-10, 1, 500, x.out, x.iters, x.converged, star.ranks,
                                    what=f"auto alpha {a}")
        # mixed requested: every column mixed
        B.pr_solve_batch([B.Instance(dg, a, 1e-10, 1, 500) for a in alphas], precision="mixed")
        assert B.pr_last_solve_stats()["mixed_columns"] == len(alphas)


def test_fp32_split_passes_beyond_the_hub_table(B, orc, gg):
    """FP32 split passes on a graph larger than the gather kernel's shared
    hub table (R-MAT scale 17: 131,072 vertices), against the oracle's fixed
    point (tau-only bound of an L1 stop)."""
    g = gg.rmat(17, 16, seed=73)
    star = orc.pagerank(g, 0.85, 1e-13, 1, 10000, threads=orc.default_threads())
    with B.Graph.from_csr(g) as dg:
        x = B.Instance(dg, 0.85, 1e-5, 1, 500)
        B.pr_solve_batch([x], precision="fp32", kernels="split")
        assert x.converged
        assert_bound_parity(orc, g, 0.85, 1e-5, 1, 500, x.out, x.iters, x.converged, star.ranks, what="fp32 split")


def test_graph_creation_reuses_device_memory(B, gg):
    """Creating and destroying the same graph many times holds the device's
    free memory steady: a graph's arrays come from the graph pool and go back
    to it, and creation's scratch goes back to the workspace pool (the
    counting sort's block scratch once leaked a few MB per graph)."""
    import torch
    g = gg.rmat(16, 16, seed=5)
    for _ in range(3):
        B.Graph.from_csr(g).close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(40):
        B.Graph.from_csr(g).close()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (8 << 20)


def test_workspace_pool_info_and_release(B, er):
    """The workspace pool lends memory only during calls and keeps it reserved
    between them; pr_workspace_release returns the reserve to the device."""
    import torch
    with B.Graph.from_csr(er) as dg:
        B.pr_solve(dg, 0.85, 1e-10, 1, 500)
        torch.cuda.synchronize()
        reserved, used, high = B.workspace_info()
        assert used == 0 and high > 0 and reserved >= high
        B.workspace_release()
        reserved2, used2, _ = B.workspace_info()
        assert used2 == 0 and reserved2 == 0
        B.pr_solve(dg, 0.85, 1e-10, 1, 500)          # reserves again as needed
        assert B.workspace_info()[0] > 0


@pytest.mark.parametrize("width", [2, 4])
@pytest.mark.parametrize("precision", ["df64", "fp64", "fp32"])
def test_hub_kernel_several_columns(B, orc, gg, precision, width):
    """Jobs of two and four columns with split passes (the hub gather kernel
    reading all columns of a source with one vector load, two for four FP64
    columns) on a graph with rows of every tile kind: short rows, rows cut
    into one chunk and rows cut into several (5,000 and 9,000 in-edges)."""
    from tests.test_gpu_parity import adversarial
    g = adversarial(gg)["thresholds"]
    alphas = (0.7, 0.9) if width == 2 else (0.6, 0.7, 0.85, 0.95)
    with B.Graph.from_csr(g) as dg:
        xs = [B.Instance(dg, a, 1e-10 if precision != "fp32" else 1e-5, 1, 500) for a in alphas]
        B.pr_solve_batch(xs, group="pack", kernels="split", precision=precision)
        for a, x in zip(alphas, xs):
            if precision == "fp32":
                star = orc.pagerank(g, a, 1e-13, 1, 10000)
                assert_bound_parity(orc, g, a, 1e-5, 1, 500, x.out, x.iters, x.converged, star.ranks,
                                    what=f"fp32 W{width} alpha {a}")
            else:
                ref = orc.pagerank(g, a, 1e-10, 1, 500, history=True)
                assert_fp64_parity(x.out, x.iters, x.err, ref, 1e-10, 1, f"{precision} W{width} alpha {a}")


def test_mixed_precision_four_column_jobs(B, orc, gg):
    """Mixed precision in jobs of four columns with split passes: the FP32
    phase and the DF64 refinement both gather with the four-column hub kernel
    (16- and 32-byte vectors); every answer within the bound."""
    g = gg.rmat(15, 16, seed=81)
    alphas = (0.6, 0.75, 0.85, 0.95)
    with B.Graph.from_csr(g) as dg:
        xs = [B.Instance(dg, a, 1e-10, 1, 500) for a in alphas]
        B.pr_solve_batch(xs, precision="mixed", group="pack", kernels="split")
        st = B.pr_last_solve_stats()
        assert st["mixed_columns"] == len(alphas)
        for a, x in zip(alphas, xs):
            assert x.converged
            star = orc.pagerank(g, a, 1e-13, 1, 10000, threads=orc.default_threads())
            assert_bound_parity(orc, g, a, 1e-10, 1, 500, x.out, x.iters, x.converged, star.ranks,
                                what=f"mixed W4 alpha {a}")


def test_prepared_batch_repeats_the_same_solve(B, orc, er):
    """A PreparedBatch marshals its instances once; every solve gives the
    answers pr_solve_batch gives for the same instances."""
    import torch
    alphas = (0.6, 0.85)
    with B.Graph.from_csr(er) as dg:
        outs = [torch.empty(er.n, dtype=torch.float64, device="cuda") for _ in range(6)]
        specs = [(a, t, nm) for a in alphas for t, nm in ((1e-6, 1), (1e-10, 1), (1e-9, 3))]
        pb = B.PreparedBatch([B.Instance(dg, a, t, nm, 500, out=outs[k]) for k, (a, t, nm) in enumerate(specs)],
                             outputs_on_device=True)
        ref = [B.Instance(dg, a, t, nm, 500) for a, t, nm in specs]
        B.pr_solve_batch(ref)
        for call in range(2):
            for o in outs:
                o.fill_(float("nan"))
            pb.solve()
            assert list(pb.iters) == [x.iters for x in ref]
            for k, x in enumerate(ref):
                assert np.array_equal(outs[k].cpu().numpy(), x.out)
        xs = pb.fill()
        for x, r, (a, t, nm) in zip(xs, ref, specs):
            assert x.iters == r.iters and x.converged == r.converged and x.err == r.err
            o = orc.pagerank(er, a, t, nm, 500, history=True)
            assert_fp64_parity(x.out.cpu().numpy(), x.iters, x.err, o, t, nm, f"prepared alpha {a} tau {t}")
