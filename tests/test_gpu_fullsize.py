"""Parity at the workloads' full sizes, in the launch configuration bench.py
times: every output element against the CPU oracle (run with all host cores on
its independent vertex loop; results are bit-identical to one thread)."""
import numpy as np
import pytest

from tests.parity import assert_bound_parity, assert_fp64_parity, previous_iterates

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def B():
    from paper_2108_02997_gb300 import binding
    binding.lib()
    return binding


S22_SPECS = [(t, nm) for t in (1e-6, 1e-10) for nm in (1, 2, 3)]


@pytest.fixture(scope="module")
def s22(orc, gg):
    """R-MAT scale 22 (seed 22) and the oracle's answers for alpha 0.85, tau
    {1e-6, 1e-10} x {L1, L2, Linf} from the uniform start."""
    g = gg.rmat(22, 16, seed=22)
    refs = orc.pagerank_taps(g, 0.85, [(t, nm, 500) for t, nm in S22_SPECS], threads=orc.default_threads())
    return g, refs


@pytest.mark.parametrize("precision", ["df64", "fp64"])
def test_rmat22_six_instances(B, s22, precision):
    """R-MAT scale 22, alpha 0.85, tau {1e-6, 1e-10} x {L1, L2, Linf}: one batch
    sharing one trajectory, device outputs, graph loop (bench default), in the
    default df64 and in native FP64."""
    import torch
    g, refs = s22
    with B.Graph.from_csr(g) as dg:
        insts = [B.Instance(dg, 0.85, t, nm, 500, out=torch.empty(g.n, dtype=torch.float64, device="cuda"))
                 for t, nm in S22_SPECS]
        B.pr_solve_batch(insts, outputs_on_device=True, precision=precision)
        for (t, nm), x, r in zip(S22_SPECS, insts, refs):
            assert_fp64_parity(x.out.cpu().numpy(), x.iters, x.err, r, t, nm, f"s22 {precision} tau {t} norm {nm}")


def test_sixty_four_graphs_one_batch(B, orc, gg):
    """64 R-MAT graphs of scale 12 + (i mod 9), edge factor 16, alpha 0.85,
    tau 1e-10, L1, one batch."""
    graphs = [gg.rmat(12 + (i % 9), 16, seed=1000 + i) for i in range(64)]
    dgs = [B.Graph.from_csr(g) for g in graphs]
    insts = [B.Instance(d, 0.85, 1e-10, 1, 500) for d in dgs]
    B.pr_solve_batch(insts)
    for g, x in zip(graphs, insts):
        ref = orc.pagerank(g, 0.85, 1e-10, 1, 500, history=True, threads=orc.default_threads())
        assert_fp64_parity(x.out, x.iters, x.err, ref, 1e-10, 1, g.name)
    for d in dgs:
        d.close()


@pytest.mark.parametrize("alpha", [0.85, 0.95])
def test_rmat24_mixed_precision(B, orc, gg, alpha):
    """R-MAT scale 24, Linf, FP32 to 1e-6 then DF64 refinement to 1e-10,
    against the oracle run at tau = 1e-13 (cap 10,000)."""
    import torch
    g = _rmat24(gg)
    ref = orc.pagerank(g, alpha, 1e-13, 1, 10000, threads=orc.default_threads())
    with B.Graph.from_csr(g) as dg:
        def solve(caps):
            xs = [B.Instance(dg, alpha, 1e-10, 3, caps[0], out=torch.empty(g.n, dtype=torch.float64, device="cuda"))]
            B.pr_solve_batch(xs, precision="mixed", outputs_on_device=True)
            return xs
        x = solve([500])[0]
        assert x.converged
        rp = previous_iterates(solve, [x])[0]
        assert_bound_parity(orc, g, alpha, 1e-10, 3, 500, x.out.cpu().numpy(), x.iters, x.converged, ref.ranks,
                            r_prev=rp, err=x.err, err_l1=x.err_l1, threads=orc.default_threads(),
                            what=f"s24 mixed alpha {alpha}")


def test_rmat20_fp32(B, orc, gg):
    """FP32 throughout on R-MAT scale 20 (seed 20), alpha 0.85: an L1 stop at
    tau 1e-5 and an Linf stop at tau 1e-9, against the oracle at tau = 1e-13."""
    g = gg.rmat(20, 16, seed=20)
    ref = orc.pagerank(g, 0.85, 1e-13, 1, 10000, threads=orc.default_threads())
    with B.Graph.from_csr(g) as dg:
        def solve(caps):
            xs = [B.Instance(dg, 0.85, 1e-5, 1, caps[0]), B.Instance(dg, 0.85, 1e-9, 3, caps[1])]
            B.pr_solve_batch(xs, precision="fp32", share=False, group="single")
            return xs
        xs = solve([500, 500])
        prev = previous_iterates(solve, xs)
        for x, rp in zip(xs, prev):
            assert x.converged
            assert_bound_parity(orc, g, 0.85, x.tol, x.norm, 500, x.out, x.iters, x.converged, ref.ranks, r_prev=rp,
                                err=x.err, err_l1=x.err_l1, threads=orc.default_threads(),
                                what=f"s20 fp32 tau {x.tol} norm {x.norm}")


_CACHE = {}


def _rmat24(gg):
    if "g" not in _CACHE:
        _CACHE["g"] = gg.rmat(24, 16, seed=24)
    return _CACHE["g"]


def test_learned_start_on_unseen_rmat22(B, orc, gg):
    """The learned start on an evaluation graph (R-MAT scale 22, seed 3022, not
    used in training): the network's start against the oracle's forward pass
    with the same BF16 weights; the df64 solve from it against the oracle from
    the same start (FP64 parity); the mixed-precision solve from it against the
    oracle's fixed point (bound from the host-recomputed last step)."""
    import torch
    sets, keep = [], []
    for i in range(6):
        gt = gg.rmat(11 + (i % 3), 16, seed=2000 + i)
        dg = B.Graph.from_csr(gt)
        keep.append(dg)
        for a in (0.5, 0.7, 0.85, 0.95):
            r = torch.empty(gt.n, dtype=torch.float64, device="cuda")
            B.pr_solve(dg, a, 1e-12, 1, 1000, out=r)
            sets.append((dg, a, r))
    flat = B.init_mlp_params(seed=11)
    m = B.MLP(flat)
    m.train(sets, epochs=60, lr=3e-3)
    params = m.params()
    g = gg.rmat(22, 16, seed=3022)
    threads = orc.default_threads()
    with B.Graph.from_csr(g) as dg:
        r0 = m.warm_start(dg, 0.85).cpu().numpy()
        p = {}
        o = 0
        for k, shape in (("W1", (64, 5)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (1, 64)),
                         ("b3", (1,))):
            cnt = int(np.prod(shape))
            v = params[o:o + cnt].reshape(shape)
            p[k] = orc.bf16_round(v) if k.startswith("W") else v.astype(np.float64)
            o += cnt
        y, _ = orc.mlp_forward(orc.features(g, 0.85), p)
        start_ref = orc.warm_start_from_logits(y)
        assert abs(r0.sum() - 1.0) < 1e-12
        assert np.abs(r0 - start_ref).sum() <= 2e-2, np.abs(r0 - start_ref).sum()
        # df64 from the learned start: the oracle from the same start vector
        res = B.pr_solve(dg, 0.85, 1e-10, 1, 500, init="learned", mlp=m, history=True)
        ref = orc.pagerank(g, 0.85, 1e-10, 1, 500, init=r0, history=True, threads=threads)
        assert_fp64_parity(res.ranks, res.iters, res.err, ref, 1e-10, 1, "s22 learned df64")
        # mixed precision from the learned start, Linf stop
        star = orc.pagerank(g, 0.85, 1e-13, 1, 10000, threads=threads)

        def solve(caps):
            xs = [B.Instance(dg, 0.85, 1e-10, 3, caps[0])]
            B.pr_solve_batch(xs, precision="mixed", init="learned", mlp=m)
            return xs
        xs = solve([500])
        prev = previous_iterates(solve, xs, start=r0)
        assert xs[0].converged
        assert_bound_parity(orc, g, 0.85, 1e-10, 3, 500, xs[0].out, xs[0].iters, xs[0].converged, star.ranks,
                            r_prev=prev[0], err=xs[0].err, err_l1=xs[0].err_l1, threads=threads,
                            what="s22 learned mixed")
    m.close()
    for d in keep:
        d.close()
