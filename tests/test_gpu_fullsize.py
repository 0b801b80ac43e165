"""Parity at the workloads' full sizes, in the launch configuration bench.py
times: every output element against the CPU oracle (run with all host cores on
its independent vertex loop; results are bit-identical to one thread)."""
import numpy as np
import pytest

from tests.parity import assert_fp64_parity, bound_l1

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def B():
    from paper_2108_02997_gb300 import binding
    binding.lib()
    return binding


def test_rmat22_six_instances(B, orc, gg):
    """R-MAT scale 22, alpha 0.85, tau {1e-6, 1e-10} x {L1, L2, Linf}: one batch
    sharing one trajectory, device outputs, graph loop (bench default)."""
    import torch
    g = gg.rmat(22, 16, seed=22)
    specs = [(t, nm) for t in (1e-6, 1e-10) for nm in (1, 2, 3)]
    refs = orc.pagerank_taps(g, 0.85, [(t, nm, 500) for t, nm in specs], threads=orc.default_threads())
    with B.Graph.from_csr(g) as dg:
        insts = [B.Instance(dg, 0.85, t, nm, 500, out=torch.empty(g.n, dtype=torch.float64, device="cuda"))
                 for t, nm in specs]
        B.pr_solve_batch(insts, outputs_on_device=True)
        for (t, nm), x, r in zip(specs, insts, refs):
            assert_fp64_parity(x.out.cpu().numpy(), x.iters, x.err, r, t, nm, f"s22 tau {t} norm {nm}")


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
        x = B.Instance(dg, alpha, 1e-10, 3, 500, out=torch.empty(g.n, dtype=torch.float64, device="cuda"))
        B.pr_solve_batch([x], precision="mixed", outputs_on_device=True)
        assert x.converged
        err = float(np.abs(x.out.cpu().numpy() - ref.ranks).sum())
        assert err <= bound_l1(alpha, 1e-10, 3, x.err_l1), (alpha, err, x.err_l1)


_CACHE = {}


def _rmat24(gg):
    if "g" not in _CACHE:
        _CACHE["g"] = gg.rmat(24, 16, seed=24)
    return _CACHE["g"]
