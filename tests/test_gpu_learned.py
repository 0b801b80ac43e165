"""GPU parity of the learned warm start (no counterpart in the paper): features,
the MLP forward pass and its gradients against the FP64 oracle evaluated with
the same BF16-rounded weights, the Adam update, and what a trained network
saves over the uniform start while converging to the same fixed point."""
import numpy as np
import pytest

from tests.parity import assert_bound_parity

pytestmark = pytest.mark.gpu

KEYS = (("W1", (64, 5)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (1, 64)), ("b3", (1,)))


@pytest.fixture(scope="module")
def B():
    from paper_2108_02997_gb300 import binding
    binding.lib()
    return binding


def unflatten(flat):
    out, o = {}, 0
    for k, s in KEYS:
        n = int(np.prod(s))
        out[k] = np.asarray(flat[o:o + n], np.float64).reshape(s)
        o += n
    return out


def oracle_params(orc, flat):
    """The values the GPU computes with: BF16 weight matrices, FP32 biases."""
    p = unflatten(flat)
    for k in ("W1", "W2", "W3"):
        p[k] = orc.bf16_round(p[k].astype(np.float32))
    return p


def flat_of(d):
    return np.concatenate([d[k].reshape(-1) for k, _ in KEYS])


@pytest.fixture(scope="module")
def setup(B, orc, gg):
    import torch
    g = gg.rmat(12, 16, seed=41)
    ref = orc.pagerank(g, 0.85, 1e-13, 1, 10000)
    dg = B.Graph.from_csr(g)
    target = torch.tensor(ref.ranks, dtype=torch.float64, device="cuda")
    return g, dg, ref, target


def test_features_match_oracle(B, orc, setup):
    g, dg, _, _ = setup
    f = B.pr_features(dg, 0.7).cpu().numpy()
    ref = orc.features(g, 0.7)
    assert np.abs(f - ref).max() <= 2e-6 * max(1.0, np.abs(ref).max())


def test_warm_start_matches_oracle_forward(B, orc, setup):
    g, dg, _, _ = setup
    flat = B.init_mlp_params(seed=5)
    m = B.MLP(flat)
    r0 = m.warm_start(dg, 0.85).cpu().numpy()
    p = oracle_params(orc, flat)
    y, _ = orc.mlp_forward(orc.features(g, 0.85), p)
    ref = orc.warm_start_from_logits(y)
    assert abs(r0.sum() - 1.0) < 1e-12
    assert np.abs(r0 - ref).sum() <= 2e-2, np.abs(r0 - ref).sum()
    m.close()


@pytest.fixture(scope="module")
def tiered(B, gg):
    """R-MAT scale 13 plus three hub vertices with 2,100, 4,000 and 8,000
    in-edges: rows for every feature worker size (a CTA per row from 2,048
    in-edges, a warp per row from 32, a thread per row below, empty rows)."""
    base = gg.rmat(13, 8, seed=43)
    s, d = base.edges()
    extra_s, extra_d = [], []
    for hub, k in ((11, 2100), (222, 4000), (3333, 8000)):
        srcs = (np.arange(k, dtype=np.int64) * 7 + hub + 1) % base.n
        srcs = srcs[srcs != hub]
        extra_s.append(srcs)
        extra_d.append(np.full(srcs.size, hub))
    g = gg.from_edges(base.n, np.concatenate([s] + extra_s), np.concatenate([d] + extra_d))
    deg = np.diff(g.offsets)
    assert (deg >= 2048).sum() >= 3 and ((deg >= 32) & (deg < 2048)).any() and (deg == 0).any()
    return g, B.Graph.from_csr(g)


def test_features_every_worker_size(B, orc, tiered):
    g, dg = tiered
    f = B.pr_features(dg, 0.9).cpu().numpy()
    ref = orc.features(g, 0.9)
    assert np.abs(f - ref).max() <= 2e-6 * max(1.0, np.abs(ref).max())


def test_warm_start_every_worker_size(B, orc, tiered):
    g, dg = tiered
    flat = B.init_mlp_params(seed=9)
    m = B.MLP(flat)
    r0 = m.warm_start(dg, 0.6).cpu().numpy()
    y, _ = orc.mlp_forward(orc.features(g, 0.6), oracle_params(orc, flat))
    ref = orc.warm_start_from_logits(y)
    assert abs(r0.sum() - 1.0) < 1e-12
    assert np.abs(r0 - ref).sum() <= 2e-2, np.abs(r0 - ref).sum()
    m.close()


def test_gradients_match_oracle(B, orc, setup):
    g, dg, ref_r, target = setup
    flat = B.init_mlp_params(seed=6)
    m = B.MLP(flat)
    loss, grad = m.loss_grad(dg, 0.85, target)
    p = oracle_params(orc, flat)
    F = orc.features(g, 0.85)
    t = np.log(g.n * ref_r.ranks)
    y, cache = orc.mlp_forward(F, p)
    og = orc.mlp_backward(p, cache, y, t)
    assert abs(loss - orc.mse_loss(y, t)) <= 2e-2 * orc.mse_loss(y, t)
    gd = unflatten(grad)
    for k, _ in KEYS:
        err = np.linalg.norm(gd[k] - og[k]) / max(np.linalg.norm(og[k]), 1e-30)
        assert err <= 2e-2, (k, err)
    m.close()


def test_adam_step_matches_oracle(B, orc, setup):
    g, dg, _, target = setup
    flat = B.init_mlp_params(seed=8)
    m = B.MLP(flat)
    _, grad = m.loss_grad(dg, 0.85, target)
    m.train([(dg, 0.85, target)], epochs=1, lr=1e-3)
    after = m.params().astype(np.float64)
    p = unflatten(flat.astype(np.float64))
    gg_ = unflatten(grad.astype(np.float64))
    mom = {k: np.zeros_like(v) for k, v in p.items()}
    vel = {k: np.zeros_like(v) for k, v in p.items()}
    orc.adam_update(p, gg_, mom, vel, 1, lr=1e-3)
    expect = flat_of(p)
    step = np.abs(expect - flat)
    assert np.abs(after - expect).max() <= 1e-5 * max(1.0, np.abs(flat).max()) + 1e-3 * step.max()
    m.close()


def test_training_lowers_loss_and_warm_start_saves_iterations(B, orc, gg):
    """Train on solver ranks of small seeded R-MAT graphs over the alpha grid,
    then solve an unseen graph from the learned start: the converged answer is
    the same fixed point (oracle bound) and fewer updates are needed."""
    import torch
    train = [gg.rmat(11 + (i % 3), 16, seed=2000 + i) for i in range(6)]
    sets, dgs = [], []
    for i, g in enumerate(train):
        dg = B.Graph.from_csr(g)
        dgs.append(dg)
        for a in (0.5, 0.7, 0.85, 0.95):
            r = torch.empty(g.n, dtype=torch.float64, device="cuda")
            B.pr_solve(dg, a, 1e-12, 1, 1000, out=r)
            sets.append((dg, a, r))
    m = B.MLP(B.init_mlp_params(seed=11))
    first, _ = m.loss_grad(*sets[0])
    last = m.train(sets, epochs=150, lr=3e-3)
    assert last < 0.5 * first, (first, last)
    test_g = gg.rmat(13, 16, seed=3013)
    dgt = B.Graph.from_csr(test_g)
    for a in (0.85, 0.95):
        ref = orc.pagerank(test_g, a, 1e-13, 1, 10000)
        uni = B.pr_solve(dgt, a, 1e-10, 1, 500)
        lrn = B.pr_solve(dgt, a, 1e-10, 1, 500, init="learned", mlp=m)
        assert lrn.converged
        assert_bound_parity(orc, test_g, a, 1e-10, 1, 500, lrn.ranks, lrn.iters, lrn.converged, ref.ranks,
                            what=f"learned alpha {a}")
        assert lrn.iters < uni.iters, (a, lrn.iters, uni.iters)
    m.close()


def test_auto_start_follows_its_cost_model(B, orc, gg):
    """PR_INIT_AUTO: training measures the network's gain over the uniform
    start; with no gain every column starts from 1/N (the uniform batch's
    answers exactly), with an overwhelming gain every column takes the learned
    start (the learned batch's answers exactly), and with the measured gain the
    answers meet the accuracy bound whichever start each column got."""
    import torch
    sets, keep = [], []
    for i in range(4):
        g = gg.rmat(11 + (i % 2), 16, seed=2100 + i)
        dg = B.Graph.from_csr(g)
        keep.append(dg)
        for a in (0.6, 0.85, 0.95):
            r = torch.empty(g.n, dtype=torch.float64, device="cuda")
            B.pr_solve(dg, a, 1e-12, 1, 1000, out=r)
            sets.append((dg, a, r))
    m = B.MLP(B.init_mlp_params(seed=12))
    assert m.gain() == (0.0, False)
    m.train(sets, epochs=80, lr=3e-3)
    gain, known = m.gain()
    assert known and gain > 0.0, gain
    g = gg.rmat(14, 16, seed=2199)
    alphas = (0.6, 0.8, 0.9)
    with B.Graph.from_csr(g) as dg:
        def run(init, mlp=m):
            xs = [B.Instance(dg, a, 1e-10, 1, 500) for a in alphas]
            B.pr_solve_batch(xs, init=init, mlp=mlp)
            return xs, B.pr_last_solve_stats()["learned_columns"]
        uni = [B.Instance(dg, a, 1e-10, 1, 500) for a in alphas]
        B.pr_solve_batch(uni)
        lrn, nl = run("learned")
        assert nl == len(alphas)
        m.set_gain(0.0)
        xs, nl = run("auto")
        assert nl == 0 and all(np.array_equal(x.out, y.out) and x.iters == y.iters for x, y in zip(xs, uni))
        m.set_gain(50.0)
        xs, nl = run("auto")
        assert nl == len(alphas) and all(np.array_equal(x.out, y.out) and x.iters == y.iters for x, y in zip(xs, lrn))
        m.set_gain(gain)
        xs, nl = run("auto")
        assert 0 <= nl <= len(alphas)
        for a, x in zip(alphas, xs):
            ref = orc.pagerank(g, a, 1e-13, 1, 10000)
            assert_bound_parity(orc, g, a, 1e-10, 1, 500, x.out, x.iters, x.converged, ref.ranks, what=f"auto alpha {a}")
    m.close()
    for d in keep:
        d.close()
