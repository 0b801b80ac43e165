"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints, the fixed point of the Google matrix solved directly, closed
forms derived by hand, exact rational arithmetic, or norm inequalities.
"""
import json
import math
from fractions import Fraction
from pathlib import Path

import numpy as np
import pytest

GOLDEN = Path(__file__).resolve().parent / "golden"


def small_graphs(gg):
    """Seeded small graphs with dangling vertices, isolated vertices and hubs."""
    out = []
    for seed, (n, m, d) in enumerate([(12, 30, 2), (50, 300, 5), (120, 900, 10), (200, 1500, 30)]):
        out.append(gg.erdos_renyi(n, m, d, seed + 100))
    out.append(gg.rmat(7, 8, seed=5))
    out.append(gg.from_edges(6, [0, 1, 2, 3], [5, 5, 5, 5]))       # in-star into a dangling hub + isolated vertex
    return out


# ---------------------------------------------------------------- Section 1

def test_iteration_estimate_matches_printed_values(orc):
    cases = json.loads((GOLDEN / "iteration_estimates.json").read_text())["cases"]
    for c in cases:
        assert orc.estimate_iterations(c["tau"], c["alpha"]) == c["iterations"], c


def test_estimate_is_tight_on_disjoint_cycles(orc, gg):
    """On two disjoint directed cycles from a start constant on each cycle, the
    error shrinks exactly by alpha per iteration: r^k = 1/N + alpha^k (r^0 - 1/N),
    so ||r^k - r^{k-1}|| = (1 - alpha) alpha^(k-1) ||r^0 - 1/N|| in every norm."""
    na, nb = 7, 13
    n = na + nb
    src = list(range(na)) + list(range(na, n))
    dst = [(i + 1) % na for i in range(na)] + [na + (i + 1) % nb for i in range(nb)]
    g = gg.from_edges(n, src, dst)
    a = 0.07
    b = (1.0 - na * a) / nb
    r0 = np.array([a] * na + [b] * nb)
    e0 = r0 - 1.0 / n
    for alpha in (0.5, 0.85, 0.95):
        for norm, e0n in ((1, np.abs(e0).sum()), (2, math.sqrt((e0 ** 2).sum())), (3, np.abs(e0).max())):
            for tau in (1e-4, 3e-7, 1e-10):
                k = 1
                while (1 - alpha) * alpha ** (k - 1) * e0n >= tau:
                    k += 1
                margin = abs((1 - alpha) * alpha ** (k - 1) * e0n - tau) / tau
                if margin < 1e-9:
                    continue  # closed form too close to tau to separate from rounding
                res = orc.pagerank(g, alpha, tau, norm, 2000, init=r0)
                assert res.converged and res.iters == k, (alpha, norm, tau, res.iters, k)
                expect = 1.0 / n + alpha ** k * e0
                assert np.abs(res.ranks - expect).max() < 1e-15


# ---------------------------------------------------------------- Section 2: fixed point

def test_converged_ranks_match_dense_solve(orc, gg):
    for g in small_graphs(gg):
        for alpha in (0.5, 0.85, 0.95):
            tau = 1e-14
            res = orc.pagerank(g, alpha, tau, 1, 10_000)
            assert res.converged
            rstar = orc.dense_solve(g, alpha)
            # ||r^i - r*||_1 <= alpha/(1-alpha) ||r^i - r^{i-1}||_1 (L1 contraction)
            bound = alpha / (1 - alpha) * res.err + 1e-13
            assert np.abs(res.ranks - rstar).sum() <= bound, (g.name, alpha)


def test_alpha_one_matches_dense_solve(orc, gg):
    g = gg.erdos_renyi(60, 400, 6, 9)
    res = orc.pagerank(g, 1.0, 1e-13, 1, 20_000)
    assert res.converged
    rstar = orc.dense_solve(g, 1.0)
    assert np.abs(res.ranks - rstar).sum() < 1e-9


def test_out_star_closed_form(orc, gg):
    # centre 0 -> L dangling leaves: r_c = 1/(N+alpha), r_leaf = (L+alpha)/(L(L+1+alpha))
    for L in (1, 5, 40):
        g = gg.from_edges(L + 1, [0] * L, list(range(1, L + 1)))
        for alpha in (0.3, 0.85, 0.99):
            res = orc.pagerank(g, alpha, 1e-15, 1, 100_000)
            n = L + 1
            assert abs(res.ranks[0] - 1 / (n + alpha)) < 1e-13
            leaf = (L + alpha) / (L * (L + 1 + alpha))
            assert np.abs(res.ranks[1:] - leaf).max() < 1e-13


def test_in_star_closed_form(orc, gg):
    # L leaves -> dangling centre 0: r_leaf = 1/(N + alpha L), r_c = (1 + alpha L)/(1 + L + alpha L)
    for L in (1, 5, 40):
        g = gg.from_edges(L + 1, list(range(1, L + 1)), [0] * L)
        for alpha in (0.3, 0.85, 0.99):
            res = orc.pagerank(g, alpha, 1e-15, 1, 100_000)
            n = L + 1
            assert abs(res.ranks[0] - (1 + alpha * L) / (1 + L + alpha * L)) < 1e-13
            assert np.abs(res.ranks[1:] - 1 / (n + alpha * L)).max() < 1e-13


def test_uniform_fixed_points_stop_after_one_update(orc, gg):
    n = 9
    cycle = gg.from_edges(n, list(range(n)), [(i + 1) % n for i in range(n)])
    s, d = zip(*[(u, v) for u in range(n) for v in range(n) if u != v])
    complete = gg.from_edges(n, list(s), list(d))
    edgeless = gg.from_edges(n, [], [])
    single = gg.from_edges(1, [], [])
    for g in (cycle, complete, edgeless, single):
        for norm in (1, 2, 3):
            res = orc.pagerank(g, 0.85, 1e-10, norm, 500)
            assert res.iters == 1 and res.converged
            assert np.abs(res.ranks - 1.0 / g.n).max() < 1e-16
            assert res.err < 1e-15  # N roundings of 1/N at most


def test_ranks_sum_to_one_every_iteration(orc, gg):
    for g in small_graphs(gg):
        r = np.full(g.n, 1.0 / g.n)
        for _ in range(40):
            r, _D = orc.step(g, 0.85, r)
            assert abs(r.sum() - 1.0) < 1e-13


def test_mass_is_conserved_on_large_skewed_graphs(orc, gg):
    """sum(r) = 1 holds analytically. On this graph (hub rows of ~40,000
    in-edges) plain sequential FP64 row sums lose 1.4e-12 of the mass; the
    oracle's compensated sums stay within rounding of 1."""
    g = gg.rmat(20, 16, seed=1017)
    res = orc.pagerank(g, 0.85, 1e-10, 1, 1000, threads=orc.default_threads())
    assert abs(res.ranks.sum() - 1.0) < 1e-14, res.ranks.sum() - 1.0


def test_compensated_sum_is_exact_on_a_cancellation_case(orc, gg):
    """A vertex whose in-edge terms are 1, 1e-16 (x 10) in CSR order: the
    compensated row sum keeps the small terms a plain FP64 sum would drop."""
    n = 12
    # vertex 0 receives from vertices 1..11; their ranks are set by the start
    g = gg.from_edges(n, list(range(1, n)), [0] * (n - 1))
    r0 = np.array([0.0, 1.0] + [1e-16] * 10)
    r1, _ = orc.step(g, 1.0, r0)
    # alpha = 1: r1[0] = c0 + sum = D/N + (1 + 10e-16), D = r0[0] (vertex 0 is dangling)
    assert r1[0] == 1.0 + 10e-16


def test_step_matches_exact_rationals(orc, gg):
    """Three updates in exact rational arithmetic (fractions), straight from the
    definition, agree with the FP64 oracle to rounding."""
    rng = np.random.default_rng(4)
    for trial in range(6):
        n = int(rng.integers(1, 9))
        m = int(rng.integers(0, n * n + 1))
        g = gg.from_edges(n, rng.integers(0, n, m), rng.integers(0, n, m))
        alpha = Fraction(int(rng.integers(1, 20)), 20)
        r = [Fraction(1, n)] * n
        rf = np.full(n, 1.0 / n)
        off, src, od = g.offsets, g.sources, g.outdeg
        for _ in range(3):
            D = sum((r[u] for u in range(n) if od[u] == 0), Fraction(0))
            c0 = (1 - alpha) / n + alpha * D / n
            r = [c0 + alpha * sum((r[int(src[e])] / int(od[src[e]]) for e in range(off[v], off[v + 1])),
                                  Fraction(0)) for v in range(n)]
            rf, _D = orc.step(g, float(alpha), rf)
            assert sum(r) == 1
            assert max(abs(float(a) - b) for a, b in zip(r, rf)) < 1e-15


# ---------------------------------------------------------------- Section 3: norms

def test_norms_on_a_worked_vector(orc):
    a = np.array([0.5, 0.1, 0.0, 0.2])
    b = np.array([0.2, 0.5, 0.0, 0.2])     # a - b = (0.3, -0.4, 0, 0)
    l1, l2, li = orc.norms(a, b)
    assert abs(l1 - 0.7) < 1e-15 and abs(l2 - 0.5) < 1e-15 and abs(li - 0.4) < 1e-15


def test_norm_order_and_tau_monotonicity(orc, gg):
    """||x||_inf <= ||x||_2 <= ||x||_1 on one trajectory gives
    iters(Linf) <= iters(L2) <= iters(L1); a smaller tau never needs fewer
    iterations."""
    for g in small_graphs(gg)[:4] + [gg.rmat(9, 16, seed=8)]:
        for alpha in (0.6, 0.85):
            prev = {1: 0, 2: 0, 3: 0}
            for tau in (1e-1, 1e-3, 1e-5, 1e-7, 1e-9):
                it = {nm: orc.pagerank(g, alpha, tau, nm, 500).iters for nm in (1, 2, 3)}
                assert it[3] <= it[2] <= it[1]
                for nm in it:
                    assert it[nm] >= prev[nm]
                prev = it


def test_history_is_consistent(orc, gg):
    g = gg.rmat(8, 16, seed=9)
    res = orc.pagerank(g, 0.85, 1e-9, 2, 500, history=True)
    h = res.err_hist
    assert h.shape == (res.iters, 3)
    assert np.all(h[:, 2] <= h[:, 1] + 1e-18) and np.all(h[:, 1] <= h[:, 0] + 1e-18)
    assert h[-1, 1] < 1e-9 <= h[-2, 1]
    assert res.err == h[-1, 1]


def test_cap_reached_reports_not_converged(orc, gg):
    g = gg.rmat(8, 16, seed=9)
    res = orc.pagerank(g, 0.85, 1e-30, 1, 7)
    assert res.iters == 7 and not res.converged


def test_threads_are_bit_identical(orc, gg):
    g = gg.rmat(11, 16, seed=12)
    a = orc.pagerank(g, 0.85, 1e-10, 1, 500, threads=1)
    b = orc.pagerank(g, 0.85, 1e-10, 1, 500, threads=4)
    assert a.iters == b.iters and np.array_equal(a.ranks, b.ranks) and a.err == b.err


def test_taps_equal_independent_solves(orc, gg):
    g = gg.erdos_renyi(300, 2500, 15, 21)
    taps = [(t, nm, 500) for t in (1e-2, 1e-5, 1e-8) for nm in (1, 2, 3)] + [(1e-30, 1, 17)]
    got = orc.pagerank_taps(g, 0.9, taps)
    for (t, nm, mi), r in zip(taps, got):
        ref = orc.pagerank(g, 0.9, t, nm, mi)
        assert r.iters == ref.iters and r.converged == ref.converged
        assert np.array_equal(r.ranks, ref.ranks) and r.err == ref.err


# ---------------------------------------------------------------- planted mistakes

def _mutant_step(g, alpha, r, mutation):
    """A deliberately wrong re-statement of one update, used to show the pins
    above catch each plausible mistake."""
    n = g.n
    od = g.outdeg
    D = sum(r[u] for u in range(n) if od[u] == 0)
    if mutation == "drop_dangling":
        D = 0.0
    c0 = (1 - alpha) / n + alpha * D / n
    out = np.empty(n)
    src, dst = g.edges()
    if mutation == "transpose":
        src, dst = dst, src
    acc = np.zeros(n)
    for u, v in zip(src, dst):
        d = od[u] if mutation != "transpose" else max(int(np.sum(g.sources == v)), 1)
        acc[v] += r[u] / max(d, 1)
    out[:] = c0 + alpha * acc
    return out


@pytest.mark.parametrize("mutation", ["drop_dangling", "transpose"])
def test_pins_catch_planted_mistakes(orc, gg, mutation):
    g = gg.erdos_renyi(40, 200, 5, 77)
    alpha = 0.85
    r = np.full(g.n, 1.0 / g.n)
    for _ in range(300):
        r = _mutant_step(g, alpha, r, mutation)
    rstar = orc.dense_solve(g, alpha)
    bad_sum = abs(r.sum() - 1.0) > 1e-6
    bad_fix = np.abs(r - rstar).sum() > 1e-6
    assert bad_sum or bad_fix
