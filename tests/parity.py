"""Tolerances and comparison rules shared by the GPU parity tests.

* FP64-class forms (df64, fp64) against the FP64 oracle from the same start:
  relative L1 error of the ranks <= 1e-12, iteration counts exact except where
  the oracle's norm at the deciding iteration lies within 1e-12 (relative) of
  tau, where either count is accepted.
* Every other form (fp32, mixed, warm starts): L1 distance to the oracle run
  at tau = 1e-13 at most 10 * max(tau_L1, delta_1) / (1 - alpha) (the L1
  contraction bound of the iteration, Section 2's update being an alpha
  contraction in L1). For an L1 stop that converged, delta_1 < tau and the
  bound is 10 tau / (1 - alpha). Otherwise delta_1 = ||r^i - r^{i-1}||_1 is
  recomputed on the host from the solver's last two iterates (the second one
  from the same call capped at i - 1 updates), never taken from the solver's
  own report; the report is checked against it, the stop is checked to be
  legitimate in its own norm, and r^i is checked to be one update of r^{i-1}
  (the oracle's step) within the update's rounding, whose measured size enters
  the bound:  ||r^i - r*|| <= (alpha delta_1 + eps) / (1 - alpha).
"""
import numpy as np

RANK_REL_L1 = 1e-12
TIE_REL = 1e-12


def rel_l1(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def iters_match(gpu_iters, ref, tau, norm):
    """Exact match, or a tie: the oracle's norm at iteration gpu_iters or
    ref.iters is within TIE_REL of tau."""
    if gpu_iters == ref.iters:
        return True
    h = ref.err_hist
    if h is None:
        return False
    for it in (gpu_iters, ref.iters):
        if 1 <= it <= len(h) and abs(h[it - 1, norm - 1] - tau) <= TIE_REL * tau:
            return True
    return False


def assert_fp64_parity(gpu_ranks, gpu_iters, gpu_err, ref, tau, norm, what=""):
    e = rel_l1(gpu_ranks, ref.ranks)
    assert e <= RANK_REL_L1, f"{what}: relative L1 {e:.3e} > {RANK_REL_L1}"
    assert iters_match(gpu_iters, ref, tau, norm), f"{what}: iterations {gpu_iters} vs oracle {ref.iters}"
    if gpu_iters == ref.iters:
        # |err_gpu - err_oracle| <= ||dr_gpu - dr_oracle|| <= ||dr_gpu - dr_oracle||_1
        #   <= ||r^i_gpu - r^i_or||_1 + ||r^{i-1}_gpu - r^{i-1}_or||_1 <= 2 * RANK_REL_L1 * ||r||_1
        bound = 2.0 * RANK_REL_L1 * float(np.abs(ref.ranks).sum())
        assert abs(gpu_err - ref.err) <= bound, (what, gpu_err, ref.err)


def bound_l1(alpha, tau, norm, delta1):
    t = tau if norm == 1 else 0.0
    return 10.0 * max(t, delta1) / max(1.0 - alpha, 1e-300)


# Rounding of one update, in L1 on a vector summing to 1: FP32 (one rounding
# per contribution and a summation depth of at most ~20 at 2^-24) and
# FP64-class (df64 carries a 48-bit significand).
UPDATE_EPS_FP32 = 1e-5
UPDATE_EPS_FP64 = 1e-12
# The solver's step norms against the host's: summation order (relative), and
# the solver forming each difference r^i - r^{i-1} in its own value type
# (df64: an absolute error up to 2^-47 of the rank itself per element, so the
# norm of the differences is off by at most 2^-47 times the same norm of the
# ranks; FP32 differences of nearby FP32 values are exact).
REPORT_REL = 1e-9
REPORT_ABS = 2.0 ** -46


def is_fp32_iterate(r):
    """True when every value is exactly an FP32 number (the answer came from
    an FP32-phase update, not from a df64/FP64 one)."""
    r = np.asarray(r, np.float64)
    return bool(np.array_equal(r.astype(np.float32).astype(np.float64), r))


def assert_bound_parity(orc, g, alpha, tau, norm, max_iter, r, iters, converged, r_star, *, r_prev=None,
                        err=None, err_l1=None, threads=1, what=""):
    """Accuracy of a non-FP64 answer against the oracle's fixed point r_star
    (the oracle run at tau = 1e-13), reading no value the solver computed about
    its own error. Returns the measured L1 error."""
    r = np.asarray(r, np.float64)
    e_star = float(np.abs(r - r_star).sum())
    if r_prev is None:
        assert converged and norm == 1, f"{what}: the previous iterate is needed for this stop"
        bound = 10.0 * tau / (1.0 - alpha)
        assert e_star <= bound, f"{what}: L1 error {e_star:.3e} > {bound:.3e}"
        return e_star
    r_prev = np.asarray(r_prev, np.float64)
    d = orc.norms(r, r_prev)                     # host: L1, L2, Linf of r^i - r^{i-1}
    rn = orc.norms(r, np.zeros_like(r))          # the same norms of r itself
    tol = [REPORT_REL * d[k] + REPORT_ABS * rn[k] for k in range(3)]
    if err is not None:
        assert abs(err - d[norm - 1]) <= tol[norm - 1], (what, err, d[norm - 1])
    if err_l1 is not None:
        assert abs(err_l1 - d[0]) <= tol[0], (what, err_l1, d[0])
    if converged:
        assert d[norm - 1] < tau + tol[norm - 1], f"{what}: step norm {d[norm - 1]:.3e} is not below {tau}"
    else:
        assert iters == max_iter, f"{what}: stopped at {iters} without converging (cap {max_iter})"
    s, _ = orc.step(g, alpha, r_prev, threads=threads)
    eps = float(np.abs(r - s).sum())             # ||r^i - F(r^{i-1})||_1
    lim = UPDATE_EPS_FP32 if is_fp32_iterate(r) else UPDATE_EPS_FP64
    assert eps <= lim, f"{what}: r^i is not one update of r^(i-1): {eps:.3e} > {lim:.0e}"
    t = tau if (norm == 1 and converged) else 0.0
    bound = (10.0 * max(t, float(d[0])) + 2.0 * eps) / (1.0 - alpha)
    assert e_star <= bound, f"{what}: L1 error {e_star:.3e} > {bound:.3e} (delta_1 {d[0]:.3e}, eps {eps:.1e})"
    return e_star


def _host(x):
    return x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x, np.float64)


def previous_iterates(solve, insts, start=None):
    """r^{i-1} of every solved instance. ``solve(max_iters)`` repeats the same
    call with instance k capped at max_iters[k] updates (same graphs, alphas,
    norms, taus, starts and options, hence the same iterate sequences and the
    same column grouping when every instance's trajectory is its own column or
    the call has one trajectory) and returns its solved instances, each of
    which must have stopped at its cap without converging. Instances that
    stopped after one update get the start (``start``: one vector, or None for
    the uniform 1/N)."""
    caps = [max(x.iters - 1, 1) for x in insts]
    again = solve(caps)
    prev = []
    for x, cap, y in zip(insts, caps, again):
        out = _host(y.out)
        if x.iters == 1:
            n = out.shape[0]
            prev.append(np.full(n, 1.0 / n) if start is None else np.asarray(start, np.float64))
        else:
            assert y.iters == cap and not y.converged, (x.iters, y.iters, y.converged)
            prev.append(out)
    return prev
