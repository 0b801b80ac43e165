"""Tolerances and comparison rules shared by the GPU parity tests.

* FP64-class forms (df64, fp64) against the FP64 oracle from the same start:
  relative L1 error of the ranks <= 1e-12, iteration counts exact except where
  the oracle's norm at the deciding iteration lies within 1e-12 (relative) of
  tau, where either count is accepted.
* Every other form (fp32, mixed, warm starts): L1 distance to the oracle run
  at tau = 1e-13 at most 10 * max(tau_L1, delta_1) / (1 - alpha), with delta_1
  the solve's own final L1 step (the L1 contraction bound of the iteration).
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
