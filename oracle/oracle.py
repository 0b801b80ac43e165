"""CPU oracle for the PageRank hot path — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this module. The product
library never calls it and shares no code with it.

Contents, each following the paper "Adjusting PageRank parameters and
Comparing results" (section cited per function):

* :func:`pagerank`        — the power iteration with the common teleport term
                            and the L1/L2/Linf stopping rule (Sections 2, 3, 4),
                            in plain C (``pagerank_oracle.c``), FP64.
* :func:`pagerank_taps`   — many (tau, norm, max_iter) stopping rules read off
                            one trajectory (the tau sweep of Section 4 and the
                            norm comparison of Section 3 share iterates).
* :func:`dense_solve`     — the fixed point of the Google matrix by a direct
                            dense solve (N <= a few hundred), the definition the
                            iteration converges to (Section 1: power iteration).
* :func:`estimate_iterations` — log10(tau) / log10(alpha) (Section 1).
* mean ratios             — AM/GM/HM-RATIO and RATIO-AM/GM/HM (Sections 1, 3).
* :func:`features`, MLP   — the learned warm start's per-vertex features and a
                            5-64-64-1 GELU MLP with MSE loss and Adam, in FP64
                            numpy (no counterpart in the paper).

Parity status: every function here is pinned by tests in ``tests/`` against
values the paper prints, closed forms, exact rational arithmetic or finite
differences, except the paper's own per-graph figures (datasets absent): those
are "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "pagerank_oracle.c"
SO = HERE / "liboracle.so"

NORM_L1, NORM_L2, NORM_LINF = 1, 2, 3
NORM_NAMES = {NORM_L1: "L1", NORM_L2: "L2", NORM_LINF: "Linf"}

_lib = None


def build(force: bool = False) -> Path:
    """Compile the C oracle (plain C, no fused multiply-add, OpenMP for the
    independent vertex loop only)."""
    if force or not SO.exists() or SO.stat().st_mtime < SRC.stat().st_mtime:
        tmp = SO.with_suffix(".so.tmp")
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
               "-o", str(tmp), str(SRC), "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stdout + r.stderr)
        os.replace(tmp, SO)
    return SO


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(str(build()))
        vp = C.c_void_p
        lib.oracle_pagerank.argtypes = [C.c_int32, vp, vp, vp, C.c_double, C.c_double, C.c_int32,
                                        C.c_int32, vp, vp, vp, vp, vp, vp, C.c_int]
        lib.oracle_pagerank.restype = C.c_int
        lib.oracle_step.argtypes = [C.c_int32, vp, vp, vp, C.c_double, vp, vp, vp, C.c_int]
        lib.oracle_step.restype = None
        lib.oracle_norms.argtypes = [C.c_int32, vp, vp, vp]
        lib.oracle_norms.restype = None
        lib.oracle_features.argtypes = [C.c_int32, vp, vp, vp, C.c_double, vp]
        lib.oracle_features.restype = None
        _lib = lib
    return _lib


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    return a.ctypes.data if a is not None and a.size else None


@dataclass
class Result:
    ranks: np.ndarray
    iters: int
    err: float
    converged: bool
    err_hist: np.ndarray | None = None   # (iters, 3): L1, L2, Linf of r^i - r^{i-1}


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def pagerank(g, alpha: float, tau: float, norm: int = NORM_L1, max_iter: int = 500,
             init=None, history: bool = False, threads: int = 1) -> Result:
    """Pull PageRank power iteration (Section 2) stopped by the chosen norm
    (Section 3) against tau, or at max_iter (Sections 2 and 4).

    ``g`` has ``offsets``, ``sources`` (in-edge CSR) and ``outdeg``."""
    lib = _load()
    off, src, od = _i32(g.offsets), _i32(g.sources), _i32(g.outdeg)
    n = od.shape[0]
    out = np.empty(n, np.float64)
    it = C.c_int32()
    err = C.c_double()
    conv = C.c_int32()
    hist = np.zeros((max_iter, 3), np.float64) if history else None
    ini = _f64(init) if init is not None else None
    if ini is not None and ini.shape[0] != n:
        raise ValueError("init must have n entries")
    rc = lib.oracle_pagerank(n, _ptr(off), _ptr(src), _ptr(od), alpha, tau, norm, max_iter,
                             _ptr(ini), out.ctypes.data, C.byref(it), C.byref(err), C.byref(conv),
                             _ptr(hist), threads)
    if rc != 0:
        raise ValueError(f"oracle_pagerank rejected its arguments (rc={rc})")
    return Result(out, it.value, err.value, bool(conv.value),
                  hist[: it.value] if hist is not None else None)


def step(g, alpha: float, r, threads: int = 1):
    """One update r -> c0 + alpha A^T (r/d) (Section 2). Returns (r_new, D)."""
    lib = _load()
    off, src, od = _i32(g.offsets), _i32(g.sources), _i32(g.outdeg)
    r = _f64(r)
    out = np.empty_like(r)
    d = C.c_double()
    lib.oracle_step(od.shape[0], _ptr(off), _ptr(src), _ptr(od), alpha, r.ctypes.data,
                    out.ctypes.data, C.byref(d), threads)
    return out, d.value


def norms(a, b):
    """(L1, L2, Linf) of a - b (Section 3)."""
    lib = _load()
    a, b = _f64(a), _f64(b)
    out = np.empty(3, np.float64)
    lib.oracle_norms(a.shape[0], a.ctypes.data, b.ctypes.data, out.ctypes.data)
    return out


@dataclass
class Tap:
    tau: float
    norm: int
    max_iter: int


def pagerank_taps(g, alpha: float, taps, init=None, threads: int = 1):
    """Stop one trajectory at several (tau, norm, max_iter) rules.

    For a fixed graph, alpha and start, the iterates do not depend on tau or
    the norm, so each rule's answer is the iterate at its own first sub-tau
    iteration (or at its cap). This equals running :func:`pagerank` once per
    rule. Returns a list of :class:`Result` in tap order."""
    taps = [t if isinstance(t, Tap) else Tap(*t) for t in taps]
    cap = max(t.max_iter for t in taps)
    n = len(g.outdeg)
    r = np.full(n, 1.0 / n) if init is None else _f64(init).copy()
    done = [None] * len(taps)
    hist = []
    for i in range(1, cap + 1):
        s, _ = step(g, alpha, r, threads)
        nv = norms(s, r)
        hist.append(nv)
        r = s
        for k, t in enumerate(taps):
            if done[k] is None:
                e = float(nv[t.norm - 1])
                if e < t.tau:
                    done[k] = Result(r.copy(), i, e, True)
                elif i >= t.max_iter:
                    done[k] = Result(r.copy(), i, e, False)
        if all(d is not None for d in done):
            break
    h = np.array(hist)
    for d in done:
        d.err_hist = h[: d.iters]
    return done


# --------------------------------------------------------------------------
# Fixed point by a dense direct solve (small graphs)

def google_matrix(g) -> np.ndarray:
    """Column-stochastic P with P[v,u] = 1/d_u for every edge u->v, and column
    u uniform 1/N when u is dangling (Section 2: a surfer on a page without
    links jumps to a random page)."""
    n = len(g.outdeg)
    P = np.zeros((n, n), np.float64)
    od = np.asarray(g.outdeg)
    off = np.asarray(g.offsets)
    src = np.asarray(g.sources)
    for v in range(n):
        for e in range(off[v], off[v + 1]):
            u = src[e]
            P[v, u] += 1.0 / od[u]
    for u in range(n):
        if od[u] == 0:
            P[:, u] = 1.0 / n
    return P


def dense_solve(g, alpha: float) -> np.ndarray:
    """r = (1-alpha)/N + alpha P r solved directly: (I - alpha P) r = (1-alpha)/N.
    For alpha = 1 the last equation is replaced by sum(r) = 1."""
    n = len(g.outdeg)
    P = google_matrix(g)
    A = np.eye(n) - alpha * P
    b = np.full(n, (1.0 - alpha) / n)
    if alpha >= 1.0:
        A[-1, :] = 1.0
        b[-1] = 1.0
    return np.linalg.solve(A, b)


# --------------------------------------------------------------------------
# Section 1: iteration estimate and the six mean ratios

def estimate_iterations(tau: float, alpha: float) -> int:
    """Iterations to reach tau when the error shrinks like alpha^k (Section 1),
    rounded to the nearest integer."""
    return int(round(math.log10(tau) / math.log10(alpha)))


def am(x) -> float:
    x = np.asarray(x, np.float64)
    return float(x.sum() / x.size)


def gm(x) -> float:
    x = np.asarray(x, np.float64)
    return float(math.exp(np.log(x).sum() / x.size))


def hm(x) -> float:
    x = np.asarray(x, np.float64)
    return float(x.size / (1.0 / x).sum())


MEANS = {"AM": am, "GM": gm, "HM": hm}


def mean_ratio(kind: str, a, base) -> float:
    """X-RATIO: the X-mean of approach a over the X-mean of the baseline
    (mean first, ratio last; Section 1)."""
    f = MEANS[kind]
    return f(a) / f(base)


def ratio_mean(kind: str, a, base) -> float:
    """RATIO-X: the X-mean of the per-test ratios a_i / base_i (ratio first;
    Section 1)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(base, np.float64)
    return MEANS[kind](a / b)


def six_ratios(a, base) -> dict:
    out = {}
    for k in ("AM", "GM", "HM"):
        out[f"{k}-RATIO"] = mean_ratio(k, a, base)
        out[f"RATIO-{k}"] = ratio_mean(k, a, base)
    return out


# --------------------------------------------------------------------------
# Learned warm start (no counterpart in the paper): features and the MLP

def features(g, alpha: float) -> np.ndarray:
    """(N, 5) features: log(1+indeg), log(1+outdeg), mean and max of
    log(1+outdeg(u)) over in-neighbours u (0 when none), alpha."""
    lib = _load()
    off, src, od = _i32(g.offsets), _i32(g.sources), _i32(g.outdeg)
    n = od.shape[0]
    f = np.empty((n, 5), np.float64)
    lib.oracle_features(n, _ptr(off), _ptr(src), _ptr(od), alpha, f.ctypes.data)
    return f


def erf(x):
    from scipy.special import erf as _erf
    return _erf(x)


def gelu(x):
    """x * Phi(x), Phi the standard normal CDF (exact erf form)."""
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    phi = np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * phi


MLP_SHAPES = {"W1": (64, 5), "b1": (64,), "W2": (64, 64), "b2": (64,), "W3": (1, 64), "b3": (1,)}


def mlp_forward(F, p):
    """y = W3 gelu(W2 gelu(W1 f + b1) + b2) + b3 for every row f of F."""
    F = np.asarray(F, np.float64)
    z1 = F @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    y = h2 @ p["W3"].T + p["b3"]
    return y[:, 0], (F, z1, h1, z2, h2)


def mse_loss(y, t) -> float:
    d = np.asarray(y, np.float64) - np.asarray(t, np.float64)
    return float((d * d).sum() / d.size)


def mlp_backward(p, cache, y, t):
    """Gradients of the MSE loss mean((y - t)^2) with respect to every
    parameter, by the chain rule."""
    F, z1, h1, z2, h2 = cache
    m = F.shape[0]
    dy = (2.0 / m) * (np.asarray(y) - np.asarray(t))[:, None]        # (M,1)
    g = {}
    g["W3"] = dy.T @ h2
    g["b3"] = dy.sum(axis=0)
    dh2 = dy @ p["W3"]
    dz2 = dh2 * gelu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * gelu_grad(z1)
    g["W1"] = dz1.T @ F
    g["b1"] = dz1.sum(axis=0)
    return g


def adam_update(p, g, m, v, step_no: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam (Kingma and Ba, 2015) with bias correction, in place."""
    for k in p:
        m[k] = beta1 * m[k] + (1.0 - beta1) * g[k]
        v[k] = beta2 * v[k] + (1.0 - beta2) * g[k] * g[k]
        mh = m[k] / (1.0 - beta1 ** step_no)
        vh = v[k] / (1.0 - beta2 ** step_no)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p, m, v


def warm_start_from_logits(y) -> np.ndarray:
    """r0 = exp(y) / sum(exp(y)), computed with the maximum subtracted."""
    y = np.asarray(y, np.float64)
    e = np.exp(y - y.max())
    return e / e.sum()


def bf16_round(x) -> np.ndarray:
    """Round FP32 values to the nearest bfloat16 (ties to even), returned as
    float64. Used to feed the oracle the same weight values the GPU holds."""
    a = np.asarray(x, np.float32).copy()
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
