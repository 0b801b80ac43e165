"""Seeded synthetic graph inputs (ctypes binding of ``csrc/graphgen.c``).

Every generator returns a :class:`Graph`: an in-edge CSR (``offsets[v]`` ..
``offsets[v+1]`` index ``sources``, the tails u of the edges u -> v) and the
out-degree of every vertex. These are the inputs both the CPU oracle and the
CUDA library take. No PageRank arithmetic lives here.

Workload recipes (stand-ins for the paper's SuiteSparse graphs, Section 2):

* ``erdos_renyi_10k()`` — N = 10,000, 100,000 unique uniform non-self edges,
  500 vertices made dangling by deleting their out-edges (seed 1).
* ``rmat(scale)`` — R-MAT a/b/c/d = .57/.19/.19/.05, edge factor 16, ids
  randomly permuted, self-loops and duplicates removed.
* ``road_grid(rows, cols)`` — road-like lattice digraph (mean out-degree about
  2.9, at most 4), ids randomly permuted.
* ``config_model(n)`` — directed configuration model, power-law in/out degree
  with exponent 2.1 and mean close to 12.
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass

import numpy as np

from . import _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        so = _build.build_graphgen()
        lib = C.CDLL(str(so))
        vp = C.c_void_p
        lib.gg_graph_n.argtypes = [vp]; lib.gg_graph_n.restype = C.c_int32
        lib.gg_graph_nnz.argtypes = [vp]; lib.gg_graph_nnz.restype = C.c_int64
        lib.gg_graph_free.argtypes = [vp]; lib.gg_graph_free.restype = None
        lib.gg_graph_copy.argtypes = [vp, vp, vp, vp]; lib.gg_graph_copy.restype = C.c_int
        lib.gg_from_edges.argtypes = [C.c_int32, C.c_int64, vp, vp, C.POINTER(vp)]
        lib.gg_from_edges.restype = C.c_int
        lib.gg_rmat.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double,
                                C.c_uint64, C.c_int32, C.POINTER(vp)]
        lib.gg_rmat.restype = C.c_int
        lib.gg_erdos_renyi.argtypes = [C.c_int32, C.c_int64, C.c_int32, C.c_uint64, C.POINTER(vp)]
        lib.gg_road_grid.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_uint64, C.c_int32,
                                     C.POINTER(vp)]
        lib.gg_road_grid.restype = C.c_int
        lib.gg_erdos_renyi.restype = C.c_int
        lib.gg_config_model.argtypes = [C.c_int32, C.c_double, C.c_int32, C.c_int32, C.c_uint64,
                                        C.POINTER(vp)]
        lib.gg_config_model.restype = C.c_int
        lib.gg_draw.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]; lib.gg_draw.restype = C.c_uint64
        lib.gg_splitmix64.argtypes = [C.c_uint64, C.c_uint64]; lib.gg_splitmix64.restype = C.c_uint64
        _lib = lib
    return _lib


@dataclass
class Graph:
    """In-edge CSR plus out-degrees (all int32, host memory)."""
    offsets: np.ndarray   # n + 1
    sources: np.ndarray   # nnz
    outdeg: np.ndarray    # n
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.outdeg.shape[0])

    @property
    def nnz(self) -> int:
        return int(self.sources.shape[0])

    @property
    def indeg(self) -> np.ndarray:
        return np.diff(self.offsets).astype(np.int32)

    def edges(self):
        """(src, dst) arrays of every edge u -> v."""
        dst = np.repeat(np.arange(self.n, dtype=np.int32), self.indeg)
        return self.sources.copy(), dst


def _take(h, name) -> Graph:
    lib = _load()
    n = lib.gg_graph_n(h)
    nnz = lib.gg_graph_nnz(h)
    off = np.empty(n + 1, np.int32)
    src = np.empty(max(nnz, 0), np.int32)
    od = np.empty(n, np.int32)
    lib.gg_graph_copy(h, off.ctypes.data, src.ctypes.data if nnz else None, od.ctypes.data)
    lib.gg_graph_free(h)
    return Graph(off, src, od, name)


def _check(rc, what):
    if rc == 1:
        raise ValueError(f"{what}: invalid arguments")
    if rc == 2:
        raise MemoryError(f"{what}: out of host memory")
    if rc != 0:
        raise RuntimeError(f"{what}: error {rc}")


def from_edges(n: int, src, dst, name: str = "edges") -> Graph:
    """Graph from an explicit edge list; self-loops and duplicates dropped."""
    lib = _load()
    s = np.ascontiguousarray(np.asarray(src, dtype=np.int32))
    d = np.ascontiguousarray(np.asarray(dst, dtype=np.int32))
    if s.shape != d.shape:
        raise ValueError("src and dst must have the same length")
    h = C.c_void_p()
    _check(lib.gg_from_edges(int(n), int(s.size), s.ctypes.data if s.size else None,
                             d.ctypes.data if d.size else None, C.byref(h)), "from_edges")
    return _take(h, name)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 22, permute: bool = True) -> Graph:
    lib = _load()
    h = C.c_void_p()
    _check(lib.gg_rmat(scale, edge_factor, a, b, c, seed, 1 if permute else 0, C.byref(h)), "rmat")
    return _take(h, f"rmat-s{scale}-ef{edge_factor}-seed{seed}")


def erdos_renyi(n: int, m_unique: int, n_dangling: int, seed: int) -> Graph:
    lib = _load()
    h = C.c_void_p()
    _check(lib.gg_erdos_renyi(n, m_unique, n_dangling, seed, C.byref(h)), "erdos_renyi")
    return _take(h, f"er-n{n}-m{m_unique}-d{n_dangling}-seed{seed}")


def road_grid(rows: int, cols: int, p_keep: float = 0.8, p_oneway: float = 0.2, seed: int = 7,
              permute: bool = True) -> Graph:
    """Road-like lattice digraph: each right/down lattice link kept with
    probability p_keep, one-way with probability p_oneway (random direction),
    else two-way; mean out-degree 2 p_keep (2 - p_oneway) (2.88 by default)."""
    lib = _load()
    h = C.c_void_p()
    _check(lib.gg_road_grid(int(rows), int(cols), float(p_keep), float(p_oneway), int(seed), 1 if permute else 0,
                            C.byref(h)), "road_grid")
    return _take(h, f"road-{rows}x{cols}-seed{seed}")


def erdos_renyi_10k(seed: int = 1) -> Graph:
    """N = 10,000; 100,000 unique uniform non-self edges; 5% dangling."""
    return erdos_renyi(10_000, 100_000, 500, seed)


def power_law_kmin(n: int, gamma: float = 2.1, mean: float = 12.0) -> tuple[int, int]:
    """Integer k_min whose truncated power law on [k_min, sqrt(mean*n)] has the
    mean closest to ``mean``; returns (k_min, k_max)."""
    k_max = int(math.isqrt(int(mean * n)))
    best = None
    for k_min in range(1, 64):
        k = np.arange(k_min, k_max + 1, dtype=np.float64)
        w = k ** (-gamma)
        mu = float((k * w).sum() / w.sum())
        if best is None or abs(mu - mean) < best[0]:
            best = (abs(mu - mean), k_min)
    return best[1], k_max


def config_model(n: int = 8_000_000, gamma: float = 2.1, mean: float = 12.0, seed: int = 3008) -> Graph:
    lib = _load()
    k_min, k_max = power_law_kmin(n, gamma, mean)
    h = C.c_void_p()
    _check(lib.gg_config_model(n, gamma, k_min, k_max, seed, C.byref(h)), "config_model")
    return _take(h, f"cm-n{n}-g{gamma}-kmin{k_min}-seed{seed}")


def splitmix64(state: int, steps: int = 0) -> int:
    """Output number ``steps`` of a SplitMix64 generator with the given state."""
    return int(_load().gg_splitmix64(state, steps))


def draw(seed: int, stream: int, counter: int) -> int:
    return int(_load().gg_draw(seed, stream, counter))


def uniform(seed: int, stream: int, count: int) -> np.ndarray:
    """``count`` doubles in [0, 1) from the counter-based generator (host)."""
    lib = _load()
    out = np.empty(count, np.float64)
    for i in range(count):
        out[i] = (lib.gg_draw(seed, stream, i) >> 11) * (1.0 / 9007199254740992.0)
    return out


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """``count`` standard normals by the Box-Muller transform of uniform()."""
    u = uniform(seed, stream, 2 * count)
    u1 = 1.0 - u[0::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u[1::2])
