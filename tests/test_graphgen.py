"""Input generators: published RNG test vectors, graph invariants, determinism."""
import numpy as np
import pytest


def test_splitmix64_published_vectors(gg):
    # SplitMix64 (Steele, Lea, Flood 2014; reference implementation by Vigna):
    # state 0 -> first output 0xE220A8397B1DCDAF; state 1234567 -> the sequence below.
    assert gg.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert [gg.splitmix64(1234567, i) for i in range(3)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423]


def _check_csr(g):
    assert g.offsets[0] == 0 and g.offsets[-1] == g.nnz
    assert np.all(np.diff(g.offsets) >= 0)
    src, dst = g.edges()
    assert np.all((src >= 0) & (src < g.n))
    assert not np.any(src == dst), "self-loop left in graph"
    key = dst.astype(np.int64) * g.n + src
    assert np.unique(key).size == key.size, "duplicate edge left in graph"
    assert np.array_equal(np.bincount(src, minlength=g.n), g.outdeg)


def test_erdos_renyi_10k(gg):
    g = gg.erdos_renyi_10k(seed=1)
    _check_csr(g)
    assert g.n == 10_000
    # 100,000 unique edges before deleting the out-edges of 500 vertices
    assert 90_000 < g.nnz < 100_000
    assert (g.outdeg == 0).sum() >= 500
    g2 = gg.erdos_renyi_10k(seed=1)
    assert np.array_equal(g.sources, g2.sources) and np.array_equal(g.offsets, g2.offsets)
    g3 = gg.erdos_renyi_10k(seed=2)
    assert not np.array_equal(g.sources[:100], g3.sources[:100])


def test_rmat_small(gg):
    g = gg.rmat(12, 16, seed=7)
    _check_csr(g)
    assert g.n == 4096
    assert 0.5 * 16 * 4096 < g.nnz <= 16 * 4096
    # skewed: the largest in-degree far above the mean
    assert g.indeg.max() > 20 * g.indeg.mean()
    g2 = gg.rmat(12, 16, seed=7)
    assert np.array_equal(g.sources, g2.sources)


def test_rmat_unpermuted_hub_is_vertex_zero(gg):
    # Without relabelling, a=.57 makes vertex 0 the top in-degree vertex.
    g = gg.rmat(10, 16, seed=3, permute=False)
    assert int(np.argmax(g.indeg)) == 0
    assert int(np.argmax(g.outdeg)) == 0


def test_from_edges_cleans(gg):
    g = gg.from_edges(4, [0, 0, 1, 2, 2, 3], [1, 1, 1, 0, 3, 3])
    _check_csr(g)
    assert g.nnz == 3  # 0->1, 2->0, 2->3 (duplicate and two self-loops dropped)
    with pytest.raises(ValueError):
        gg.from_edges(3, [0], [5])


def test_config_model_small(gg):
    g = gg.config_model(20_000, seed=11)
    _check_csr(g)
    mean = g.nnz / g.n
    assert 6 < mean < 14


def test_road_grid_shape(gg):
    g = gg.road_grid(200, 300, seed=5)
    assert g.n == 60000
    src, dst = g.edges()
    assert np.all(src != dst)
    assert np.unique(dst.astype(np.int64) * g.n + src).size == g.nnz        # no duplicates
    assert g.outdeg.max() <= 4 and g.indeg.max() <= 4
    # links kept with p = 0.8, two-way with p = 0.8: about 2 * 0.8 * 1.8 = 2.88 per vertex
    assert abs(g.nnz / g.n - 2.88) < 0.05
    # unpermuted: every edge joins lattice neighbours
    h = gg.road_grid(40, 50, seed=5, permute=False)
    s, d = h.edges()
    di, dj = np.abs(s // 50 - d // 50), np.abs(s % 50 - d % 50)
    assert np.all(di + dj == 1)
    # deterministic in the seed
    assert np.array_equal(gg.road_grid(40, 50, seed=5, permute=False).sources, h.sources)
