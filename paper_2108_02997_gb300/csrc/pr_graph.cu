// pr_graph.cu — device-resident graph: validation, relabelling, work units.
//
// The pull update of Section 2 needs, for every vertex v, its in-neighbours u
// and their out-degrees d_u. The graph arrives as an in-edge CSR in the
// caller's vertex order. It is relabelled so that vertices are grouped by
// in-degree class (floor(log2(indeg)), largest first) and, inside a class, by
// out-degree class (largest first), ties kept in caller order:
//   * rows of one class have in-degrees within a factor of two, so one lane
//     group size fits the whole class (load balance without per-row bins);
//   * on skewed graphs the vertices with the largest out-degree, whose
//     contributions are gathered most often, end up packed together at the
//     low ids, so their cache lines are shared instead of scattered.
// Rank vectors cross the ABI in caller order; the kernels map through perm.
#include <algorithm>
#include <cstring>
#include <new>

#include "pr_internal.cuh"

namespace {

int deg_class(int32_t d) {   // 0 for d = 0, else 1 + floor(log2 d)
    if (d <= 0) return 0;
    int c = 0;
    while (d) { c++; d >>= 1; }
    return c;
}

template <typename T>
pr_status dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            return pr_fail(PR_ENOMEM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
        }
        return pr_cuda_fail(e, "cudaMalloc");
    }
    return PR_OK;
}

void free_tables(pr_graph *g) {
    for (auto &t : g->tables) {
        cudaFree(t.d_tiles);
        cudaFree(t.d_slot_base);
        t = TileTable();
    }
}

void free_graph(pr_graph *g) {
    if (!g) return;
    cudaFree(g->d_off);
    cudaFree(g->d_src);
    cudaFree(g->d_outdeg);
    cudaFree(g->d_perm);
    cudaFree(g->d_inv);
    free_tables(g);
    g->magic = 0;
    delete g;
}

}  // namespace

int w_index(int W) {
    switch (W) {
        case 1: return 0;
        case 2: return 1;
        case 4: return 2;
        case 8: return 3;
        case 16: return 4;
        case 32: return 5;
        default: return -1;
    }
}

bool pr_graph_valid(const pr_graph *g) { return g && registry_has(g) && g->magic == kGraphMagic; }

// Tiles of width W (see Tile in pr_internal.cuh). Rows of one in-degree class
// are packed into warp tiles of at most tile_rows(W) rows and tile_edges(W)
// in-edges; a group of es lanes shares one row when the row sums are formed
// (each lane adds every W columns of its in-edges, or every vec_cols of them
// per column group), es sized so that each lane adds about four in-edges.
// Classes with rows longer than tile_edges(W) are cut into chunks of
// chunk_edges(W) in-edges, each chunk a warp's tile.
pr_status pr_graph_tiles(pr_graph *g, int W, const TileTable **out) {
    int wi = w_index(W);
    if (wi < 0) return pr_fail(PR_EINVAL, "unsupported column width");
    TileTable &t = g->tables[wi];
    if (t.d_tiles) {
        *out = &t;
        return PR_OK;
    }
    const int TE = tile_edges(W), TR = tile_rows(W), CH = chunk_edges(W);
    const int max_es = 32;
    std::vector<Tile> tiles;
    std::vector<int32_t> slot_base;
    int32_t n_chunk_slots = 0;
    double work = 0.0;
    const std::vector<int32_t> &off = g->h_off;
    for (const ClassRange &cr : g->classes) {
        if (cr.end <= cr.begin) continue;
        if (cr.max_deg > TE) {
            for (int32_t v = cr.begin; v < cr.end; v++) {
                int32_t e0 = off[v], e1 = off[v + 1];
                int32_t deg = e1 - e0;
                int32_t nch = std::max<int32_t>(1, (deg + CH - 1) / CH);
                int32_t slot = -1;
                if (nch > 1) {
                    slot = (int32_t)slot_base.size();
                    slot_base.push_back(n_chunk_slots);
                    n_chunk_slots += nch;
                }
                for (int32_t k = 0; k < nch; k++) {
                    int32_t a = e0 + k * CH, b = std::min(e1, a + CH);
                    tiles.push_back({v, v + 1, a, b, -1, slot, k, nch});
                }
                work += (double)deg * W + W * 4.0;
            }
            continue;
        }
        int es = 1;
        while (es < max_es && es * 4 < cr.max_deg) es <<= 1;
        int glog = 0;
        while ((1 << glog) < es) glog++;
        int32_t r = cr.begin;
        while (r < cr.end) {
            int32_t r1 = r;
            while (r1 < cr.end && r1 - r < TR && off[r1 + 1] - off[r] <= TE) r1++;
            if (r1 == r) r1 = r + 1;   // cannot happen (deg <= TE), kept for safety
            tiles.push_back({r, r1, off[r], off[r1], glog, -1, 0, 0});
            work += (double)(off[r1] - off[r]) * W + (double)(r1 - r) * W * 4.0;
            r = r1;
        }
    }
    TileTable nt;
    nt.W = W;
    nt.ntiles = (int32_t)tiles.size();
    nt.n_long = (int32_t)slot_base.size();
    nt.n_chunk_slots = n_chunk_slots;
    nt.work = work;
    pr_status s = dalloc(&nt.d_tiles, tiles.size());
    if (s != PR_OK) return s;
    s = dalloc(&nt.d_slot_base, slot_base.size());
    if (s != PR_OK) { cudaFree(nt.d_tiles); return s; }
    cudaError_t e = cudaSuccess;
    if (!tiles.empty())
        e = cudaMemcpy(nt.d_tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !slot_base.empty())
        e = cudaMemcpy(nt.d_slot_base, slot_base.data(), slot_base.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(nt.d_tiles);
        cudaFree(nt.d_slot_base);
        return pr_cuda_fail(e, "cudaMemcpy tiles");
    }
    t = nt;
    *out = &t;
    return PR_OK;
}

namespace {

// Device validation of the in-edge sources: every source in [0, n), and the
// number of times each vertex occurs equal to its out-degree. Records the
// smallest offending edge / vertex index (or INT64_MAX when none).
__global__ void count_sources_kernel(const int32_t *__restrict__ src, int64_t nnz, int32_t n, int32_t *count,
                                     unsigned long long *bad_edge) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = src[e];
        if (u < 0 || u >= n) atomicMin(bad_edge, (unsigned long long)e);
        else atomicAdd(&count[u], 1);
    }
}
__global__ void check_outdeg_kernel(const int32_t *__restrict__ count, const int32_t *__restrict__ outdeg, int32_t n,
                                    unsigned long long *bad_vertex) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        if (count[v] != outdeg[v]) atomicMin(bad_vertex, (unsigned long long)v);
}
// Relabelled rows: row i of the new CSR is caller row perm[i], its sources
// mapped through inv. One warp per row.
__global__ void remap_rows_kernel(const int32_t *__restrict__ old_off, const int32_t *__restrict__ old_src,
                                  const int32_t *__restrict__ new_off, const int32_t *__restrict__ perm,
                                  const int32_t *__restrict__ inv, int32_t n, int32_t *__restrict__ new_src) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < n; i += nw) {
        const int32_t v = perm[i];
        const int32_t a = old_off[v], len = old_off[v + 1] - a, o = new_off[i];
        for (int32_t k = lane; k < len; k += 32) new_src[o + k] = inv[old_src[a + k]];
    }
}

int blocks_for(int64_t work, int threads) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t want = (work + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 16));
}

struct DevTmp {
    void *p = nullptr;
    ~DevTmp() { if (p) cudaFree(p); }
};

}  // namespace

// Graph creation. The host does the O(n) work (offset checks, the
// relabelling sort, new offsets, class ranges and tile tables); the device does
// the O(nnz) work (validation of every source and the remapped copy of the rows).
extern "C" pr_status pr_graph_create(int32_t n, int64_t nnz, const int32_t *in_offsets,
                                     const int32_t *in_sources, const int32_t *out_degree, pr_graph **out) {
    pr_clear_error();
    if (!out) return pr_fail(PR_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1) return pr_fail(PR_EINVAL, "n must be >= 1");
    if (nnz < 0 || nnz >= (int64_t)INT32_MAX) return pr_fail(PR_EINVAL, "nnz must be in [0, 2^31-1)");
    if (!in_offsets || !out_degree) return pr_fail(PR_EINVAL, "in_offsets and out_degree are required");
    if (nnz > 0 && !in_sources) return pr_fail(PR_EINVAL, "in_sources is NULL but nnz > 0");
    // ---- O(n) checks on the host
    if (in_offsets[0] != 0) return pr_fail(PR_EINVAL, "in_offsets[0] must be 0");
    if ((int64_t)in_offsets[n] != nnz) return pr_fail(PR_EINVAL, "in_offsets[n] must equal nnz");
    int64_t deg_sum = 0;
    int32_t n_dangling = 0;
    for (int32_t v = 0; v < n; v++) {
        if (in_offsets[v + 1] < in_offsets[v]) return pr_fail(PR_EINVAL, "in_offsets is not non-decreasing at row " + std::to_string(v));
        if (out_degree[v] < 0) return pr_fail(PR_EINVAL, "out_degree[" + std::to_string(v) + "] is negative");
        deg_sum += out_degree[v];
        if (out_degree[v] == 0) n_dangling++;
    }
    if (deg_sum != nnz) return pr_fail(PR_EINVAL, "out_degree does not sum to nnz (it must match the edges in in_sources)");
    // ---- caller arrays on the device, sources validated there
    DevTmp d_old_off, d_old_src, d_cnt, d_bad;
    cudaError_t e = cudaSuccess;
    const size_t n_off = (size_t)n + 1 + kPad, n_src = (size_t)nnz + kPad, n_od = (size_t)n + kPad;
    pr_graph *g = new (std::nothrow) pr_graph();
    if (!g) return pr_fail(PR_ENOMEM, "host allocation failed");
    g->magic = kGraphMagic;
    g->n = n;
    g->nnz = nnz;
    g->n_dangling = n_dangling;
    cudaGetDevice(&g->device);
    pr_status s;
    if ((s = dalloc(&g->d_off, n_off)) != PR_OK || (s = dalloc(&g->d_src, n_src)) != PR_OK ||
        (s = dalloc(&g->d_outdeg, n_od)) != PR_OK || (s = dalloc(&g->d_perm, (size_t)n)) != PR_OK ||
        (s = dalloc(&g->d_inv, (size_t)n)) != PR_OK) {
        free_graph(g);
        return s;
    }
    e = cudaMalloc(&d_old_off.p, sizeof(int32_t) * ((size_t)n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&d_old_src.p, sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1));
    if (e == cudaSuccess) e = cudaMalloc(&d_cnt.p, sizeof(int32_t) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&d_bad.p, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpy(d_old_off.p, in_offsets, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nnz > 0) e = cudaMemcpy(d_old_src.p, in_sources, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(d_cnt.p, 0, sizeof(int32_t) * (size_t)n);
    if (e == cudaSuccess) e = cudaMemset(d_bad.p, 0xFF, 2 * sizeof(unsigned long long));
    // the caller's out-degrees go straight into the final array's scratch use: copy to d_outdeg first
    if (e == cudaSuccess) e = cudaMemcpy(g->d_outdeg, out_degree, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_graph(g);
        return pr_cuda_fail(e, "graph upload");
    }
    unsigned long long *bad = static_cast<unsigned long long *>(d_bad.p);
    if (nnz > 0)
        count_sources_kernel<<<blocks_for(nnz, 256), 256>>>(static_cast<const int32_t *>(d_old_src.p), nnz, n,
                                                            static_cast<int32_t *>(d_cnt.p), bad);
    check_outdeg_kernel<<<blocks_for(n, 256), 256>>>(static_cast<const int32_t *>(d_cnt.p), g->d_outdeg, n, bad + 1);
    unsigned long long hbad[2] = {~0ull, ~0ull};
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        free_graph(g);
        return pr_cuda_fail(e, "graph validation");
    }
    if (hbad[0] != ~0ull) {
        free_graph(g);
        return pr_fail(PR_EINVAL, "in_sources[" + std::to_string(hbad[0]) + "] out of range");
    }
    if (hbad[1] != ~0ull) {
        free_graph(g);
        return pr_fail(PR_EINVAL, "out_degree[" + std::to_string(hbad[1]) + "] does not match the edges in in_sources");
    }
    // ---- relabel on the host: stable counting sort by (in-class desc, out-class desc), O(n)
    std::vector<int32_t> perm, inv, new_off, new_od, tmp;
    try {
        perm.resize((size_t)n);
        inv.resize((size_t)n);
        tmp.resize((size_t)n);
        new_off.resize((size_t)n + 1);
        new_od.resize((size_t)n);
    } catch (const std::bad_alloc &) {
        free_graph(g);
        return pr_fail(PR_ENOMEM, "host allocation failed");
    }
    {
        size_t cnt[33];
        std::memset(cnt, 0, sizeof(cnt));
        for (int32_t v = 0; v < n; v++) cnt[32 - deg_class(out_degree[v])]++;
        size_t acc = 0;
        for (int b = 0; b < 33; b++) { size_t c = cnt[b]; cnt[b] = acc; acc += c; }
        for (int32_t v = 0; v < n; v++) tmp[cnt[32 - deg_class(out_degree[v])]++] = v;
        std::memset(cnt, 0, sizeof(cnt));
        for (int32_t v = 0; v < n; v++) cnt[32 - deg_class(in_offsets[v + 1] - in_offsets[v])]++;
        acc = 0;
        for (int b = 0; b < 33; b++) { size_t c = cnt[b]; cnt[b] = acc; acc += c; }
        for (int32_t i = 0; i < n; i++) {
            const int32_t v = tmp[i];
            perm[cnt[32 - deg_class(in_offsets[v + 1] - in_offsets[v])]++] = v;
        }
    }
    new_off[0] = 0;
    for (int32_t i = 0; i < n; i++) {
        const int32_t v = perm[i];
        inv[v] = i;
        new_off[i + 1] = new_off[i] + (in_offsets[v + 1] - in_offsets[v]);
        new_od[i] = out_degree[v];
    }
    {
        int32_t i = 0;
        while (i < n) {
            const int c = deg_class(new_off[i + 1] - new_off[i]);
            ClassRange cr{i, i, 0};
            while (i < n && deg_class(new_off[i + 1] - new_off[i]) == c) {
                cr.max_deg = std::max(cr.max_deg, new_off[i + 1] - new_off[i]);
                i++;
            }
            cr.end = i;
            g->classes.push_back(cr);
        }
    }
    // ---- relabelled arrays on the device (padding zeroed), rows remapped there
    e = cudaMemset(g->d_off, 0, sizeof(int32_t) * n_off);
    if (e == cudaSuccess) e = cudaMemset(g->d_src, 0, sizeof(int32_t) * n_src);
    if (e == cudaSuccess) e = cudaMemset(g->d_outdeg, 0, sizeof(int32_t) * n_od);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_off, new_off.data(), sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_outdeg, new_od.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_perm, perm.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_inv, inv.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nnz > 0) {
        remap_rows_kernel<<<blocks_for((int64_t)n * 32, 256), 256>>>(static_cast<const int32_t *>(d_old_off.p),
                                                                     static_cast<const int32_t *>(d_old_src.p), g->d_off,
                                                                     g->d_perm, g->d_inv, n, g->d_src);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_graph(g);
        return pr_cuda_fail(e, "graph relabel");
    }
    // signature for caches keyed by graph shape: FNV-1a over n, nnz and each
    // in-degree class's (first row, end row, largest in-degree, edges)
    {
        uint64_t h = 1469598103934665603ull;
        auto mix = [&h](uint64_t x) {
            for (int b = 0; b < 8; b++) {
                h ^= (x >> (8 * b)) & 0xffu;
                h *= 1099511628211ull;
            }
        };
        mix((uint64_t)n);
        mix((uint64_t)nnz);
        for (const ClassRange &cr : g->classes) {
            mix((uint64_t)cr.begin);
            mix((uint64_t)cr.end);
            mix((uint64_t)cr.max_deg);
            mix((uint64_t)(new_off[cr.end] - new_off[cr.begin]));
        }
        g->signature = h;
    }
    g->h_off.swap(new_off);
    // the single-column work table is built now so that solves on this graph
    // never need to allocate it later
    const TileTable *t1 = nullptr;
    if ((s = pr_graph_tiles(g, 1, &t1)) != PR_OK) {
        free_graph(g);
        return s;
    }
    registry_add(g);
    *out = g;
    return PR_OK;
}

extern "C" pr_status pr_graph_destroy(pr_graph *g) {
    pr_clear_error();
    if (!g) return PR_OK;
    if (!pr_graph_valid(g)) return pr_fail(PR_ESTATE, "not a live graph handle");
    registry_remove(g);
    free_graph(g);
    return PR_OK;
}

extern "C" pr_status pr_graph_info(const pr_graph *g, int32_t *n, int64_t *nnz, int32_t *n_dangling) {
    pr_clear_error();
    if (!pr_graph_valid(g)) return pr_fail(PR_ESTATE, "not a live graph handle");
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    if (n_dangling) *n_dangling = g->n_dangling;
    return PR_OK;
}
