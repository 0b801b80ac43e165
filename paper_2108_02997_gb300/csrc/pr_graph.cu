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
#include <system_error>
#include <thread>
#include <new>

#include "pr_internal.cuh"

namespace {

void free_tables(pr_graph *g) {
    for (auto &t : g->tables) {
        pr_graph_free(t.d_mem, t.d_mem_pooled);
        t = TileTable();
    }
    for (auto &t : g->hub_tables) {
        pr_graph_free(t.d_mem, t.d_mem_pooled);
        t = TileTable();
    }
}

void free_graph(pr_graph *g) {
    if (!g) return;
    pr_graph_free(g->d_mem, g->d_mem_pooled);
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
namespace {

// Temporary device buffer of graph creation, taken from the stream-ordered
// workspace pool on the default stream, so that repeated creations reuse the
// memory instead of paying cudaMalloc and a synchronising cudaFree.
struct DevTmp {
    PoolBuf b;
    void *p = nullptr;
    cudaError_t alloc(size_t bytes) {
        if (b.alloc(bytes, 0) != PR_OK) return cudaErrorMemoryAllocation;
        p = b.p;
        return cudaSuccess;
    }
};

// Tile builder segment: rows [r0, r1) of one in-degree class, tiled
// independently of the other segments (a rows tile never spans two segments;
// a row's sum does not depend on the tile it sits in). glog >= 0: rows tiles
// with 2^glog lanes per row; -1: the class's rows are cut into chunks.
struct TileSeg {
    int32_t r0, r1, glog;
};
constexpr int32_t kSegRows = 1024;

// One warp per segment. Pass 1 (kWrite = false) counts the segment's tiles,
// chunk partial slots and long rows (cnt, 3 per segment); pass 2 writes them
// from the segment's exclusive sums (base, 3 per segment): tiles in row order,
// and for every row cut into several chunks its long-row index (the chunks'
// slot) and its first chunk partial (slot_base). Rows tiles are the greedy
// runs (extend while the tile keeps at most TR rows and TE in-edges); the
// lanes test 32 candidate rows at once and a ballot gives the run length.
// Chunked rows take 32 rows at a time with warp prefix sums.
template <bool kWrite>
__global__ void tile_segments_kernel(const TileSeg *__restrict__ segs, int32_t nseg, const int32_t *__restrict__ off,
                                     int TE, int TR, int CH, int32_t *__restrict__ cnt,
                                     const int64_t *__restrict__ base, Tile *__restrict__ tiles,
                                     int32_t *__restrict__ slot_base) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= nseg) return;   // whole warps
    const TileSeg sg = segs[i];
    int64_t nt = 0, ns = 0, nl = 0;   // the same in every lane
    const int64_t t0 = kWrite ? base[3 * i] : 0;
    const int64_t s0 = kWrite ? base[3 * i + 1] : 0;
    const int64_t l0 = kWrite ? base[3 * i + 2] : 0;
    if (sg.glog < 0) {
        for (int32_t v0 = sg.r0; v0 < sg.r1; v0 += 32) {
            const int32_t v = v0 + lane;
            int32_t e0 = 0, e1 = 0, nch = 0;
            if (v < sg.r1) {
                e0 = off[v];
                e1 = off[v + 1];
                nch = max(1, (e1 - e0 + CH - 1) / CH);
            }
            const int32_t lg = nch > 1 ? 1 : 0, sl = nch > 1 ? nch : 0;
            int32_t a_t = nch, a_l = lg, a_s = sl;   // inclusive prefix sums over the lanes
            for (int m = 1; m < 32; m <<= 1) {
                const int32_t x_t = __shfl_up_sync(0xffffffffu, a_t, m);
                const int32_t x_l = __shfl_up_sync(0xffffffffu, a_l, m);
                const int32_t x_s = __shfl_up_sync(0xffffffffu, a_s, m);
                if (lane >= m) {
                    a_t += x_t;
                    a_l += x_l;
                    a_s += x_s;
                }
            }
            if (kWrite && v < sg.r1) {
                int32_t slot = -1;
                if (lg) {
                    slot = (int32_t)(l0 + nl + a_l - 1);
                    slot_base[slot] = (int32_t)(s0 + ns + a_s - sl);
                }
                const int64_t at = t0 + nt + a_t - nch;
                for (int32_t k = 0; k < nch; k++) {
                    const int32_t a = e0 + k * CH;
                    tiles[at + k] = Tile{v, v + 1, a, min(e1, a + CH), -1, slot, k, nch};
                }
            }
            nt += __shfl_sync(0xffffffffu, a_t, 31);
            nl += __shfl_sync(0xffffffffu, a_l, 31);
            ns += __shfl_sync(0xffffffffu, a_s, 31);
        }
    } else {
        int32_t r = sg.r0;
        while (r < sg.r1) {
            const int32_t e0 = off[r];
            int32_t r1 = r;
            for (;;) {
                const int32_t row = r1 + lane;
                const bool ok = row < sg.r1 && row - r < TR && off[row + 1] - e0 <= TE;
                const unsigned int m = __ballot_sync(0xffffffffu, ok);
                const int run = m == 0xffffffffu ? 32 : __ffs(~m) - 1;   // the conditions only turn false
                r1 += run;
                if (run < 32) break;
            }
            if (r1 == r) r1 = r + 1;   // cannot happen (in-degree <= TE), kept for safety
            if (kWrite && lane == 0) tiles[t0 + nt] = Tile{r, r1, e0, off[r1], sg.glog, -1, 0, 0};
            nt++;
            r = r1;
        }
    }
    if (!kWrite && lane == 0) {
        cnt[3 * i] = (int32_t)nt;
        cnt[3 * i + 1] = (int32_t)ns;
        cnt[3 * i + 2] = (int32_t)nl;
    }
}

}  // namespace

// Work table of width W, built on the device from the relabelled offsets:
// classes whose rows fit a rows tile (at most tile_edges(W) in-edges) get
// rows tiles of consecutive rows (at most tile_rows(W) rows and
// tile_edges(W) in-edges each), lanes per row the smallest power of two
// (at most 32) with four in-edges per lane for the class's longest row; the
// other classes get chunks of chunk_edges(W) in-edges per row.
namespace {

pr_status build_tile_table(pr_graph *g, int W, int TE, int TR, int CH, TileTable &t) {
    const int max_es = 32;
    std::vector<TileSeg> segs;
    try {
        for (const ClassRange &cr : g->classes) {
            int glog = -1;
            if (cr.max_deg <= TE) {
                int es = 1;
                while (es < max_es && es * 4 < cr.max_deg) es <<= 1;
                glog = 0;
                while ((1 << glog) < es) glog++;
            }
            for (int32_t r = cr.begin; r < cr.end; r += kSegRows)
                segs.push_back(TileSeg{r, (int32_t)std::min<int64_t>((int64_t)r + kSegRows, cr.end), glog});
        }
    } catch (const std::bad_alloc &) {
        return pr_fail(PR_ENOMEM, "host allocation failed");
    }
    const int32_t nseg = (int32_t)segs.size();
    std::vector<int32_t> cnt((size_t)nseg * 3 + 3, 0);
    std::vector<int64_t> base((size_t)nseg * 3 + 3, 0);
    DevTmp d_segs, d_cnt, d_base;
    cudaError_t e = d_segs.alloc(sizeof(TileSeg) * (size_t)std::max(nseg, 1));
    if (e == cudaSuccess) e = d_cnt.alloc(sizeof(int32_t) * cnt.size());
    if (e == cudaSuccess) e = d_base.alloc(sizeof(int64_t) * base.size());
    if (e == cudaSuccess && nseg > 0)
        e = cudaMemcpy(d_segs.p, segs.data(), sizeof(TileSeg) * (size_t)nseg, cudaMemcpyHostToDevice);
    const int blocks = std::max(1, (int)(((int64_t)nseg * 32 + 127) / 128));   // a warp per segment
    if (e == cudaSuccess && nseg > 0) {
        tile_segments_kernel<false><<<blocks, 128>>>(static_cast<const TileSeg *>(d_segs.p), nseg, g->d_off, TE, TR, CH,
                                                     static_cast<int32_t *>(d_cnt.p), nullptr, nullptr, nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(cnt.data(), d_cnt.p, sizeof(int32_t) * (size_t)nseg * 3, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return pr_cuda_fail(e, "tile table (count)");
    int64_t tot[3] = {0, 0, 0};
    for (int32_t i = 0; i < nseg; i++)
        for (int c = 0; c < 3; c++) {
            base[3 * (size_t)i + c] = tot[c];
            tot[c] += cnt[3 * (size_t)i + c];
        }
    if (tot[0] > INT32_MAX || tot[1] > INT32_MAX) return pr_fail(PR_EINVAL, "graph needs more than 2^31 work tiles");
    TileTable nt;
    nt.W = W;
    nt.ntiles = (int32_t)tot[0];
    nt.n_chunk_slots = (int32_t)tot[1];
    nt.n_long = (int32_t)tot[2];
    // every row adds its in-edges and a fixed per-row cost, W columns each
    nt.work = ((double)g->nnz + 4.0 * (double)g->n) * W;
    // tiles and long-row slot bases in one allocation
    const size_t tiles_bytes = ((sizeof(Tile) * (size_t)std::max(nt.ntiles, 1)) + 255) & ~size_t(255);
    void *vmem = nullptr;
    bool pooled = false;
    pr_status s = pr_graph_alloc(&vmem, tiles_bytes + sizeof(int32_t) * (size_t)std::max(nt.n_long, 1), &pooled);
    if (s != PR_OK) return s;
    unsigned char *mem = static_cast<unsigned char *>(vmem);
    nt.d_mem = mem;
    nt.d_mem_pooled = pooled;
    nt.d_tiles = reinterpret_cast<Tile *>(mem);
    nt.d_slot_base = reinterpret_cast<int32_t *>(mem + tiles_bytes);
    e = cudaMemcpy(d_base.p, base.data(), sizeof(int64_t) * (size_t)nseg * 3, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nseg > 0) {
        tile_segments_kernel<true><<<blocks, 128>>>(static_cast<const TileSeg *>(d_segs.p), nseg, g->d_off, TE, TR, CH,
                                                    nullptr, static_cast<const int64_t *>(d_base.p), nt.d_tiles,
                                                    nt.d_slot_base);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        pr_graph_free(nt.d_mem, nt.d_mem_pooled);
        return pr_cuda_fail(e, "tile table (write)");
    }
    t = nt;
    return PR_OK;
}

}  // namespace

pr_status pr_graph_tiles(pr_graph *g, int W, const TileTable **out) {
    int wi = w_index(W);
    if (wi < 0) return pr_fail(PR_EINVAL, "unsupported column width");
    TileTable &t = g->tables[wi];
    if (!t.d_tiles) {
        pr_status s = build_tile_table(g, W, tile_edges(W), tile_rows(W), chunk_edges(W), t);
        if (s != PR_OK) return s;
    }
    *out = &t;
    return PR_OK;
}

// The hub gather kernel (one, two or four columns) stages hub_tile_edges(W)
// vectors per warp, so its rows tiles have a size of their own.
pr_status pr_graph_hub_tiles(pr_graph *g, int W, const TileTable **out) {
    if (W != 1 && W != 2 && W != 4) return pr_fail(PR_EINVAL, "internal: hub tiles for one, two or four columns");
    TileTable &t = g->hub_tables[w_index(W)];
    if (!t.d_tiles) {
        pr_status s = build_tile_table(g, W, hub_tile_edges(W), tile_rows(1), chunk_edges(1), t);
        if (s != PR_OK) return s;
    }
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
// mapped through inv: one warp per row for rows of 32 to 1023 in-edges, one
// thread per row below (the relabelling orders rows by in-degree class, longest
// first; the longest rows get a CTA each, remap_hub_rows_kernel).
// Rows of 1024 or more in-edges (first in the new order): one CTA per row.
__global__ void remap_hub_rows_kernel(const int32_t *__restrict__ old_off, const int32_t *__restrict__ old_src,
                                      const int32_t *__restrict__ new_off, const int32_t *__restrict__ perm,
                                      const int32_t *__restrict__ inv, int32_t n_hub, int32_t *__restrict__ new_src) {
    for (int32_t i = blockIdx.x; i < n_hub; i += gridDim.x) {
        const int32_t v = perm[i];
        const int32_t a = old_off[v], len = old_off[v + 1] - a, o = new_off[i];
        for (int32_t k = threadIdx.x; k < len; k += blockDim.x) new_src[o + k] = inv[old_src[a + k]];
    }
}
__global__ void remap_short_rows_kernel(const int32_t *__restrict__ old_off, const int32_t *__restrict__ old_src,
                                        const int32_t *__restrict__ new_off, const int32_t *__restrict__ perm,
                                        const int32_t *__restrict__ inv, int32_t i0, int32_t n,
                                        int32_t *__restrict__ new_src) {
    for (int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = perm[i];
        const int32_t a = old_off[v], len = old_off[v + 1] - a, o = new_off[i];
        for (int32_t k = 0; k < len; k++) new_src[o + k] = inv[old_src[a + k]];
    }
}
__global__ void remap_rows_kernel(const int32_t *__restrict__ old_off, const int32_t *__restrict__ old_src,
                                  const int32_t *__restrict__ new_off, const int32_t *__restrict__ perm,
                                  const int32_t *__restrict__ inv, int32_t i0, int32_t n, int32_t *__restrict__ new_src) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = i0 + w0; i < n; i += nw) {
        const int32_t v = perm[i];
        const int32_t a = old_off[v], len = old_off[v + 1] - a, o = new_off[i];
        for (int32_t k = lane; k < len; k += 32) new_src[o + k] = inv[old_src[a + k]];
    }
}

// ---------------------------------------------------------------- device relabelling
// Sort key of a vertex: in-degree class descending, then out-degree class
// descending (classes 0..32: 0 for degree 0, else 1 + floor(log2 d)). The
// relabelled order is the stable sort by key (ties by caller id).
constexpr int kClasses = 33;
constexpr int kKeys = kClasses * kClasses;
constexpr int kSortChunk = 2048;     // vertices per CTA of the counting sort
constexpr int kSortThreads = 256;

__device__ __forceinline__ int dev_class(int32_t d) { return d > 0 ? 32 - __clz(d) : 0; }

// Keys, and the largest in-degree of every in-degree class.
__global__ void class_keys_kernel(const int32_t *__restrict__ off, const int32_t *__restrict__ outdeg, int32_t n,
                                  int32_t *__restrict__ key, int32_t *__restrict__ class_max) {
    __shared__ int32_t s_max[kClasses];
    for (int i = threadIdx.x; i < kClasses; i += blockDim.x) s_max[i] = 0;
    __syncthreads();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t din = off[v + 1] - off[v];
        const int cin = dev_class(din), cout = dev_class(outdeg[v]);
        key[v] = (32 - cin) * kClasses + (32 - cout);
        atomicMax(&s_max[cin], din);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kClasses; i += blockDim.x)
        if (s_max[i] > 0) atomicMax(&class_max[i], s_max[i]);
}

// Per chunk of kSortChunk vertices, the count of every key: M[key * nchunks + chunk].
__global__ void __launch_bounds__(kSortThreads) chunk_hist_kernel(const int32_t *__restrict__ key, int32_t n,
                                                                  int32_t nchunks, int32_t *__restrict__ M) {
    __shared__ int32_t h[kKeys];
    const int chunk = blockIdx.x;
    for (int i = threadIdx.x; i < kKeys; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t v0 = (int64_t)chunk * kSortChunk;
    for (int i = threadIdx.x; i < kSortChunk; i += blockDim.x) {
        const int64_t v = v0 + i;
        if (v < n) atomicAdd(&h[key[v]], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kKeys; i += blockDim.x) M[(int64_t)i * nchunks + chunk] = h[i];
}

// Stable scatter: a vertex goes to (first slot of its key in its chunk) + (the
// vertices of the same key before it in the chunk). The chunk is walked in
// rounds of 256 consecutive vertices; within a round, lanes of equal key find
// their order by warp match, warps in order through per-warp key counts.
__global__ void __launch_bounds__(kSortThreads) chunk_scatter_kernel(const int32_t *__restrict__ key, int32_t n,
                                                                     int32_t nchunks, const int32_t *__restrict__ Mscan,
                                                                     int32_t *__restrict__ perm, int32_t *__restrict__ inv) {
    constexpr int kW = kSortThreads / 32;
    __shared__ int32_t running[kKeys];
    __shared__ int32_t wcnt[kW][kKeys];
    const int chunk = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < kKeys; i += blockDim.x) {
        running[i] = 0;
        for (int w = 0; w < kW; w++) wcnt[w][i] = 0;
    }
    __syncthreads();
    const int64_t v0 = (int64_t)chunk * kSortChunk;
    for (int r = 0; r < kSortChunk; r += kSortThreads) {
        const int64_t v = v0 + r + tid;
        const bool valid = v < n;
        const int k = valid ? key[v] : kKeys;   // kKeys: no vertex
        const unsigned int mask = __match_any_sync(0xffffffffu, k);
        const int rank_in_warp = __popc(mask & ((1u << lane) - 1u));
        const bool leader = rank_in_warp == 0;
        if (valid && leader) wcnt[warp][k] = __popc(mask);
        __syncthreads();
        if (valid) {
            int before = running[k] + rank_in_warp;
            for (int w = 0; w < warp; w++) before += wcnt[w][k];
            const int32_t dest = Mscan[(int64_t)k * nchunks + chunk] + before;
            perm[dest] = (int32_t)v;
            inv[v] = dest;
        }
        __syncthreads();
        if (valid && leader) {
            atomicAdd(&running[k], __popc(mask));
            wcnt[warp][k] = 0;
        }
        __syncthreads();
    }
}

// Relabelled in-degrees and out-degrees: row i is caller row perm[i].
__global__ void relabel_degrees_kernel(const int32_t *__restrict__ perm, const int32_t *__restrict__ old_off,
                                       const int32_t *__restrict__ old_od, int32_t n, int32_t *__restrict__ new_deg,
                                       int32_t *__restrict__ new_od) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = perm[i];
        new_deg[i] = old_off[v + 1] - old_off[v];
        new_od[i] = old_od[v];
    }
}

// First relabelled row of every in-degree class (in-key ik = 32 - class),
// read from the scanned key counts: bucket (ik, out-key 0) of chunk 0.
// out[ik] = off[starts[ik]] for the 33 in-key classes, out[33] = off[n]
__global__ void class_bounds_kernel(const int32_t *off, const int32_t *starts, int32_t n, int32_t *out) {
    const int ik = threadIdx.x;
    if (ik < kClasses) out[ik] = off[min(max(starts[ik], 0), n)];
    if (ik == kClasses) out[ik] = off[n];
}
__global__ void class_starts_kernel(const int32_t *__restrict__ Mscan, int32_t nchunks, int32_t *__restrict__ starts) {
    const int ik = threadIdx.x;
    if (ik < kClasses) starts[ik] = Mscan[(int64_t)ik * kClasses * nchunks];
}

// ---------------------------------------------------------------- exclusive scan (int32)
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Exclusive scan of one tile per CTA; the tile's total goes to sums[block].
__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(const int32_t *__restrict__ in, int64_t len,
                                                                  int32_t *__restrict__ out, int32_t *__restrict__ sums) {
    __shared__ int32_t warp_tot[kScanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)tid * kScanItems;
    int32_t x[kScanItems];
    int32_t t = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        x[i] = base + i < len ? in[base + i] : 0;
        t += x[i];
    }
    int32_t incl = t;
    for (int m = 1; m < 32; m <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, incl, m);
        if (lane >= m) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    int32_t woff = 0;
    for (int w = 0; w < warp; w++) woff += warp_tot[w];
    int32_t run = woff + incl - t;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        if (base + i < len) out[base + i] = run;
        run += x[i];
    }
    if (tid == kScanThreads - 1) sums[blockIdx.x] = woff + incl;
}
// Exclusive scan of the tile totals, one CTA, in order.
__global__ void scan_sums_kernel(int32_t *sums, int32_t nsums) {
    __shared__ int32_t carry;
    __shared__ int32_t warp_tot[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int32_t b = 0; b < nsums; b += blockDim.x) {
        const int32_t i = b + tid;
        const int32_t x = i < nsums ? sums[i] : 0;
        int32_t incl = x;
        for (int m = 1; m < 32; m <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, incl, m);
            if (lane >= m) incl += y;
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        int32_t woff = 0;
        for (int w = 0; w < warp; w++) woff += warp_tot[w];
        const int32_t c = carry;
        if (i < nsums) sums[i] = c + woff + incl - x;
        __syncthreads();
        if (tid == blockDim.x - 1) carry = c + woff + incl;
        __syncthreads();
    }
}
__global__ void add_tile_offsets_kernel(int32_t *__restrict__ out, int64_t len, const int32_t *__restrict__ sums) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) out[i] += sums[i / kScanTile];
}

int blocks_for(int64_t work, int threads) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t want = (work + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 16));
}


// out[i] = in[0] + .. + in[i-1] for i < len (int32; the caller guarantees the
// total fits); sums: scratch of at least ceil(len / kScanTile) int32.
cudaError_t exclusive_scan(const int32_t *in, int64_t len, int32_t *out, int32_t *sums) {
    if (len <= 0) return cudaSuccess;
    const int64_t tiles = (len + kScanTile - 1) / kScanTile;
    scan_tiles_kernel<<<(unsigned int)tiles, kScanThreads>>>(in, len, out, sums);
    scan_sums_kernel<<<1, 1024>>>(sums, (int32_t)tiles);
    add_tile_offsets_kernel<<<(unsigned int)((len + 255) / 256), 256>>>(out, len, sums);
    return cudaGetLastError();
}

}  // namespace

// Graph creation. The host checks the offsets and out-degrees (O(n) reads of
// the caller's arrays) and builds the tile tables from the relabelled offsets;
// the device validates every source, sorts the vertices into the relabelled
// order (stable counting sort by degree classes), forms the new offsets by a
// scan and writes the remapped rows.
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
    // (split over host threads for large n; the first offending row is reported)
    int64_t deg_sum = 0;
    int32_t n_dangling = 0;
    {
        struct Part { int64_t sum = 0; int32_t dangling = 0, bad_off = INT32_MAX, bad_od = INT32_MAX; };
        const int nthreads = n >= (1 << 20) ? (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency())) : 1;
        std::vector<Part> parts((size_t)nthreads);
        auto scan = [&](int k) {
            const int32_t a = (int32_t)((int64_t)n * k / nthreads), b = (int32_t)((int64_t)n * (k + 1) / nthreads);
            Part &p = parts[(size_t)k];
            for (int32_t v = a; v < b; v++) {
                if (in_offsets[v + 1] < in_offsets[v] && p.bad_off == INT32_MAX) p.bad_off = v;
                if (out_degree[v] < 0 && p.bad_od == INT32_MAX) p.bad_od = v;
                p.sum += out_degree[v];
                p.dangling += out_degree[v] == 0;
            }
        };
        std::vector<std::thread> pool;
        try {
            for (int k = 1; k < nthreads; k++) pool.emplace_back(scan, k);
        } catch (const std::system_error &) {
            for (int k = 1 + (int)pool.size(); k < nthreads; k++) scan(k);
        }
        scan(0);
        for (auto &th : pool) th.join();
        int32_t bad_off = INT32_MAX, bad_od = INT32_MAX;
        for (const Part &p : parts) {
            deg_sum += p.sum;
            n_dangling += p.dangling;
            bad_off = std::min(bad_off, p.bad_off);
            bad_od = std::min(bad_od, p.bad_od);
        }
        if (bad_off != INT32_MAX && bad_off <= bad_od)
            return pr_fail(PR_EINVAL, "in_offsets is not non-decreasing at row " + std::to_string(bad_off));
        if (bad_od != INT32_MAX) return pr_fail(PR_EINVAL, "out_degree[" + std::to_string(bad_od) + "] is negative");
    }
    if (deg_sum != nnz) return pr_fail(PR_EINVAL, "out_degree does not sum to nnz (it must match the edges in in_sources)");
    // ---- caller arrays on the device, sources validated there
    DevTmp d_old_off, d_old_src, d_old_od, d_cnt, d_bad;
    cudaError_t e = cudaSuccess;
    const size_t n_off = (size_t)n + 1 + kPad, n_src = (size_t)nnz + kPad, n_od = (size_t)n + kPad;
    pr_graph *g = new (std::nothrow) pr_graph();
    if (!g) return pr_fail(PR_ENOMEM, "host allocation failed");
    g->magic = kGraphMagic;
    g->n = n;
    g->nnz = nnz;
    g->n_dangling = n_dangling;
    cudaGetDevice(&g->device);
    // the graph's five arrays in one allocation (256-byte aligned sections)
    pr_status s;
    {
        auto sec = [](size_t count) { return (sizeof(int32_t) * count + 255) & ~size_t(255); };
        const size_t o_src = sec(n_off), o_od = o_src + sec(n_src), o_perm = o_od + sec(n_od),
                     o_inv = o_perm + sec((size_t)n), total = o_inv + sec((size_t)n);
        void *vmem = nullptr;
        if ((s = pr_graph_alloc(&vmem, total, &g->d_mem_pooled)) != PR_OK) {
            free_graph(g);
            return s;
        }
        unsigned char *mem = static_cast<unsigned char *>(vmem);
        g->d_mem = mem;
        g->d_off = reinterpret_cast<int32_t *>(mem);
        g->d_src = reinterpret_cast<int32_t *>(mem + o_src);
        g->d_outdeg = reinterpret_cast<int32_t *>(mem + o_od);
        g->d_perm = reinterpret_cast<int32_t *>(mem + o_perm);
        g->d_inv = reinterpret_cast<int32_t *>(mem + o_inv);
    }
    e = d_old_off.alloc(sizeof(int32_t) * ((size_t)n + 1));
    if (e == cudaSuccess) e = d_old_src.alloc(sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1));
    if (e == cudaSuccess) e = d_old_od.alloc(sizeof(int32_t) * (size_t)n);
    if (e == cudaSuccess) e = d_cnt.alloc(sizeof(int32_t) * (size_t)n);
    if (e == cudaSuccess) e = d_bad.alloc(2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpy(d_old_off.p, in_offsets, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nnz > 0) e = cudaMemcpy(d_old_src.p, in_sources, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(d_cnt.p, 0, sizeof(int32_t) * (size_t)n);
    if (e == cudaSuccess) e = cudaMemset(d_bad.p, 0xFF, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpy(d_old_od.p, out_degree, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_graph(g);
        return pr_cuda_fail(e, "graph upload");
    }
    unsigned long long *bad = static_cast<unsigned long long *>(d_bad.p);
    if (nnz > 0)
        count_sources_kernel<<<blocks_for(nnz, 256), 256>>>(static_cast<const int32_t *>(d_old_src.p), nnz, n,
                                                            static_cast<int32_t *>(d_cnt.p), bad);
    check_outdeg_kernel<<<blocks_for(n, 256), 256>>>(static_cast<const int32_t *>(d_cnt.p),
                                                     static_cast<const int32_t *>(d_old_od.p), n, bad + 1);
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
    // ---- relabel on the device: stable counting sort by (in-class desc,
    // out-class desc, caller id); new offsets by a scan of the relabelled degrees
    const int32_t *old_off = static_cast<const int32_t *>(d_old_off.p);
    const int32_t *old_od = static_cast<const int32_t *>(d_old_od.p);
    const int32_t nchunks = (int32_t)(((int64_t)n + kSortChunk - 1) / kSortChunk);
    const int64_t mlen = (int64_t)kKeys * nchunks;
    const int64_t nsums = std::max<int64_t>((mlen + kScanTile - 1) / kScanTile, ((int64_t)n + kScanTile - 1) / kScanTile);
    // class starts, largest in-degrees and new-offset bounds share one block
    // (one read-back)
    DevTmp d_key, d_M, d_Ms, d_sums, d_meta, d_newdeg;
    e = d_key.alloc(sizeof(int32_t) * (size_t)n);
    if (e == cudaSuccess) e = d_M.alloc(sizeof(int32_t) * (size_t)mlen);
    if (e == cudaSuccess) e = d_Ms.alloc(sizeof(int32_t) * (size_t)mlen);
    if (e == cudaSuccess) e = d_sums.alloc(sizeof(int32_t) * (size_t)nsums);
    if (e == cudaSuccess) e = d_meta.alloc(sizeof(int32_t) * (3 * kClasses + 1));
    if (e == cudaSuccess) e = d_newdeg.alloc(sizeof(int32_t) * (size_t)n);
    int32_t *m_starts = static_cast<int32_t *>(d_meta.p), *m_cmax = m_starts + kClasses, *m_bound = m_cmax + kClasses;
    if (e == cudaSuccess) e = cudaMemset(m_cmax, 0, sizeof(int32_t) * kClasses);
    if (e == cudaSuccess) e = cudaMemset(g->d_off, 0, sizeof(int32_t) * n_off);
    if (e == cudaSuccess) e = cudaMemset(g->d_src, 0, sizeof(int32_t) * n_src);
    if (e == cudaSuccess) e = cudaMemset(g->d_outdeg, 0, sizeof(int32_t) * n_od);
    int32_t *key = static_cast<int32_t *>(d_key.p), *M = static_cast<int32_t *>(d_M.p), *Ms = static_cast<int32_t *>(d_Ms.p);
    int32_t *sums = static_cast<int32_t *>(d_sums.p), *cmax = m_cmax;
    if (e == cudaSuccess) {
        class_keys_kernel<<<blocks_for(n, 256), 256>>>(old_off, old_od, n, key, cmax);
        chunk_hist_kernel<<<nchunks, kSortThreads>>>(key, n, nchunks, M);
        e = exclusive_scan(M, mlen, Ms, sums);
    }
    if (e == cudaSuccess) {
        chunk_scatter_kernel<<<nchunks, kSortThreads>>>(key, n, nchunks, Ms, g->d_perm, g->d_inv);
        relabel_degrees_kernel<<<blocks_for(n, 256), 256>>>(g->d_perm, old_off, old_od, n,
                                                           static_cast<int32_t *>(d_newdeg.p), g->d_outdeg);
        e = exclusive_scan(static_cast<const int32_t *>(d_newdeg.p), n, g->d_off, sums);
    }
    if (e == cudaSuccess) {
        const int32_t total = (int32_t)nnz;
        class_starts_kernel<<<1, 64>>>(Ms, nchunks, m_starts);
        e = cudaMemcpy(g->d_off + n, &total, sizeof(int32_t), cudaMemcpyHostToDevice);
    }
    // the new offsets at the class starts (and at n), for the signature
    int32_t h_meta[3 * kClasses + 1];
    const int32_t *h_starts = h_meta, *h_cmax = h_meta + kClasses, *h_bound = h_meta + 2 * kClasses;
    if (e == cudaSuccess) {
        class_bounds_kernel<<<1, 64>>>(g->d_off, m_starts, n, m_bound);
        e = cudaMemcpy(h_meta, d_meta.p, sizeof(h_meta), cudaMemcpyDeviceToHost);
    }
    if (e == cudaSuccess && nnz > 0) {
        // rows in the new order: 1024+ in-edges (classes 11 and up), then
        // 32..1023 (classes 6..10), then the rest
        const int32_t i_hub = h_starts[32 - 10], i_short = h_starts[32 - 5];
        if (i_hub > 0)
            remap_hub_rows_kernel<<<std::min<int32_t>(i_hub, 65535), 256>>>(
                old_off, static_cast<const int32_t *>(d_old_src.p), g->d_off, g->d_perm, g->d_inv, i_hub, g->d_src);
        if (i_short > i_hub)
            remap_rows_kernel<<<blocks_for((int64_t)(i_short - i_hub) * 32, 256), 256>>>(
                old_off, static_cast<const int32_t *>(d_old_src.p), g->d_off, g->d_perm, g->d_inv, i_hub, i_short,
                g->d_src);
        if (i_short < n)
            remap_short_rows_kernel<<<blocks_for((int64_t)(n - i_short), 256), 256>>>(
                old_off, static_cast<const int32_t *>(d_old_src.p), g->d_off, g->d_perm, g->d_inv, i_short, n, g->d_src);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_graph(g);
        return pr_cuda_fail(e, "graph relabel");
    }
    // in-degree classes in relabelled order: in-key ik = 32 - class, ascending
    for (int ik = 0; ik < kClasses; ik++) {
        const int32_t begin = h_starts[ik], end = ik + 1 < kClasses ? h_starts[ik + 1] : n;
        if (end > begin) g->classes.push_back(ClassRange{begin, end, h_cmax[32 - ik]});
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
        for (int ik = 0; ik < kClasses; ik++) {
            const int32_t begin = h_starts[ik], end = ik + 1 < kClasses ? h_starts[ik + 1] : n;
            if (end <= begin) continue;
            mix((uint64_t)begin);
            mix((uint64_t)end);
            mix((uint64_t)h_cmax[32 - ik]);
            mix((uint64_t)(h_bound[ik + 1] - h_bound[ik]));
        }
        g->signature = h;
    }
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
