// pr_solve.cu — the solve driver: lays out jobs, runs the device loop.
//
// A request is a list of columns (iterate sequences) with their stopping taps,
// and its jobs: columns of one graph, at most 32, whose rank matrices are
// N x W vertex-major (W = columns padded to a power of two), so that one read
// of a row's in-edge indices serves W gathers (the planner in pr_plan.cu
// chooses the jobs). One pass per iteration: a gather kernel and an update
// kernel, or one fused kernel for small requests. The passes run inside a CUDA
// graph whose while-node repeats the pass until the device reports that every
// column has stopped and every answer has been copied out; or, for fused
// passes whose grid fits on the device, inside one cooperative launch in which
// each job's CTAs loop until the job is done (persistent passes); or one
// launch at a time from the host.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <atomic>
#include <mutex>

#include "pr_kernels.cuh"

size_t gather_smem_bytes(int prec, int W);   // below, beside pr_tile_smem_bytes

namespace {

// Per-device memory pools: one for the solve workspaces (stream-ordered
// allocations that return to the pool when a call ends) and one for the
// arrays of live graphs (returned when the graph is destroyed), so that
// repeated calls and graphs reuse memory instead of paying cudaMalloc/cudaFree,
// which synchronise and map or unmap pages (host-device copies issued right
// after an unmapping were measured at 15-30 GB/s against 210 GB/s). Up to
// kPoolKeepBytes per pool stay reserved between uses; the rest goes back to
// the device at the next synchronisation.
constexpr unsigned long long kPoolKeepBytes = 16ull << 30;

std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools, g_graph_pools;

// The device's pool if one has been created (no creation).
cudaMemPool_t existing_pool(int dev, bool graphs = false) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto &pools = graphs ? g_graph_pools : g_pools;
    auto it = pools.find(dev);
    return it == pools.end() ? nullptr : it->second;
}

cudaMemPool_t workspace_pool(int dev, bool graphs = false) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto &pools = graphs ? g_graph_pools : g_pools;
    auto it = pools.find(dev);
    if (it != pools.end()) return it->second;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    unsigned long long keep = kPoolKeepBytes;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = pool;
    return pool;
}

struct Arena {
    PoolBuf buf;
    char *base = nullptr;
    size_t size = 0;
    size_t reserve(size_t bytes) {   // returns offset
        size_t off = (size + 255) & ~size_t(255);
        size = off + bytes;
        return off;
    }
    pr_status alloc(cudaStream_t st) {
        if (size == 0) size = 256;
        pr_status s = buf.alloc(size, st);
        base = static_cast<char *>(buf.p);
        return s;
    }
    template <typename T> T *at(size_t off) { return reinterpret_cast<T *>(base + off); }
};

}  // namespace

pr_status PoolBuf::alloc(size_t bytes, cudaStream_t st) {
    release();
    if (bytes == 0) bytes = 256;
    stream = st;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool = workspace_pool(dev);
    cudaError_t e = cudaErrorMemoryAllocation;
    if (pool) {
        e = cudaMallocFromPoolAsync(&p, bytes, pool, st);
        pooled = e == cudaSuccess;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        e = cudaMalloc(&p, bytes);
    }
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        return pr_fail(e == cudaErrorMemoryAllocation ? PR_ENOMEM : PR_ECUDA,
                       "device workspace of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
    }
    return PR_OK;
}

extern "C" pr_status pr_workspace_info(int64_t *reserved_bytes, int64_t *used_bytes, int64_t *used_high_bytes) {
    pr_clear_error();
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    unsigned long long res = 0, used = 0, high = 0;   // the attributes are 64-bit counts
    if (cudaMemPool_t pool = existing_pool(dev)) {
        PR_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &res));
        PR_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
        PR_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &high));
    }
    if (reserved_bytes) *reserved_bytes = (int64_t)res;
    if (used_bytes) *used_bytes = (int64_t)used;
    if (used_high_bytes) *used_high_bytes = (int64_t)high;
    return PR_OK;
}

extern "C" pr_status pr_workspace_release(void) {
    pr_clear_error();
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    for (bool graphs : {false, true})
        if (cudaMemPool_t pool = existing_pool(dev, graphs)) {
            PR_CUDA(cudaDeviceSynchronize());   // frees issued on any stream have completed
            PR_CUDA(cudaMemPoolTrimTo(pool, 0));
        }
    return PR_OK;
}

// Graph arrays: from the device's graph pool on the legacy default stream
// (graph creation works there), else cudaMalloc; *pooled says which.
pr_status pr_graph_alloc(void **p, size_t bytes, bool *pooled) {
    *p = nullptr;
    *pooled = false;
    if (bytes == 0) bytes = 256;
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    cudaError_t e = cudaErrorMemoryAllocation;
    if (cudaMemPool_t pool = workspace_pool(dev, true)) {
        e = cudaMallocFromPoolAsync(p, bytes, pool, 0);
        *pooled = e == cudaSuccess;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        e = cudaMalloc(p, bytes);
    }
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return pr_fail(e == cudaErrorMemoryAllocation ? PR_ENOMEM : PR_ECUDA,
                       "graph arrays of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
    }
    return PR_OK;
}

// Frees what pr_graph_alloc gave after all device work that may still read it
// (any stream) has finished, as cudaFree would.
void pr_graph_free(void *p, bool pooled) {
    if (!p) return;
    cudaDeviceSynchronize();
    if (pooled) cudaFreeAsync(p, 0);
    else cudaFree(p);
}

void PoolBuf::release() {
    if (!p) return;
    if (pooled) cudaFreeAsync(p, stream);
    else cudaFree(p);
    p = nullptr;
    pooled = false;
}

namespace {

template <typename V>
void *iter_ptr(int W) {
    switch (W) {
        case 1: return (void *)pr_iter_kernel<V, 1>;
        case 2: return (void *)pr_iter_kernel<V, 2>;
        case 4: return (void *)pr_iter_kernel<V, 4>;
        case 8: return (void *)pr_iter_kernel<V, 8>;
        case 16: return (void *)pr_iter_kernel<V, 16>;
        default: return (void *)pr_iter_kernel<V, 32>;
    }
}
// Persistent passes: the fused pass repeated in one cooperative launch.
template <typename V>
void *persist_ptr(int W) {
    switch (W) {
        case 1: return (void *)pr_iter_kernel<V, 1, kModePersist>;
        case 2: return (void *)pr_iter_kernel<V, 2, kModePersist>;
        case 4: return (void *)pr_iter_kernel<V, 4, kModePersist>;
        case 8: return (void *)pr_iter_kernel<V, 8, kModePersist>;
        case 16: return (void *)pr_iter_kernel<V, 16, kModePersist>;
        default: return (void *)pr_iter_kernel<V, 32, kModePersist>;
    }
}
void *persist_kernel_for(int prec, int W) {
    switch (prec) {
        case PR_PREC_FP64: return persist_ptr<double>(W);
        case PR_PREC_FP32: return persist_ptr<float>(W);
        default: return persist_ptr<df64>(W);
    }
}
// Split passes: the gather-only and update kernels.
template <typename V>
void *gather_ptr(int W) {
    switch (W) {
        case 1: return (void *)pr_iter_kernel<V, 1, kModeGather>;
        case 2: return (void *)pr_iter_kernel<V, 2, kModeGather>;
        case 4: return (void *)pr_iter_kernel<V, 4, kModeGather>;
        case 8: return (void *)pr_iter_kernel<V, 8, kModeGather>;
        case 16: return (void *)pr_iter_kernel<V, 16, kModeGather>;
        default: return (void *)pr_iter_kernel<V, 32, kModeGather>;
    }
}
template <typename V>
void *update_ptr(int W) {
    switch (W) {
        case 1: return (void *)pr_update_kernel<V, 1>;
        case 2: return (void *)pr_update_kernel<V, 2>;
        case 4: return (void *)pr_update_kernel<V, 4>;
        case 8: return (void *)pr_update_kernel<V, 8>;
        case 16: return (void *)pr_update_kernel<V, 16>;
        default: return (void *)pr_update_kernel<V, 32>;
    }
}
// Split passes of one, two or four columns gather with the hub kernel (a
// vertex's values fill at most one 32-byte sector in every value type, so both
// phases of mixed precision use it alike); wider jobs with the multi-column
// gather kernel.
bool hub_gather(int W) { return kHubGather && hub_width_ok(W, 8); }
template <typename V>
void *hub_ptr(int W) {
    switch (W) {
        case 1: return (void *)pr_gather_hub1_kernel<V>;
        case 2: return (void *)pr_gather_hub_kernel<V, 2>;
        default: return (void *)pr_gather_hub_kernel<V, 4>;
    }
}
void *hub_gather_kernel_for(int prec, int W) {
    switch (prec) {
        case PR_PREC_FP64: return hub_ptr<double>(W);
        case PR_PREC_FP32: return hub_ptr<float>(W);
        default: return hub_ptr<df64>(W);
    }
}
int gather_block(int W) { return hub_gather(W) ? kHubBlock : kBlock; }
void *gather_kernel_for(int prec, int W) {
    if (hub_gather(W)) return hub_gather_kernel_for(prec, W);
    switch (prec) {
        case PR_PREC_FP64: return gather_ptr<double>(W);
        case PR_PREC_FP32: return gather_ptr<float>(W);
        default: return gather_ptr<df64>(W);
    }
}
// One column: the bulk-copy form of the update kernel (kUpdateBulk), with
// kUpdStages tiles of dynamic shared memory.
bool update_bulk(int W) { return kUpdateBulk && W == 1; }
size_t update_smem_bytes(int prec, int W) {
    if (!update_bulk(W)) return 0;
    return (size_t)kUpdStages * upd_stage_bytes(prec == PR_PREC_FP32 ? 4 : 8);
}
void *update_kernel_for(int prec, int W) {
    if (update_bulk(W)) {
        switch (prec) {
            case PR_PREC_FP64: return (void *)pr_update_bulk_kernel<double>;
            case PR_PREC_FP32: return (void *)pr_update_bulk_kernel<float>;
            default: return (void *)pr_update_bulk_kernel<df64>;
        }
    }
    switch (prec) {
        case PR_PREC_FP64: return update_ptr<double>(W);
        case PR_PREC_FP32: return update_ptr<float>(W);
        default: return update_ptr<df64>(W);
    }
}
int resident_ctas(void *k, size_t smem, int block = kBlock) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, block, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return std::max(occ, 1);
}

// Shared-memory carveout of an iteration kernel k launched with smem bytes of
// dynamic shared memory (see kSmemCarveout); `minimal` selects the smallest
// carveout that keeps the kernel's residency, else the driver chooses. The
// one-column gather kernel's random gathers are served from L1, whose capacity
// is what the carveout leaves: measured on GB300 (df64), 245 -> 237 us per
// launch at scale 22, 981 -> 949 us at scale 24, 361 -> 339 us on the 8M-vertex
// configuration-model graph (FP32: 6-8 % faster). The fused and multi-column
// kernels keep the driver's choice (no gain measured; W = 4 df64 lost 15 %).
pr_status set_carveout(void *k, size_t smem, bool minimal, int block = kBlock) {
    if (kSmemCarveout == -2) return PR_OK;
    if (kSmemCarveout >= 0) {
        PR_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, kSmemCarveout));
        return PR_OK;
    }
    if (!minimal) return PR_OK;
    cudaFuncAttributes fa;
    PR_CUDA(cudaFuncGetAttributes(&fa, k));
    int dev = 0, per_sm = 0, reserved = 0, occ = 0;
    PR_CUDA(cudaGetDevice(&dev));
    PR_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    PR_CUDA(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
    PR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, block, smem));   // largest carveout
    if (occ < 1 || per_sm <= 0) return PR_OK;
    const double need = (double)occ * ((double)fa.sharedSizeBytes + (double)smem + (double)reserved);
    for (int pct = std::max(1, (int)std::ceil(100.0 * need / per_sm)); pct <= 100; pct++) {
        PR_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
        int got = 0;
        PR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&got, k, block, smem));
        if (got >= occ) return PR_OK;
    }
    PR_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, -1));
    return PR_OK;
}

// Kernel attributes (dynamic shared memory, carveout) are set per device
// context, so the setup and the residencies it measures are kept per device
// ordinal, precision and width. A cudaDeviceReset discards the attributes but
// not this record: the library does not survive a reset of a device it used.
struct SetupKey {
    int dev, prec, wi;
    bool operator<(const SetupKey &o) const {
        return dev != o.dev ? dev < o.dev : (prec != o.prec ? prec < o.prec : wi < o.wi);
    }
};

// Split passes: opt the gather kernel into its dynamic shared memory (once per
// device, precision and width) and report both kernels' residency.
pr_status setup_split(int prec, int W, int *occ_gather, int *occ_update) {
    static std::mutex mu;
    static std::map<SetupKey, std::pair<int, int>> done;   // residencies (gather, update), queried once
    void *kg = gather_kernel_for(prec, W);
    const size_t smem = gather_smem_bytes(prec, W);
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    const SetupKey key{dev, prec & 3, w_index(W)};
    std::lock_guard<std::mutex> lk(mu);
    auto it = done.find(key);
    if (it == done.end()) {
        PR_CUDA(cudaFuncSetAttribute(kg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        pr_status s = set_carveout(kg, smem, W == 1 || hub_gather(W), gather_block(W));
        if (s != PR_OK) return s;
        void *ku = update_kernel_for(prec, W);
        const size_t usmem = update_smem_bytes(prec, W);
        if (usmem > 0) PR_CUDA(cudaFuncSetAttribute(ku, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)usmem));
        const std::pair<int, int> occ{resident_ctas(kg, smem, gather_block(W)), resident_ctas(ku, usmem)};
        it = done.emplace(key, occ).first;
    }
    *occ_gather = it->second.first;
    *occ_update = it->second.second;
    return PR_OK;
}

template <typename V>
void *init_ptr(int W) {
    switch (W) {
        case 1: return (void *)pr_init_kernel<V, 1>;
        case 2: return (void *)pr_init_kernel<V, 2>;
        case 4: return (void *)pr_init_kernel<V, 4>;
        case 8: return (void *)pr_init_kernel<V, 8>;
        case 16: return (void *)pr_init_kernel<V, 16>;
        default: return (void *)pr_init_kernel<V, 32>;
    }
}
void store_value(double *dst, int prec, double x) {
    dst[0] = 0.0;
    dst[1] = 0.0;
    if (prec == PR_PREC_FP64) {
        std::memcpy(dst, &x, 8);
    } else if (prec == PR_PREC_FP32) {
        float f = (float)x;
        std::memcpy(dst, &f, 4);
    } else {
        df64 d = df_from_double(x);
        std::memcpy(dst, &d, 8);
    }
}

int pow2_at_least(int k) {
    int w = 1;
    while (w < k) w <<= 1;
    return w;
}

struct HostJob {
    const pr_graph *g = nullptr;
    std::vector<int> cols;           // request column indices
    const TileTable *tt = nullptr;
    int cta_count = 0;
    int gcta_count = 0;              // split passes: CTAs of the gather kernel
    size_t off_r[2] = {0, 0}, off_c[2] = {0, 0}, off_cp = 0, off_part = 0, off_hist = 0, off_rowsum = 0;
    int ntaps = 0;
    int hist_total = 0;
};

using LoopStats = SolveStats;

std::mutex g_stats_mu;
SolveStats g_last_stats;

}  // namespace

// CTAs worth giving a job of ntiles warp tiles: at least kMinTilesPerWarp
// tiles per warp, so that small graphs do not spread over idle CTAs whose
// partials the job's finalizer must then reduce.
int tile_ctas(int32_t ntiles) {
    const int64_t per_cta = kMinTilesPerWarp > 0 ? (int64_t)kWarps * kMinTilesPerWarp : 1;
    return (int)std::max<int64_t>(1, ((int64_t)std::max(ntiles, 1) + per_cta - 1) / per_cta);
}

void *pr_iter_kernel_for(int prec, int W) {
    switch (prec) {
        case PR_PREC_FP64: return iter_ptr<double>(W);
        case PR_PREC_FP32: return iter_ptr<float>(W);
        default: return iter_ptr<df64>(W);
    }
}
void *pr_init_kernel_for(int prec, int W) {
    switch (prec) {
        case PR_PREC_FP64: return init_ptr<double>(W);
        case PR_PREC_FP32: return init_ptr<float>(W);
        default: return init_ptr<df64>(W);
    }
}
// Dynamic shared memory of the iteration kernel: none for one column (static
// buffers only); for several columns, the per-warp tile buffers (vec_warp_bytes).
size_t pr_tile_smem_bytes(int prec, int W) {
    const int vbytes = prec == PR_PREC_FP32 ? 4 : 8;
    if (W == 1) return 0;
    return (size_t)kWarps * vec_warp_bytes(vbytes, W, false);
}
// The gather-only kernel's: no previous ranks or out-degrees staged; the hub
// gather kernel's: every warp's staged vectors, then the hub table (at most
// hub_bytes(W) of vectors).
size_t gather_smem_bytes(int prec, int W) {
    const int vbytes = prec == PR_PREC_FP32 ? 4 : 8;
    if (hub_gather(W)) return (size_t)kHubWarps * hub_tile_edges(W) * W * vbytes + (size_t)hub_bytes(W);
    if (W == 1) return 0;
    return (size_t)kWarps * vec_warp_bytes(vbytes, W, true);
}

// Opt the iteration kernel into its dynamic shared memory (once per device,
// precision and width) and report its resident CTAs per SM.
pr_status pr_kernel_setup(int prec, int W, int *blocks_per_sm) {
    static std::mutex mu;
    static std::map<SetupKey, int> done;   // residency, queried once
    void *k = pr_iter_kernel_for(prec, W);
    const size_t smem = pr_tile_smem_bytes(prec, W);
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    const SetupKey key{dev, prec & 3, w_index(W)};
    std::lock_guard<std::mutex> lk(mu);
    auto it = done.find(key);
    if (it == done.end()) {
        PR_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        pr_status s = set_carveout(k, smem, false);
        if (s != PR_OK) return s;
        int occ = 0;
        PR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kBlock, smem));
        it = done.emplace(key, std::max(occ, 1)).first;
    }
    *blocks_per_sm = it->second;
    return PR_OK;
}

namespace {
// Persistent passes: opt the persistent kernel into the fused kernel's dynamic
// shared memory (once per device, precision and width) and report how many of
// its CTAs are resident per SM; 0 where the device has no cooperative launch
// (a cooperative grid must be resident as a whole).
pr_status persist_setup(int prec, int W, int *blocks_per_sm) {
    static std::mutex mu;
    static std::map<SetupKey, int> done;
    void *k = persist_kernel_for(prec, W);
    const size_t smem = pr_tile_smem_bytes(prec, W);
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    const SetupKey key{dev, prec & 3, w_index(W)};
    std::lock_guard<std::mutex> lk(mu);
    auto it = done.find(key);
    if (it == done.end()) {
        int coop = 0, occ = 0;
        PR_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        if (coop) {
            PR_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            PR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kBlock, smem));
        }
        it = done.emplace(key, std::max(occ, 0)).first;
    }
    *blocks_per_sm = it->second;
    return PR_OK;
}
}  // namespace

void pr_record_last_stats(const SolveStats &st) {
    std::lock_guard<std::mutex> lk(g_stats_mu);
    g_last_stats = st;
}

extern "C" pr_status pr_kernel_occupancy(int32_t precision, int32_t width, int32_t *ctas_per_sm) {
    pr_clear_error();
    if (precision < PR_PREC_DF64 || precision > PR_PREC_FP32 || precision == PR_PREC_MIXED)
        return pr_fail(PR_EINVAL, "precision must be PR_PREC_DF64, PR_PREC_FP64 or PR_PREC_FP32");
    if (w_index(width) < 0) return pr_fail(PR_EINVAL, "width must be 1, 2, 4, 8, 16 or 32");
    int occ = 0;
    pr_status s = pr_kernel_setup(precision, width, &occ);
    if (s != PR_OK) return s;
    if (kSplitPasses) {
        int ou = 1;
        if ((s = setup_split(precision, width, &occ, &ou)) != PR_OK) return s;
    }
    if (ctas_per_sm) *ctas_per_sm = occ;
    return PR_OK;
}

extern "C" pr_status pr_last_solve_kernel_ms(double *gather_ms, double *update_ms) {
    std::lock_guard<std::mutex> lk(g_stats_mu);
    if (gather_ms) *gather_ms = g_last_stats.gather_ms;
    if (update_ms) *update_ms = g_last_stats.update_ms;
    return PR_OK;
}

extern "C" pr_status pr_last_solve_columns(int32_t *columns, int32_t *mixed_columns, int32_t *learned_columns) {
    std::lock_guard<std::mutex> lk(g_stats_mu);
    if (columns) *columns = g_last_stats.columns;
    if (mixed_columns) *mixed_columns = g_last_stats.mixed_columns;
    if (learned_columns) *learned_columns = g_last_stats.learned_columns;
    return PR_OK;
}

namespace {
std::atomic<int> g_hold_decisions{0};
}
bool pr_hold_decisions() { return g_hold_decisions.load() != 0; }

extern "C" pr_status pr_test_hold_decisions(int32_t on) {
    g_hold_decisions.store(on ? 1 : 0);
    return PR_OK;
}

extern "C" pr_status pr_last_solve_loops(int32_t *graph_phases, int32_t *host_phases, int32_t *persistent_phases) {
    std::lock_guard<std::mutex> lk(g_stats_mu);
    if (graph_phases) *graph_phases = g_last_stats.loop_phases[PR_LOOP_GRAPH];
    if (host_phases) *host_phases = g_last_stats.loop_phases[PR_LOOP_HOST];
    if (persistent_phases) *persistent_phases = g_last_stats.loop_phases[PR_LOOP_PERSISTENT];
    return PR_OK;
}

extern "C" pr_status pr_last_solve_stats(int32_t *launches, int32_t *passes, double *kernel_ms, double *total_ms) {
    std::lock_guard<std::mutex> lk(g_stats_mu);
    if (launches) *launches = g_last_stats.launches;
    if (passes) *passes = g_last_stats.passes;
    if (kernel_ms) *kernel_ms = g_last_stats.kernel_ms;
    if (total_ms) *total_ms = g_last_stats.total_ms;
    return PR_OK;
}

namespace {

// One phase of a solve in one value type: init pass + loop of iteration passes.
pr_status run_phase(int prec, int W, bool split, std::vector<HostJob> &jobs, Arena &ar, size_t off_jobs,
                    size_t off_glob, size_t off_ctajob, int total_ctas, size_t off_gctajob, int total_gctas,
                    int pass_cap, int loop, int wait_us, cudaStream_t st, LoopStats &stats) {
    // split passes: the pass is the gather kernel then the update kernel
    void *kiter = split ? update_kernel_for(prec, W) : pr_iter_kernel_for(prec, W);
    void *kgather = split ? gather_kernel_for(prec, W) : nullptr;
    void *kinit = pr_init_kernel_for(prec, W);
    const size_t smem = pr_tile_smem_bytes(prec, W);
    int occ = 0;
    pr_status s0 = pr_kernel_setup(prec, W, &occ);
    if (s0 != PR_OK) return s0;
    JobDev *d_jobs = ar.at<JobDev>(off_jobs);
    GlobalDev *d_glob = ar.at<GlobalDev>(off_glob);
    const int32_t *d_ctajob = ar.at<int32_t>(off_ctajob);
    const int32_t *d_gctajob = split ? ar.at<int32_t>(off_gctajob) : nullptr;
    GlobalDev hg;
    std::memset(&hg, 0, sizeof(hg));
    hg.njobs = (int32_t)jobs.size();
    hg.pass_cap = pass_cap;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    PR_CUDA(cudaEventCreate(&ev0));
    PR_CUDA(cudaEventCreate(&ev1));
    struct EvGuard { cudaEvent_t a, b; ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); } } evg{ev0, ev1};
    void *args[] = {(void *)&d_jobs, (void *)&d_glob, (void *)&d_ctajob};
    void *gargs[] = {(void *)&d_jobs, (void *)&d_glob, (void *)&d_gctajob};
    dim3 grid(total_ctas), ggrid(split ? total_gctas : 1), block(kBlock), gblock(gather_block(W));
    const size_t iter_smem = split ? update_smem_bytes(prec, W) : smem, gather_smem = split ? gather_smem_bytes(prec, W) : 0;
    PR_CUDA(cudaEventRecord(ev0, st));
    if (loop >= PR_LOOP_GRAPH && loop <= PR_LOOP_PERSISTENT) stats.loop_phases[loop]++;
    if (loop == PR_LOOP_PERSISTENT) {
        // the init pass, then every iteration pass in one cooperative launch
        // (the caller checked that the grid is resident as a whole)
        hg.cond = 0;
        hg.wait_us = (uint32_t)wait_us;
        hg.hold = pr_hold_decisions() ? 1 : 0;
        PR_CUDA(cudaMemcpyAsync(d_glob, &hg, sizeof(hg), cudaMemcpyHostToDevice, st));
        PR_CUDA(cudaLaunchKernel(kinit, grid, block, args, 0, st));
        PR_CUDA(cudaLaunchCooperativeKernel(persist_kernel_for(prec, W), grid, block, args, iter_smem, st));
        PR_CUDA(cudaEventRecord(ev1, st));
        stats.launches += 2;
        GlobalDev back;
        std::memset(&back, 0, sizeof(back));
        PR_CUDA(cudaMemcpyAsync(&back, d_glob, sizeof(back), cudaMemcpyDeviceToHost, st));
        PR_CUDA(cudaStreamSynchronize(st));
        stats.passes += back.pass;
        if (back.error == kErrWait) return pr_fail(PR_ETIMEOUT, "a persistent pass waited too long for its job's CTAs");
        if (back.error) return pr_fail(PR_ETIMEOUT, "device loop did not finish within its pass cap");
    } else if (loop == PR_LOOP_HOST) {
        hg.cond = 0;
        PR_CUDA(cudaMemcpyAsync(d_glob, &hg, sizeof(hg), cudaMemcpyHostToDevice, st));
        PR_CUDA(cudaLaunchKernel(kinit, grid, block, args, 0, st));
        stats.launches++;
        cudaEvent_t k0 = nullptr, km = nullptr, k1 = nullptr;
        PR_CUDA(cudaEventCreate(&k0));
        PR_CUDA(cudaEventCreate(&km));
        PR_CUDA(cudaEventCreate(&k1));
        struct KGuard {
            cudaEvent_t a, b, c;
            ~KGuard() { cudaEventDestroy(a); cudaEventDestroy(b); cudaEventDestroy(c); }
        } kg{k0, km, k1};
        GlobalDev back;
        std::memset(&back, 0, sizeof(back));
        for (int p = 0; p < pass_cap + 1; p++) {
            PR_CUDA(cudaEventRecord(k0, st));
            if (split) {
                PR_CUDA(cudaLaunchKernel(kgather, ggrid, gblock, gargs, gather_smem, st));
                PR_CUDA(cudaEventRecord(km, st));
                stats.launches++;
            }
            PR_CUDA(cudaLaunchKernel(kiter, grid, block, args, iter_smem, st));
            PR_CUDA(cudaEventRecord(k1, st));
            stats.launches++;
            PR_CUDA(cudaMemcpyAsync(&back, d_glob, sizeof(back), cudaMemcpyDeviceToHost, st));
            PR_CUDA(cudaStreamSynchronize(st));
            float ms = 0.f;
            PR_CUDA(cudaEventElapsedTime(&ms, k0, k1));
            stats.kernel_ms += ms;
            if (split) {
                float mg = 0.f;
                PR_CUDA(cudaEventElapsedTime(&mg, k0, km));
                stats.gather_ms += mg;
                stats.update_ms += ms - mg;
            }
            if (!back.alive || back.error) break;
        }
        PR_CUDA(cudaEventRecord(ev1, st));
        stats.passes += back.pass;
        if (back.error) return pr_fail(PR_ETIMEOUT, "device loop did not finish within its pass cap");
    } else {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        PR_CUDA(cudaGraphCreate(&graph, 0));
        struct GGuard {
            cudaGraph_t *g; cudaGraphExec_t *x;
            ~GGuard() { if (*x) cudaGraphExecDestroy(*x); if (*g) cudaGraphDestroy(*g); }
        } gg{&graph, &exec};
        cudaGraphConditionalHandle h;
        PR_CUDA(cudaGraphConditionalHandleCreate(&h, graph, 1u, cudaGraphCondAssignDefault));
        hg.cond = (unsigned long long)h;
        PR_CUDA(cudaMemcpyAsync(d_glob, &hg, sizeof(hg), cudaMemcpyHostToDevice, st));
        cudaKernelNodeParams kp{};
        kp.func = kinit;
        kp.gridDim = grid;
        kp.blockDim = block;
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        cudaGraphNode_t n_init, n_cond, n_body;
        PR_CUDA(cudaGraphAddKernelNode(&n_init, graph, nullptr, 0, &kp));
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        PR_CUDA(cudaGraphAddNode(&n_cond, graph, &n_init, nullptr, 1, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaGraphNode_t n_gather = nullptr;
        if (split) {
            cudaKernelNodeParams gp = kp;
            gp.func = kgather;
            gp.gridDim = ggrid;
            gp.blockDim = gblock;
            gp.sharedMemBytes = (unsigned int)gather_smem;
            gp.kernelParams = gargs;
            PR_CUDA(cudaGraphAddKernelNode(&n_gather, body, nullptr, 0, &gp));
        }
        kp.func = kiter;
        kp.sharedMemBytes = (unsigned int)iter_smem;
        PR_CUDA(cudaGraphAddKernelNode(&n_body, body, split ? &n_gather : nullptr, split ? 1 : 0, &kp));
        PR_CUDA(cudaGraphInstantiate(&exec, graph, 0));
        PR_CUDA(cudaGraphLaunch(exec, st));
        PR_CUDA(cudaEventRecord(ev1, st));
        GlobalDev back;
        std::memset(&back, 0, sizeof(back));
        PR_CUDA(cudaMemcpyAsync(&back, d_glob, sizeof(back), cudaMemcpyDeviceToHost, st));
        PR_CUDA(cudaStreamSynchronize(st));
        stats.launches += 1 + (split ? 2 : 1) * (int)back.body_count;
        stats.passes += back.pass;
        if (back.error) return pr_fail(PR_ETIMEOUT, "device loop did not finish within its pass cap");
    }
    // ev1 was recorded right after the loop's last launch (the read-back
    // synchronisation above has already waited for it)
    PR_CUDA(cudaEventSynchronize(ev1));
    float ms = 0.f;
    PR_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
    stats.total_ms += ms;
    return PR_OK;
}

}  // namespace

namespace {

// One device-to-device copy of a stopping rule's answer that aliases another
// rule's (both fired on the same iterate).
struct CopyItem {
    double *dst;
    const double *src;
    int64_t n;
};
// All alias copies of a solve in one launch: blockIdx.y picks the copy,
// blockIdx.x strides over its elements.
__global__ void alias_copy_kernel(const CopyItem *__restrict__ items) {
    const CopyItem it = items[blockIdx.y];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < it.n; i += (int64_t)gridDim.x * blockDim.x)
        it.dst[i] = it.src[i];
}

}  // namespace

pr_status pr_run_solve(SolveRequest &req, std::vector<std::vector<Tap>> &tap_out) {
    LoopStats stats;
    const int ncols = (int)req.cols.size();
    if (ncols == 0) return PR_OK;
    cudaStream_t st = req.stream;
    const bool mixed = req.precision == PR_PREC_MIXED;
    const int prec1 = mixed ? PR_PREC_FP32 : req.precision;
    // ---- group columns into jobs (same graph, <= 32 columns)
    std::vector<HostJob> jobs;
    if (!req.jobs.empty()) {
        for (const auto &jc : req.jobs) {
            if (jc.empty() || jc.size() > 32) return pr_fail(PR_EINVAL, "internal: job of bad size");
            HostJob j;
            j.g = req.cols[jc[0]].g;
            for (int c : jc)
                if (c < 0 || c >= ncols || req.cols[c].g != j.g) return pr_fail(PR_EINVAL, "internal: bad job column");
            j.cols = jc;
            jobs.push_back(j);
        }
    } else {
        std::map<const pr_graph *, std::vector<int>> by_graph;
        std::vector<const pr_graph *> order;
        for (int c = 0; c < ncols; c++) {
            if (!by_graph.count(req.cols[c].g)) order.push_back(req.cols[c].g);
            by_graph[req.cols[c].g].push_back(c);
        }
        for (const pr_graph *g : order) {
            const auto &v = by_graph[g];
            for (size_t i = 0; i < v.size(); i += 32) {
                HostJob j;
                j.g = g;
                j.cols.assign(v.begin() + i, v.begin() + std::min(v.size(), i + 32));
                jobs.push_back(j);
            }
        }
    }
    int W = 1;
    for (auto &j : jobs) W = std::max(W, pow2_at_least((int)j.cols.size()));
    // ---- tile tables and CTA split
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    int sms = 0;
    PR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int occ = 1;
    pr_status s = pr_kernel_setup(prec1, W, &occ);
    if (s != PR_OK) return s;
    if (mixed) {
        int occ2 = 1;
        if ((s = pr_kernel_setup(PR_PREC_DF64, W, &occ2)) != PR_OK) return s;
        occ = std::min(occ, occ2);
    }
    // split passes or one fused kernel per pass (PR_KERNELS_AUTO: split from
    // kSplitMinWork in-edge columns on)
    double edge_cols = 0.0;
    for (auto &j : jobs) edge_cols += (double)j.g->nnz * W;
    const bool split = req.kernels == PR_KERNELS_SPLIT ||
                       (req.kernels == PR_KERNELS_AUTO && kSplitPasses && edge_cols >= kSplitMinWork);
    int occ_gather = 1;
    if (split) {
        // split passes: the update kernel's grid carries the pass bookkeeping,
        // the gather kernel gets its own (more resident CTAs)
        if ((s = setup_split(prec1, W, &occ_gather, &occ)) != PR_OK) return s;
        if (mixed) {
            int og = 1, ou = 1;
            if ((s = setup_split(PR_PREC_DF64, W, &og, &ou)) != PR_OK) return s;
            occ = std::min(occ, ou);
            occ_gather = std::min(occ_gather, og);
        }
    }
    const int budget = sms * occ, gbudget = sms * occ_gather;
    // split one-column passes gather with the hub kernel, which has tiles of its own
    const bool hub = split && hub_gather(W);
    double total_work = 0.0;
    for (auto &j : jobs) {
        s = hub ? pr_graph_hub_tiles(const_cast<pr_graph *>(j.g), W, &j.tt)
                : pr_graph_tiles(const_cast<pr_graph *>(j.g), W, &j.tt);
        if (s != PR_OK) return s;
        total_work += std::max(j.tt->work, 1.0);
    }
    int total_ctas = 0, total_gctas = 0;
    for (auto &j : jobs) {
        const double share = std::max(j.tt->work, 1.0) / total_work;
        int want = (int)std::lround(budget * share);
        if (split) {
            // update kernel: rows grid-stride
            // update kernel: rows grid-stride (the bulk-copy form: tiles of kUpdRows rows)
            const int64_t unit = update_bulk(W) ? kUpdRows : kBlock;
            j.cta_count = std::max(1, std::min<int>(want, (int)(((int64_t)j.g->n * W + unit - 1) / unit)));
            int gwant = (int)std::lround(gbudget * share);
            const int gcap = hub ? (int)std::max<int64_t>(1, ((int64_t)j.tt->ntiles + kHubWarps - 1) / kHubWarps)
                                 : tile_ctas(j.tt->ntiles);
            j.gcta_count = std::max(1, std::min(gwant, gcap));
            total_gctas += j.gcta_count;
        } else {
            j.cta_count = std::max(1, std::min(want, tile_ctas(j.tt->ntiles)));
        }
        total_ctas += j.cta_count;
    }
    // ---- workspace layout (value buffers padded for 16-byte tile copies)
    Arena ar;
    const size_t vs_max = 8;
    int max_iter_all = 1;
    for (auto &c : req.cols)
        for (auto &t : c.taps) max_iter_all = std::max(max_iter_all, t.max_iter);
    for (auto &j : jobs) {
        const size_t n = (size_t)j.g->n;
        for (int b = 0; b < 2; b++) {
            j.off_r[b] = ar.reserve((n * W + kPad) * vs_max);
            j.off_c[b] = ar.reserve((n * W + kPad) * vs_max);
        }
        j.off_cp = ar.reserve((size_t)std::max(j.tt->n_chunk_slots, 1) * W * vs_max);
        // two sets of CTA partials: persistent passes alternate between them
        j.off_part = ar.reserve(2 * (size_t)j.cta_count * W * kPartials * sizeof(double));
        if (split) j.off_rowsum = ar.reserve((n * W + kPad) * vs_max);
        for (int c : j.cols) j.ntaps += (int)req.cols[c].taps.size();
        for (int c : j.cols) j.hist_total += req.cols[c].hist_host ? req.cols[c].hist_cap : 0;
        j.off_hist = ar.reserve((size_t)std::max(j.hist_total, 1) * 3 * sizeof(double));
    }
    // all jobs' column states and stopping taps in one block (one upload, one
    // read-back), and all chunk counters in another (one memset)
    size_t total_taps = 0, total_cnt = 0;
    std::vector<size_t> tap_base(jobs.size()), cnt_base(jobs.size());
    for (size_t ji = 0; ji < jobs.size(); ji++) {
        tap_base[ji] = total_taps;
        total_taps += (size_t)jobs[ji].ntaps;
        cnt_base[ji] = total_cnt;
        total_cnt += (size_t)std::max(jobs[ji].tt->n_long, 1);
    }
    const size_t cols_bytes = jobs.size() * (size_t)W * sizeof(ColState);
    const size_t state_bytes = cols_bytes + std::max<size_t>(total_taps, 1) * sizeof(Tap);
    const size_t off_state = ar.reserve(state_bytes);
    const size_t off_cnt = ar.reserve(total_cnt * sizeof(uint32_t));
    // mixed precision keeps the FP32 phase buffers alive while the refinement
    // phase starts from them
    std::vector<size_t> off_r32;
    if (mixed)
        for (auto &j : jobs) {
            off_r32.push_back(ar.reserve(((size_t)j.g->n * W + kPad) * 4));
            off_r32.push_back(ar.reserve(((size_t)j.g->n * W + kPad) * 4));
        }
    // staging for host outputs: taps whose out is null get a device buffer,
    // reserved in the order the job loop below hands them out
    std::vector<size_t> stage_off;
    for (auto &j : jobs)
        for (int c : j.cols)
            for (auto &t : req.cols[c].taps)
                if (!t.out) stage_off.push_back(ar.reserve((size_t)j.g->n * sizeof(double)));
    const size_t off_jobs = ar.reserve(jobs.size() * sizeof(JobDev));
    const size_t off_glob = ar.reserve(sizeof(GlobalDev));
    const size_t off_ctajob = ar.reserve((size_t)total_ctas * sizeof(int32_t));
    const size_t off_gctajob = ar.reserve((size_t)std::max(total_gctas, 1) * sizeof(int32_t));
    s = ar.alloc(st);
    if (s != PR_OK) return s;
    // ---- fill job and column state on the host
    std::vector<JobDev> hjobs(jobs.size());
    std::vector<int32_t> ctajob(total_ctas), gctajob(std::max(total_gctas, 1), 0);
    int gcta_at = 0;
    std::vector<unsigned char> hstate(state_bytes, 0);
    ColState *hcols_all = reinterpret_cast<ColState *>(hstate.data());
    Tap *htaps_all = reinterpret_cast<Tap *>(hstate.data() + cols_bytes);
    ColState *dcols_all = ar.at<ColState>(off_state);
    Tap *dtaps_all = reinterpret_cast<Tap *>(ar.at<unsigned char>(off_state) + cols_bytes);
    size_t stage_i = 0;
    int cta_at = 0;
    for (size_t ji = 0; ji < jobs.size(); ji++) {
        HostJob &j = jobs[ji];
        JobDev &d = hjobs[ji];
        std::memset(&d, 0, sizeof(d));
        d.off = j.g->d_off;
        d.src = j.g->d_src;
        d.outdeg = j.g->d_outdeg;
        d.perm = j.g->d_perm;
        d.tiles = j.tt->d_tiles;
        d.slot_base = j.tt->d_slot_base;
        d.n = j.g->n;
        d.ntiles = j.tt->ntiles;
        d.cta_begin = cta_at;
        d.cta_count = j.cta_count;
        for (int q = 0; q < j.cta_count; q++) ctajob[cta_at + q] = (int32_t)ji;
        cta_at += j.cta_count;
        if (split) {
            d.gcta_begin = gcta_at;
            d.gcta_count = j.gcta_count;
            for (int q = 0; q < j.gcta_count; q++) gctajob[gcta_at + q] = (int32_t)ji;
            gcta_at += j.gcta_count;
            d.rowsum = ar.at<void>(j.off_rowsum);
            d.hub_n = hub ? j.g->n : 0;   // the kernel clamps to its value type's capacity
        }
        d.ncols = (int32_t)j.cols.size();
        d.alive = 1;
        d.cur = 0;
        if (mixed) {
            d.r[0] = ar.at<void>(off_r32[2 * ji]);
            d.r[1] = ar.at<void>(off_r32[2 * ji + 1]);
        } else {
            d.r[0] = ar.at<void>(j.off_r[0]);
            d.r[1] = ar.at<void>(j.off_r[1]);
        }
        d.contrib[0] = ar.at<void>(j.off_c[0]);
        d.contrib[1] = ar.at<void>(j.off_c[1]);
        d.chunk_part = ar.at<void>(j.off_cp);
        d.chunk_cnt = ar.at<uint32_t>(off_cnt) + cnt_base[ji];
        d.cta_part = ar.at<double>(j.off_part);
        d.cols = dcols_all + ji * (size_t)W;
        d.taps = dtaps_all + tap_base[ji];
        ColState *hcols = hcols_all + ji * (size_t)W;
        Tap *htaps = htaps_all + tap_base[ji];
        int tap_at = 0, hist_at = 0;
        for (size_t k = 0; k < j.cols.size(); k++) {
            SolveColumn &sc = req.cols[j.cols[k]];
            ColState &cs = hcols[k];
            cs.alpha = sc.alpha;
            cs.c0_base = (1.0 - sc.alpha) / (double)j.g->n;
            cs.c0_coef = sc.alpha / (double)j.g->n;
            store_value(cs.v_alpha, prec1, sc.alpha);
            store_value(cs.v_c0, prec1, 1.0 / (double)j.g->n);   // init pass: uniform start value
            cs.active = 1;
            cs.cur = 0;
            cs.tap_begin = tap_at;
            for (auto &t : sc.taps) {
                Tap tt = t;
                tt.fired = 0;
                tt.alias_of = -1;
                if (!tt.out) tt.out = ar.at<double>(stage_off[stage_i++]);
                htaps[tap_at] = tt;
                tap_at++;
            }
            cs.tap_end = tap_at;
            if (sc.hist_host) {
                cs.hist = ar.at<double>(j.off_hist) + 3 * (size_t)hist_at;
                cs.hist_cap = sc.hist_cap;
                hist_at += sc.hist_cap;
            }
            cs.init_src = sc.init_dev;
            cs.init_order = sc.init_relabelled ? 1 : 0;
            cs.init_col_stride = 1;
            cs.init_col = 0;
            if (mixed) {
                // switch on the strictest norm among the column's taps (L1 >= L2 >= Linf)
                int sn = 3;
                for (auto &t : sc.taps) sn = std::min(sn, (int)t.norm);
                cs.switch_norm = sn;
                cs.switch_tol = req.switch_tol;
            }
        }
    }
    PR_CUDA(cudaMemcpyAsync(dcols_all, hstate.data(), state_bytes, cudaMemcpyHostToDevice, st));
    PR_CUDA(cudaMemsetAsync(ar.at<uint32_t>(off_cnt), 0, total_cnt * sizeof(uint32_t), st));
    PR_CUDA(cudaMemcpyAsync(ar.at<JobDev>(off_jobs), hjobs.data(), hjobs.size() * sizeof(JobDev), cudaMemcpyHostToDevice, st));
    PR_CUDA(cudaMemcpyAsync(ar.at<int32_t>(off_ctajob), ctajob.data(), ctajob.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    PR_CUDA(cudaMemcpyAsync(ar.at<int32_t>(off_gctajob), gctajob.data(), gctajob.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    const int pass_cap = req.max_passes > 0 ? req.max_passes : max_iter_all + 3;
    // ---- loop form: persistent passes where they are asked for (or left to
    // the library), the pass is one fused kernel and its whole grid is
    // resident at once; else the CUDA graph's while-loop (or the host loop)
    int loop = req.loop;
    if (loop == PR_LOOP_AUTO || loop == PR_LOOP_PERSISTENT) {
        loop = PR_LOOP_GRAPH;
        if (!split) {
            int op = 0;
            if ((s = persist_setup(prec1, W, &op)) != PR_OK) return s;
            if (mixed) {
                int op2 = 0;
                if ((s = persist_setup(PR_PREC_DF64, W, &op2)) != PR_OK) return s;
                op = std::min(op, op2);
            }
            // every CTA of a job holds the job's stopping rules in shared memory
            bool taps_fit = true;
            for (auto &j : jobs) taps_fit = taps_fit && j.ntaps <= kPersistTaps;
            if (op > 0 && taps_fit && total_ctas <= sms * op) loop = PR_LOOP_PERSISTENT;
        }
    }
    // ---- phase 1 (or the only phase)
    s = run_phase(prec1, W, split, jobs, ar, off_jobs, off_glob, off_ctajob, total_ctas, off_gctajob, total_gctas,
                  pass_cap, loop, req.persist_wait_us, st, stats);
    if (s != PR_OK) return s;
    // ---- mixed precision: refinement phase in DF64 from the FP32 iterates
    if (mixed) {
        bool any = false;
        PR_CUDA(cudaMemcpyAsync(hstate.data(), dcols_all, state_bytes, cudaMemcpyDeviceToHost, st));
        PR_CUDA(cudaStreamSynchronize(st));
        for (size_t ji = 0; ji < jobs.size(); ji++) {
            HostJob &j = jobs[ji];
            ColState *back = hcols_all + ji * (size_t)W;
            const Tap *tback = htaps_all + tap_base[ji];
            for (size_t k = 0; k < j.cols.size(); k++) {
                ColState &cs = back[k];
                bool pending = false;
                for (int q = cs.tap_begin; q < cs.tap_end; q++) pending |= !tback[q].fired;
                cs.active = pending ? 1 : 0;
                if (pending) any = true;
                cs.switch_norm = 0;
                cs.init_src = reinterpret_cast<const double *>(ar.at<float>(off_r32[2 * ji + cs.cur]));
                cs.init_order = 1;
                cs.init_float = 1;
                cs.init_col_stride = W;
                cs.init_col = (int32_t)k;
                cs.cur = 0;
                cs.copy_dst = nullptr;
                store_value(cs.v_alpha, PR_PREC_DF64, cs.alpha);
            }
            hjobs[ji].r[0] = ar.at<void>(j.off_r[0]);
            hjobs[ji].r[1] = ar.at<void>(j.off_r[1]);
            hjobs[ji].alive = 1;
            hjobs[ji].arrive = 0;
            hjobs[ji].cur = 0;
        }
        PR_CUDA(cudaMemcpyAsync(dcols_all, hstate.data(), cols_bytes, cudaMemcpyHostToDevice, st));
        if (any) {
            PR_CUDA(cudaMemcpyAsync(ar.at<JobDev>(off_jobs), hjobs.data(), hjobs.size() * sizeof(JobDev),
                                    cudaMemcpyHostToDevice, st));
            s = run_phase(PR_PREC_DF64, W, split, jobs, ar, off_jobs, off_glob, off_ctajob, total_ctas, off_gctajob,
                          total_gctas, pass_cap, loop, req.persist_wait_us, st, stats);
            if (s != PR_OK) return s;
        }
    }
    // ---- results: taps, aliases, host copies, histories (one synchronisation
    // for all jobs' tap and column states, one launch for all alias copies)
    tap_out.assign(ncols, {});
    PR_CUDA(cudaMemcpyAsync(hstate.data(), dcols_all, state_bytes, cudaMemcpyDeviceToHost, st));
    PR_CUDA(cudaStreamSynchronize(st));
    std::vector<CopyItem> copies;
    int64_t max_n = 0;
    for (size_t ji = 0; ji < jobs.size(); ji++) {
        const Tap *tb = htaps_all + tap_base[ji];
        for (int q = 0; q < jobs[ji].ntaps; q++) {
            const Tap &t = tb[q];
            if (!t.fired) return pr_fail(PR_ETIMEOUT, "a stopping rule never fired");
            if (t.alias_of >= 0) {
                copies.push_back(CopyItem{t.out, tb[t.alias_of].out, (int64_t)jobs[ji].g->n});
                max_n = std::max<int64_t>(max_n, jobs[ji].g->n);
            }
        }
    }
    PoolBuf d_copies;
    for (size_t c0 = 0; c0 < copies.size(); c0 += 65535) {
        const size_t nc = std::min<size_t>(65535, copies.size() - c0);
        if (c0 == 0 && (s = d_copies.alloc(std::min<size_t>(copies.size(), 65535) * sizeof(CopyItem), st)) != PR_OK)
            return s;
        PR_CUDA(cudaMemcpyAsync(d_copies.p, copies.data() + c0, nc * sizeof(CopyItem), cudaMemcpyHostToDevice, st));
        const dim3 grid((unsigned)std::min<int64_t>((max_n + 1023) / 1024, 64), (unsigned)nc);
        alias_copy_kernel<<<grid, 256, 0, st>>>(static_cast<const CopyItem *>(d_copies.p));
        PR_CUDA(cudaGetLastError());
        if (c0 + nc < copies.size()) PR_CUDA(cudaStreamSynchronize(st));   // the item buffer is reused
    }
    for (size_t ji = 0; ji < jobs.size(); ji++) {
        HostJob &j = jobs[ji];
        for (size_t k = 0; k < j.cols.size(); k++) {
            SolveColumn &sc = req.cols[j.cols[k]];
            const ColState &cs = hcols_all[ji * (size_t)W + k];
            const Tap *tb = htaps_all + tap_base[ji];
            std::vector<Tap> mine(tb + cs.tap_begin, tb + cs.tap_end);
            for (size_t q = 0; q < mine.size() && q < sc.host_dst.size(); q++)
                if (sc.host_dst[q])
                    PR_CUDA(cudaMemcpyAsync(sc.host_dst[q], mine[q].out, (size_t)j.g->n * sizeof(double),
                                            cudaMemcpyDeviceToHost, st));
            tap_out[j.cols[k]] = mine;
            if (sc.final_dev && !mine.empty()) {
                // the tap that fired last holds the column's final iterate (after the alias copies above)
                size_t last = 0;
                for (size_t q = 1; q < mine.size(); q++)
                    if (mine[q].iters > mine[last].iters) last = q;
                PR_CUDA(cudaMemcpyAsync(sc.final_dev, mine[last].out, (size_t)j.g->n * sizeof(double),
                                        cudaMemcpyDeviceToDevice, st));
            }
            if (sc.hist_host && cs.hist) {
                int nh = std::min(cs.iters, sc.hist_cap);
                if (nh > 0)
                    PR_CUDA(cudaMemcpyAsync(sc.hist_host, cs.hist, (size_t)nh * 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
            }
        }
    }
    PR_CUDA(cudaStreamSynchronize(st));
    stats.columns = ncols;
    stats.mixed_columns = mixed ? ncols : 0;
    for (const auto &c : req.cols) stats.learned_columns += c.learned ? 1 : 0;
    req.stats = stats;
    return PR_OK;
}
