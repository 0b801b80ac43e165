// pr_internal.cuh — shared definitions of libpagerank.so (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "pagerank.h"

// ------------------------------------------------------------------ launch geometry
constexpr int kBlock = 256;          // threads per CTA of every iteration kernel
constexpr int kWarps = kBlock / 32;
constexpr int kPartials = 5;         // L1, sum of squares, Linf, dangling sum, sum of ranks
// Warp tiles. One column (W = 1): a rows tile holds at most kTileValues
// in-edges and 128 rows; longer rows are cut into chunks of kChunkValues
// in-edges. 224 values keep the gather kernel's staging buffers (8-byte
// values) at 14 KB per CTA, so that four CTAs fit the 64 KB shared-memory
// configuration and L1 keeps the rest (measured on GB300, df64 gather launch:
// 7-10 % faster than 256 values on R-MAT and configuration-model graphs). Several columns (W > 1): a lane reads the values of one in-edge for
// vec_cols adjacent columns with one vector load, a rows tile holds at most 256
// in-edges and 192 / W rows, and chunks hold 8192 / W in-edges (at least 256). The sizes are compile-time tuning constants.
#ifndef PR_TILE_VALUES
#define PR_TILE_VALUES 224
#endif
#ifndef PR_CHUNK_VALUES
#define PR_CHUNK_VALUES 4096
#endif
#ifndef PR_MIN_BLOCKS
#define PR_MIN_BLOCKS 3
#endif
#ifndef PR_SPLIT_PASSES
#define PR_SPLIT_PASSES 1
#endif
#ifndef PR_GATHER_MIN_BLOCKS
#define PR_GATHER_MIN_BLOCKS 4
#endif
#ifndef PR_UPDATE_MIN_BLOCKS
#define PR_UPDATE_MIN_BLOCKS 3
#endif
// One-column update kernel: pairs of rows (vector loads) in flight per thread.
// One column, split passes: the update kernel streams its rows' inputs into
// shared memory with 1-D bulk copies (1), or loads them per thread (0).
#ifndef PR_UPDATE_BULK
#define PR_UPDATE_BULK 1
#endif
constexpr bool kUpdateBulk = PR_UPDATE_BULK != 0;
constexpr int kUpdRows = 1024;     // rows per bulk-copied tile
constexpr int kUpdStages = 3;      // tiles in flight per CTA
__host__ __device__ constexpr int upd_stage_bytes(int vbytes) { return kUpdRows * (2 * vbytes + 4); }
#ifndef PR_UPDATE_PAIRS
#define PR_UPDATE_PAIRS 2
#endif
#ifndef PR_TILE_UPDATE
#define PR_TILE_UPDATE 1
#endif
#ifndef PR_STREAM_INDEX
#define PR_STREAM_INDEX 1
#endif
#ifndef PR_SMEM_CARVEOUT
#define PR_SMEM_CARVEOUT -1
#endif
#ifndef PR_VEC_MIN_BLOCKS_4B
#define PR_VEC_MIN_BLOCKS_4B 3
#endif
#ifndef PR_VEC_MIN_BLOCKS_8B
#define PR_VEC_MIN_BLOCKS_8B 2
#endif
#ifndef PR_VEC_GATHER_BATCH
#define PR_VEC_GATHER_BATCH 4
#endif
// One column, 8-byte values: a rows tile's row sums go to shared memory and all
// 32 lanes then update the tile's rows (consecutive rows on consecutive lanes),
// instead of the one lane per lane group that formed each sum (measured: 2-3 %
// faster for df64, 1-3 % slower for float, whose update is cheap).
constexpr bool kTileUpdate = PR_TILE_UPDATE != 0;
// Each pass runs as two kernels: a gather kernel that only forms the row sums
// (fewer registers, more resident warps) and a streaming update kernel (new
// ranks, contributions, norms, stopping rules).
constexpr bool kSplitPasses = PR_SPLIT_PASSES != 0;
// PR_KERNELS_AUTO splits passes from this many in-edge columns per sub-solve
// (smaller solves are launch-bound and one launch per pass is cheaper).
constexpr double kSplitMinWork = 16.0e6;
constexpr int kGatherMinBlocks = PR_GATHER_MIN_BLOCKS;
constexpr int kUpdateMinBlocks = PR_UPDATE_MIN_BLOCKS;
#ifndef PR_VEC_GATHER_MIN_BLOCKS
#define PR_VEC_GATHER_MIN_BLOCKS 3
#endif
constexpr int kVecGatherMinBlocks = PR_VEC_GATHER_MIN_BLOCKS;   // several columns, gather kernel
// One column: in-edge indices loaded evict-first (read once per pass; 1-4 %
// faster than default caching, measured).
constexpr bool kStreamIndex = PR_STREAM_INDEX != 0;
// Shared-memory carveout of the iteration kernels: -1 (default) asks, for the
// one-column gather kernel, for the smallest share of the unified L1/shared
// storage that still holds as many CTAs per SM as the registers allow (the
// rest caches the random gathers in L1) and leaves the driver's choice for the
// others; -2 leaves the driver's choice everywhere; 0..100 forces a percentage.
constexpr int kSmemCarveout = PR_SMEM_CARVEOUT;
constexpr int kTileValues = PR_TILE_VALUES;
// Resident CTAs per SM asked of the compiler for W > 1, by value size: with
// 8-byte values (df64, FP64) three CTAs force register spills that cost more
// than the third CTA gains (measured: 1.4-1.8x slower per launch).
__host__ __device__ constexpr int vec_min_blocks(int vbytes) { return vbytes == 4 ? PR_VEC_MIN_BLOCKS_4B : PR_VEC_MIN_BLOCKS_8B; }
constexpr int kVecGatherBatch = PR_VEC_GATHER_BATCH;  // vector gathers per lane issued together (W > 1)
// A job gets at most one CTA per kMinTilesPerWarp * kWarps of its warp tiles
// (0: one CTA per tile).
#ifndef PR_MIN_TILES_PER_WARP
#define PR_MIN_TILES_PER_WARP 1
#endif
constexpr int kMinTilesPerWarp = PR_MIN_TILES_PER_WARP;
constexpr int kChunkValues = PR_CHUNK_VALUES;
// One column, split passes: the gather kernel runs one CTA of kHubBlock
// threads per SM and keeps the contributions of the first vertices in the
// relabelled order (the highest in-/out-degree classes, the most gathered
// sources) in shared memory, up to kHubBytes; their gathers read shared memory
// instead of L1/L2. Its warps stage kHubTile gathered values each.
#ifndef PR_HUB_GATHER
#define PR_HUB_GATHER 1
#endif
#ifndef PR_HUB_TILE_VALUES
#define PR_HUB_TILE_VALUES 224
#endif
#ifndef PR_HUB_BYTES
#define PR_HUB_BYTES (96 * 1024)
#endif
#ifndef PR_HUB_CHUNK_PER
#define PR_HUB_CHUNK_PER 8
#endif
constexpr bool kHubGather = PR_HUB_GATHER != 0;
constexpr int kHubBlock = 1024;
constexpr int kHubWarps = kHubBlock / 32;
constexpr int kHubTile = PR_HUB_TILE_VALUES;
constexpr int kHubBytes = PR_HUB_BYTES;
// Jobs of two and four columns keep a smaller hub table: their gathers read a
// whole vector per source, and the L1 that a smaller table leaves serves them
// better (measured on GB300, df64, R-MAT s24: two columns 1249 -> 1096 us and
// four columns 2036 -> 1826 us per pass from 96 KB to 32 KB of hubs).
#ifndef PR_HUB_BYTES_VEC
#define PR_HUB_BYTES_VEC (32 * 1024)
#endif
__host__ __device__ constexpr int hub_bytes(int W) { return W == 1 ? PR_HUB_BYTES : PR_HUB_BYTES_VEC; }
constexpr int kHubChunkPer = PR_HUB_CHUNK_PER;   // chunk tiles: gathers in flight per lane
static_assert(kHubTile % 32 == 0 && kHubTile <= 256, "hub tiles hold 32..256 values");
// Gathers of 32 bytes (four df64 or FP64 columns of a source): one 256-bit
// load per lane (1) or two 128-bit loads (0). Measured on GB300, df64, four
// columns: R-MAT s22 554 -> 484 us, s24 2165 -> 2036 us per gather pass.
#ifndef PR_GATHER_V8
#define PR_GATHER_V8 1
#endif
constexpr bool kGatherV8 = PR_GATHER_V8 != 0;
#ifndef PR_HUB_TILE_VECTORS
#define PR_HUB_TILE_VECTORS 128
#endif
// In-edges per rows tile of the hub gather kernel: kHubTile for one column,
// PR_HUB_TILE_VECTORS for two, half that for four (their staged vectors are
// wider).
__host__ __device__ constexpr int hub_tile_edges(int W) {
    return W == 1 ? kHubTile : (W == 2 ? PR_HUB_TILE_VECTORS : PR_HUB_TILE_VECTORS / 2);
}
// Jobs of W columns gather with the hub kernel when a vertex's W values fill at
// most one 32-byte sector.
__host__ __device__ constexpr bool hub_width_ok(int W, int vbytes) { return (W == 1 || W == 2 || W == 4) && W * vbytes <= 32; }
constexpr int kMinBlocks = PR_MIN_BLOCKS;
constexpr int kVecTileEdges = 256;
__host__ __device__ constexpr int tile_edges(int W) { return W == 1 ? kTileValues : kVecTileEdges; }
__host__ __device__ constexpr int tile_rows(int W) { return W == 1 ? 128 : 192 / W; }
__host__ __device__ constexpr int chunk_edges(int W) { return W == 1 ? kChunkValues : (8192 / W > 256 ? 8192 / W : 256); }

// Several columns: columns per vector load (16 bytes, or the whole row of W
// values when that is shorter) for values of vbytes bytes.
__host__ __device__ constexpr int vec_cols(int vbytes, int W) { return W * vbytes >= 16 ? 16 / vbytes : W; }
__host__ __device__ constexpr int round16(int b) { return (b + 15) & ~15; }
// Per-warp shared buffers of a multi-column tile, in bytes and in this order:
// gathered vectors [kVecTileEdges], row sums [tile_rows * W], in-edge sources
// [kVecTileEdges], row offsets [tile_rows + 1], and, when the kernel also
// updates the rows (not the gather-only kernel), previous ranks
// [tile_rows * W] and out-degrees [tile_rows].
__host__ __device__ constexpr int vec_vals_bytes(int vbytes, int W) { return kVecTileEdges * vec_cols(vbytes, W) * vbytes; }
__host__ __device__ constexpr int vec_rows_bytes(int vbytes, int W) { return round16(tile_rows(W) * W * vbytes); }
__host__ __device__ constexpr int vec_warp_bytes(int vbytes, int W, bool gather_only) {
    return vec_vals_bytes(vbytes, W) + vec_rows_bytes(vbytes, W) + kVecTileEdges * 4 + round16((tile_rows(W) + 1) * 4) +
           (gather_only ? 0 : vec_rows_bytes(vbytes, W) + round16(tile_rows(W) * 4));
}

// ------------------------------------------------------------------ work tiles
// A tile is one warp's work item of one pass: either a run of consecutive rows
// of one in-degree class (at most tile_rows rows and tile_edges in-edges in
// total), or one chunk of the in-edges of a row longer than tile_edges.
//   rows : [r0, r1) rows, [e0, e1) = their in-edges, glog = log2(lanes per row)
//   chunk: r0 = the row, r1 = r0 + 1, [e0, e1) = this chunk, glog = -1,
//          slot = long-row slot (-1 when the row has one chunk), k = chunk index,
//          nch = chunks of the row
struct Tile {
    int32_t r0, r1, e0, e1;
    int32_t glog, slot, k, nch;
};

struct TileTable {
    int W = 0;                   // column width this table was built for
    void *d_mem = nullptr;       // one device allocation holding d_tiles and d_slot_base
    bool d_mem_pooled = false;   //   from the graph pool (else cudaMalloc)
    Tile *d_tiles = nullptr;
    int32_t ntiles = 0;
    int32_t n_long = 0;          // rows split into more than one chunk
    int32_t n_chunk_slots = 0;   // chunk partial slots
    int32_t *d_slot_base = nullptr;  // n_long: first chunk partial of each long row
    double work = 0.0;           // relative work estimate
};

struct ClassRange {
    int32_t begin, end;   // rows [begin, end) in the relabelled order
    int32_t max_deg;      // largest in-degree in the range
};

// ------------------------------------------------------------------ device state
// One column of a job: one iterate sequence (an instance, or a shared
// trajectory feeding several instances).
struct ColState {
    double alpha;
    double c0;            // teleport term of the next update (FP64)
    double c0_base;       // (1 - alpha)/N and alpha/N: c0 = c0_base + c0_coef * (dangling sum),
    double c0_coef;       //   the two divisions of Section 2's c0 done once on the host
    double v_alpha[2];    // alpha in the job's value type (raw bits: 4 or 8 bytes used)
    double v_c0[2];       // c0 in the job's value type (init pass: the uniform start 1/N)
    int32_t active;       // 1 while the column still updates
    int32_t cur;          // buffer (0/1) holding the current iterate
    int32_t iters;        // updates performed so far
    int32_t tap_begin, tap_end;   // this column's taps in the tap array
    double *copy_dst;     // tap output to fill from the current iterate in the next pass
    double *hist;         // optional: 3 doubles per iteration (L1, L2, Linf)
    int32_t hist_cap;
    int32_t switch_norm;  // mixed precision: norm of the phase-switch test (0 = none)
    double switch_tol;
    int32_t switched;     // set when the phase-switch test has passed
    int32_t pad;
    double last_err[3];
    double last_sum;      // sum of the latest iterate (diagnostic)
    const double *init_src;   // init pass: start vector (nullptr = uniform)
    int32_t init_order;   // 0: caller order (index by perm), 1: relabelled order
    int32_t init_float;   // 1: init_src points to floats (phase switch from FP32)
    int32_t init_col_stride;  // elements between consecutive vertices in init_src
    int32_t init_col;     // column offset in init_src
};

// A stopping rule read off a column (Section 3 norm, Section 4 tau).
struct Tap {
    double tau;
    int32_t norm;
    int32_t max_iter;
    int32_t fired;        // 0 pending, 1 fired
    int32_t iters;
    int32_t converged;
    int32_t alias_of;     // -1, or the tap whose output this one copies (same iterate)
    double err;
    double err_l1;        // L1 norm of the deciding step
    double *out;          // device, n doubles, caller order
};

struct JobDev {
    const int32_t *off;
    const int32_t *src;
    const int32_t *outdeg;
    const int32_t *perm;      // relabelled -> caller id
    const Tile *tiles;
    const int32_t *slot_base;
    int32_t n;
    int32_t ntiles;
    int32_t cta_begin, cta_count;
    int32_t ncols;
    int32_t alive;            // 1 while any column is active or a copy is pending
    void *r[2];               // n x W value arrays
    void *contrib[2];
    void *chunk_part;         // n_chunk_slots x W values
    uint32_t *chunk_cnt;      // n_long counters
    double *cta_part;         // cta_count x W x kPartials
    ColState *cols;           // W
    Tap *taps;
    uint32_t arrive;          // CTAs of this job that finished the pass
    int32_t cur;              // buffer parity shared by the job's active columns
    void *rowsum;             // one column, split passes: the n row sums of the pass
    int32_t gcta_begin, gcta_count;   // CTAs of the gather pass (split passes)
    int32_t hub_n;            // hub gather kernel: contributions of ids [0, hub_n) held in shared memory
    int32_t pad_hub;
};

struct GlobalDev {
    // jobs that finished the current pass (high 32 bits) and, of those, the
    // ones still alive (low 32 bits): one atomic per job finalizer
    unsigned long long arrive_alive;
    int32_t njobs;
    int32_t pass;             // body executions so far
    int32_t pass_cap;         // hard cap on body executions
    int32_t alive;            // set by the last job to finish a pass
    int32_t error;            // nonzero: a device-side check failed
    int32_t hold;             // persistent passes, test hook: CTAs never announce the end of a pass
    unsigned long long cond;  // cudaGraphConditionalHandle (0 in host-loop mode)
    uint32_t body_count;      // iteration launches started (independent loop guard)
    uint32_t wait_us;         // persistent passes: bound of one wait for the job's CTAs (0: kPersistWaitNs)
};

// Error codes a kernel can leave in GlobalDev::error.
enum DeviceError { kErrNone = 0, kErrPassCap = 2, kErrLoopGuard = 3, kErrWait = 4 };

// Persistent passes: the longest a CTA waits for the other CTAs of its job
// (global timer nanoseconds) before it records kErrWait and stops.
#ifndef PR_PERSIST_WAIT_NS
#define PR_PERSIST_WAIT_NS 2000000000ull
#endif
constexpr unsigned long long kPersistWaitNs = PR_PERSIST_WAIT_NS;

// Host-side objects (graph handle, solve requests, planner, registry).
#include "pr_host.h"
