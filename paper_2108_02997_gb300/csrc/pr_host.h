// pr_host.h — host-side objects of the library: the graph handle, solve
// requests and their accounting, the grouping planner's interface, kernel
// selection and the live-handle registry. Included by pr_internal.cuh after
// the device-visible structures it builds on.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "pagerank.h"

// ------------------------------------------------------------------ graph object
struct pr_graph {
    uint32_t magic;
    int32_t n;
    int64_t nnz;
    int32_t n_dangling;
    int32_t device;
    void *d_mem = nullptr;           // one device allocation holding the five arrays below
    bool d_mem_pooled = false;       //   from the graph pool (else cudaMalloc)
    int32_t *d_off = nullptr;        // n+1 (padded for 16-byte bulk copies)
    int32_t *d_src = nullptr;        // nnz (padded)
    int32_t *d_outdeg = nullptr;     // n (padded)
    int32_t *d_perm = nullptr;       // relabelled -> caller
    int32_t *d_inv = nullptr;        // caller -> relabelled
    std::vector<ClassRange> classes; // in-degree classes in relabelled order
    TileTable tables[6];             // W = 1, 2, 4, 8, 16, 32
    TileTable hub_tables[3];         // W = 1, 2, 4: tiles of the hub gather kernel
    uint64_t signature = 0;          // hash of n, nnz and the in-degree class layout
};
constexpr uint32_t kGraphMagic = 0x50524731u;   // "PRG1"
constexpr uint32_t kMlpMagic = 0x50524d31u;     // "PRM1"

// Elements of padding after each graph array and value buffer, so that
// 16-byte-rounded bulk copies of any tile stay inside the allocation.
constexpr int kPad = 8;

// ------------------------------------------------------------------ errors
void pr_set_error(const std::string &msg);
void pr_clear_error();
pr_status pr_fail(pr_status s, const std::string &msg);
pr_status pr_cuda_fail(cudaError_t e, const char *what);

#define PR_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return pr_cuda_fail(_e, #call);          \
    } while (0)

// ------------------------------------------------------------------ internals
int w_index(int W);   // 1,2,4,..,32 -> 0..5
pr_status pr_graph_tiles(pr_graph *g, int W, const TileTable **out);
pr_status pr_graph_hub_tiles(pr_graph *g, int W, const TileTable **out);
bool pr_graph_valid(const pr_graph *g);

// Solve driver (pr_solve.cu)
struct SolveColumn {
    const pr_graph *g;
    double alpha;
    std::vector<Tap> taps;          // filled with out pointers (device, caller order)
    std::vector<int32_t> inst;      // instance index of each tap
    std::vector<double *> host_dst; // per tap: host buffer to receive the answer, or null
    const double *init_dev = nullptr;   // device start vector, or null
    bool init_relabelled = false;       // init_dev in relabelled order (else caller order)
    double *hist_host = nullptr;
    int32_t hist_cap = 0;
    bool learned = false;               // init_dev is the learned start
    double *final_dev = nullptr;        // optional: device, n doubles (caller order) receiving the
                                        // column's final iterate (its last stopping rule's answer)
};

// Launch accounting of one solve (or the sum over a request's sub-solves).
struct SolveStats {
    int launches = 0;       // kernel launches, init passes included
    int passes = 0;         // iteration passes the device performed
    double kernel_ms = 0.0; // PR_LOOP_HOST: sum of the iteration launches' event times
    double total_ms = 0.0;  // device time of the whole solve
    double gather_ms = 0.0; // PR_LOOP_HOST, split passes: the gather kernels' share of kernel_ms
    double update_ms = 0.0; //   and the update kernels' share
    int columns = 0;        // columns (iterate sequences) solved
    int mixed_columns = 0;  //   of which in mixed precision
    int learned_columns = 0;//   of which from the learned start
    int loop_phases[3] = {0, 0, 0};  // phases run per loop form (pr_loop: graph, host, persistent)
    void add(const SolveStats &o) {
        launches += o.launches; passes += o.passes; kernel_ms += o.kernel_ms; total_ms += o.total_ms;
        gather_ms += o.gather_ms; update_ms += o.update_ms; columns += o.columns;
        mixed_columns += o.mixed_columns; learned_columns += o.learned_columns;
        for (int i = 0; i < 3; i++) loop_phases[i] += o.loop_phases[i];
    }
};

struct SolveRequest {
    int precision = PR_PREC_DF64;
    int loop = PR_LOOP_GRAPH;
    double switch_tol = 1e-6;
    cudaStream_t stream = nullptr;
    std::vector<SolveColumn> cols;
    // Optional explicit jobs: lists of column indices, all on one graph, at most
    // 32 each; empty = the columns of each graph packed 32 at a time.
    std::vector<std::vector<int>> jobs;
    int max_passes = 0;     // 0: the largest max_iter + 3
    int kernels = PR_KERNELS_AUTO;
    int persist_wait_us = 0;   // persistent passes: bound of one wait (0: the default)
    SolveStats stats;       // out
};

// Test hook: while set, the CTAs of persistent passes never announce the end
// of a pass, so that every wait runs out (pr_test_hold_decisions).
bool pr_hold_decisions();

pr_status pr_run_solve(SolveRequest &req, std::vector<std::vector<Tap>> &tap_out);
void pr_record_last_stats(const SolveStats &s);

// Column grouping (pr_plan.cu). A sub-solve is one pr_run_solve: jobs of one
// width W, given as lists of request column indices.
struct SubSolve {
    int W = 1;
    int precision = PR_PREC_DF64;   // never PR_PREC_AUTO
    std::vector<std::vector<int>> jobs;
};
pr_status pr_plan_request(const SolveRequest &req, int group, std::vector<SubSolve> &plan);

// Kernel selection and launch geometry (pr_solve.cu)
void *pr_iter_kernel_for(int precision, int W);
void *pr_init_kernel_for(int precision, int W);
size_t pr_tile_smem_bytes(int precision, int W);
pr_status pr_kernel_setup(int precision, int W, int *blocks_per_sm);
// CTAs a job of ntiles warp tiles is given in a fused pass (at most one per
// kMinTilesPerWarp tiles of each warp).
int tile_ctas(int32_t ntiles);

// Graph arrays from the per-device graph pool (pr_solve.cu); pr_graph_free
// waits for the device, as cudaFree does, before returning them.
pr_status pr_graph_alloc(void **p, size_t bytes, bool *pooled);
void pr_graph_free(void *p, bool pooled);

// Stream-ordered device buffer from the per-device workspace pool
// (pr_solve.cu): released with cudaFreeAsync on the stream it was taken on,
// so repeated calls reuse memory without the synchronising cudaMalloc and
// cudaFree. Falls back to cudaMalloc when the pool cannot serve the request.
struct PoolBuf {
    void *p = nullptr;
    cudaStream_t stream = nullptr;
    bool pooled = false;
    PoolBuf() = default;
    PoolBuf(const PoolBuf &) = delete;
    PoolBuf &operator=(const PoolBuf &) = delete;
    ~PoolBuf() { release(); }
    pr_status alloc(size_t bytes, cudaStream_t st);
    void release();
};

// Learned warm start (pr_learn.cu). The features of the network's input
// depend on the graph only (alpha enters the network separately), so a batch
// computes them once per graph: pr_learned_features writes them (relabelled
// order, pr_learned_features_bytes(g) bytes) and pr_learned_start takes them
// (or computes its own when feat is null). The start vector is FP64 on the
// device, in relabelled order when `relabelled`, else caller order.
bool pr_mlp_valid(const pr_mlp *m);
size_t pr_learned_features_bytes(const pr_graph *g);
pr_status pr_learned_features(const pr_graph *g, void *feat, cudaStream_t st);
pr_status pr_learned_start(const pr_mlp *m, const pr_graph *g, double alpha, double *d_out, bool relabelled,
                           cudaStream_t st, const void *feat = nullptr);
// PR_INIT_AUTO's inputs: the network's gain (e-folds of start error removed;
// 0 when unknown), the learned start's device time on g (features once per
// graph, network per alpha; measured once per device and graph signature),
// and the tuned one-column launch time, the latency that jobs sharing a
// launch share, and the L1 decay rate of g (pr_plan.cu).
double pr_mlp_gain_value(const pr_mlp *m);
pr_status pr_learned_cost(const pr_mlp *m, const pr_graph *g, cudaStream_t st, double *feat_us, double *net_us);
pr_status pr_graph_pass_model(pr_graph *g, cudaStream_t st, double *t1_us, double *lat_us, double *rho_l1);

// Live-handle registry: guards every entry point against stale handles.
void registry_add(const void *p);
void registry_remove(const void *p);
bool registry_has(const void *p);
