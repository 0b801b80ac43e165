/*
 * pagerank.h — C ABI of libpagerank.so: pull power-iteration PageRank with
 * L1 / L2 / Linf convergence checks on one NVIDIA GB300 (sm_103a).
 *
 * The method (paper "Adjusting PageRank parameters and Comparing results"):
 *   r^0       = 1/N (or a given start)
 *   c0        = (1 - alpha)/N + alpha * (sum of r over dangling vertices)/N   (Section 2)
 *   r^i[v]    = c0 + alpha * sum_{u -> v} r^{i-1}[u] / outdeg(u)             (Section 2)
 *   err       = ||r^i - r^{i-1}||, L1 = sum|.|, L2 = sqrt(sum|.|^2),
 *               Linf = max|.|                                                 (Section 3)
 *   stop when err < tau (converged) or after max_iter updates (not converged;
 *   the paper caps at 500, Section 2, and halts there, Section 4).
 * The iteration count returned is the number of updates performed, including
 * the one whose error passed the test.
 *
 * Conventions for every entry point:
 *   - Return PR_OK (0) or an error code; on error pr_last_error() gives a
 *     message (thread-local, valid until the next call on that thread) and no
 *     caller-owned output buffer has been written.
 *   - Non-convergence is not an error: PR_OK with converged = 0 and
 *     iterations = max_iter.
 *   - Host pointers are plain CPU memory. Device pointers are CUDA global
 *     memory of the current device. Which one an argument is, is stated per
 *     argument.
 *   - Device memory. A graph's arrays are allocated by pr_graph_create and
 *     freed by pr_graph_destroy, from a stream-ordered memory pool of their
 *     own per device (graph pool). Everything else (solve and training
 *     workspaces, graph-creation scratch) comes from a second stream-ordered
 *     memory pool per device, the workspace pool (cudaMallocFromPoolAsync on
 *     the call's stream, cudaFreeAsync before the call returns). Either falls
 *     back to cudaMalloc only if its pool cannot serve a request. Each pool
 *     keeps up to 16 GiB of freed memory reserved so that repeated calls and
 *     graphs do not pay the synchronising cudaMalloc/cudaFree and the page
 *     mapping behind them; pr_workspace_info reports what the workspace pool
 *     holds and pr_workspace_release returns the unused part of both pools
 *     to the device. pr_graph_destroy waits for the device before it returns
 *     a graph's memory.
 *     pr_solve_noalloc allocates nothing (see there).
 *   - Per-device set-up (kernel attributes, residencies, the tuning table,
 *     the no-alloc array's address) is done once per device and process; the
 *     library does not survive a cudaDeviceReset of a device it has used.
 *   - A graph handle may be used by one solve at a time.
 *   - Calls are synchronous with respect to the host unless stated otherwise;
 *     device work is issued on the stream given in pr_options (NULL: the
 *     legacy default stream).
 */
#ifndef PAGERANK_H
#define PAGERANK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pr_graph pr_graph;   /* opaque device-resident graph */

typedef enum pr_status {
    PR_OK = 0,
    PR_EINVAL = 1,    /* invalid argument or malformed graph */
    PR_ENOMEM = 2,    /* host or device allocation failed */
    PR_ECUDA = 3,     /* a CUDA runtime call failed */
    PR_ETIMEOUT = 4,  /* a bounded device-side wait ran out */
    PR_ESTATE = 5,    /* handle in the wrong state (e.g. destroyed) */
    PR_ENOTSUP = 6    /* option combination not supported */
} pr_status;

/* Convergence norms of Section 3. */
typedef enum pr_norm { PR_NORM_L1 = 1, PR_NORM_L2 = 2, PR_NORM_LINF = 3 } pr_norm;

/* Arithmetic of the device iteration.
 *  PR_PREC_DF64 : ranks and contributions stored as float pairs (hi + lo,
 *                 about 48 significant bits); every per-edge and per-vertex
 *                 operation runs on the FP32 pipes; block/grid reductions,
 *                 c0 and the norms finish in FP64. Default: GB300 executes
 *                 FP64 at about 1/69 of its FP32 rate, so this is the
 *                 FP64-class path that stays memory-bound.
 *  PR_PREC_FP64 : native IEEE double everywhere (FP64-pipe bound on GB300).
 *  PR_PREC_MIXED: FP32 ranks, gathers and accumulation until the norm is at
 *                 or below switch_tol, then DF64 refinement to tau. The
 *                 dangling sum, c0 and the norms stay FP64-class throughout.
 *  PR_PREC_FP32 : FP32 ranks/gathers/accumulation throughout (norms FP64-class).
 *  PR_PREC_AUTO : per graph of a pr_solve_batch call, PR_PREC_MIXED where the
 *                 grouping planner's cost model (the launch times pr_graph_tune
 *                 measures for FP32 and DF64, and each column's estimated
 *                 iterations in both phases, the refinement phase damping the
 *                 FP32 iterate's rounding noise at the rate alpha) predicts it
 *                 cheaper than DF64 throughout, else PR_PREC_DF64. Graphs with a
 *                 single column, and every graph under PR_GROUP_PACK or
 *                 PR_GROUP_SINGLE, run DF64. The accuracy is that of the
 *                 precision chosen.
 */
typedef enum pr_precision {
    PR_PREC_DF64 = 0,
    PR_PREC_FP64 = 1,
    PR_PREC_MIXED = 2,
    PR_PREC_FP32 = 3,
    PR_PREC_AUTO = 4
} pr_precision;

/* Start vector r^0. */
typedef enum pr_init {
    PR_INIT_UNIFORM = 0,  /* 1/N everywhere */
    PR_INIT_USER = 1,     /* caller's vector, used as given (not renormalised) */
    PR_INIT_LEARNED = 2,  /* MLP warm start (pr_mlp), renormalised to sum 1 */
    PR_INIT_CHAIN = 3,    /* alpha continuation (pr_solve_batch): on each graph
                             the columns (iterate sequences) are taken in
                             increasing alpha; the first starts from 1/N and each
                             later one from the final iterate of the one before
                             it (its answer at its last stopping rule). The
                             columns of one graph then run one after another
                             (those of different graphs side by side); the
                             alpha sweep of Section 2 in the order it is swept */
    PR_INIT_AUTO = 4      /* pr_solve_batch with a pr_mlp: per (graph, alpha)
                             column, the learned start where its predicted
                             saving exceeds its measured cost, else 1/N. The
                             network removes about `gain` e-folds of the start's
                             L1 error (pr_mlp_gain), which at the column's
                             contraction rate (alpha times the graph's decay
                             measured by pr_graph_tune, relative to 0.85) saves
                             gain / ln(1/rate) updates, each worth the tuned
                             one-column launch time (less the latency that
                             jobs sharing a launch share, when the graph has
                             several columns); the cost is the network's device time
                             per alpha plus the features' per graph, divided
                             over the graph's alphas (both measured on first
                             use per graph signature). A network without a
                             positive gain is never used. */
} pr_init;

/* Device-side loop control (Section 2's iteration until the stopping rule
 * holds or the cap is reached). */
typedef enum pr_loop {
    PR_LOOP_GRAPH = 0,    /* one CUDA graph whose while-node repeats the
                             iteration kernel(s) until every instance has
                             stopped; the stop decision is taken on the device */
    PR_LOOP_HOST = 1,     /* one launch per iteration and a device-to-host read
                             of the stop flag after each (the plain per-instance
                             baseline; also used to time single launches) */
    PR_LOOP_PERSISTENT = 2, /* every iteration pass in one cooperative launch:
                             the CTAs stay resident; at the end of a pass each
                             CTA waits, on its job's device counter, for the
                             job's other CTAs, and takes the job's stop
                             decision itself from all their partials (no
                             launch between passes, no CTA deciding for the
                             others). Used where a pass is one fused kernel,
                             its whole grid fits on the device at once and no
                             job has more than 256 stopping rules; otherwise
                             the solve runs as PR_LOOP_GRAPH. Each wait is
                             bounded (2 s of device time): a wait that runs
                             out ends the solve with PR_ETIMEOUT and leaves
                             the context usable */
    PR_LOOP_AUTO = 3      /* default: PR_LOOP_PERSISTENT where it applies, else
                             PR_LOOP_GRAPH */
} pr_loop;

/* How pr_solve_batch packs its columns (iterate sequences) into jobs. A job
 * holds up to W columns of one graph as an N x W vertex-major matrix, so that
 * one read of a row's in-edge indices serves all W columns; every job of a
 * solve advances in the same kernel launches, and a job stops costing time
 * once its last column has stopped. Packing columns whose iteration counts
 * differ makes the short ones wait on the long one, and a wide job gathers
 * more bytes per in-edge, so the best packing depends on the graph.
 * Grouping changes only the order of floating-point additions: every
 * grouping meets the same accuracy bounds. */
typedef enum pr_group {
    PR_GROUP_AUTO = 0,    /* default: per graph, columns sorted by their
                             estimated iteration counts (the error decay that
                             pr_graph_tune measures, scaled to each alpha; else
                             log(tau)/log(alpha), Section 1) are cut into the
                             contiguous jobs that minimise the sum over jobs of
                             (iterations x launch time at the job's width); as
                             jobs of one width share each launch and its
                             latency, the cheapest of that partition, the one
                             for launch times less the latency, and one job per
                             column is kept (pr_plan_columns_shared). Launch
                             times and latency come from pr_graph_tune, run
                             automatically the first time a graph with two or
                             more columns meets this mode (cached per process by
                             graph signature: vertices, edges and in-degree
                             class layout). The grouping can differ between
                             processes, hence so can the last bits. */
    PR_GROUP_PACK = 1,    /* the columns of each graph packed 32 at a time */
    PR_GROUP_SINGLE = 2   /* one column per job (W = 1) */
} pr_group;

/* How an iteration pass runs on the device. */
typedef enum pr_kernels {
    PR_KERNELS_AUTO = 0,   /* default: split passes when a sub-solve's work (in-edges
                              x column width, summed over its jobs) is at least
                              16 million, one fused kernel below that (where one
                              launch per pass is cheaper) */
    PR_KERNELS_FUSED = 1,  /* one kernel per pass: gathers, row sums, updates,
                              norms and stopping rules */
    PR_KERNELS_SPLIT = 2   /* two kernels per pass: a gather kernel that forms the
                              row sums, then a streaming update kernel */
} pr_kernels;

typedef struct pr_mlp pr_mlp;   /* learned warm start, see pr_mlp_* below */

typedef struct pr_options {
    int32_t precision;          /* pr_precision; default PR_PREC_DF64 */
    int32_t init;               /* pr_init; default PR_INIT_UNIFORM */
    const double *init_vec;     /* PR_INIT_USER: n doubles in the caller's vertex
                                   order (host, or device if init_on_device) */
    int32_t init_on_device;     /* 1: init_vec is a device pointer */
    int32_t outputs_on_device;  /* 1: every ranks_out is a device pointer */
    double switch_tol;          /* PR_PREC_MIXED: FP32 phase ends when err <= this;
                                   default 1e-6 */
    void *stream;               /* cudaStream_t, or NULL for the default stream */
    int32_t share_trajectories; /* pr_solve_batch: 1 (default) lets instances that
                                   share (graph, alpha, start, precision) read their
                                   answers off one iterate sequence; 0 gives every
                                   instance its own column */
    int32_t loop;               /* pr_loop; default PR_LOOP_AUTO */
    const pr_mlp *mlp;          /* PR_INIT_LEARNED: trained network */
    double *err_history;        /* pr_solve only, optional host buffer of
                                   3*max_iter doubles: row i-1 = (L1, L2, Linf)
                                   of r^i - r^{i-1} */
    int32_t group;              /* pr_group; default PR_GROUP_AUTO */
    int32_t max_passes;         /* watchdog: iteration passes the device may run
                                   in one phase before the solve is abandoned
                                   with PR_ETIMEOUT (the device stops itself;
                                   the context stays usable); 0 (default) =
                                   the largest max_iter + 3 */
    int32_t kernels;            /* pr_kernels; default PR_KERNELS_AUTO */
    int32_t persist_wait_us;    /* PR_LOOP_PERSISTENT: bound of one wait for the
                                   other CTAs of a job, microseconds; 0
                                   (default) = 2,000,000 */
    int32_t reserved[4];        /* zero */
} pr_options;

/* Fill *opt with the defaults listed above. */
void pr_options_default(pr_options *opt);

/*
 * Create a device-resident graph from an in-edge CSR (Section 2: the pull
 * update reads, for each vertex v, its in-neighbours u and their out-degrees).
 *   n           : vertices, 1 <= n < 2^31
 *   nnz         : edges, 0 <= nnz < 2^31
 *   in_offsets  : host, n+1 int32, in_offsets[0] = 0, non-decreasing,
 *                 in_offsets[n] = nnz
 *   in_sources  : host, nnz int32 in [0, n): the tails u of the edges u -> v,
 *                 row v at in_offsets[v] .. in_offsets[v+1]-1 (NULL if nnz = 0)
 *   out_degree  : host, n int32 >= 0; must equal the number of times each
 *                 vertex occurs in in_sources (vertices with 0 are dangling)
 *   out         : receives the handle
 * The library copies the arrays; the caller keeps ownership. The device copy
 * is relabelled by in-degree (hubs first) for load balance and gather
 * locality; every rank vector crossing the ABI is in the caller's order.
 * Errors: PR_EINVAL for a malformed CSR, PR_ENOMEM, PR_ECUDA.
 */
pr_status pr_graph_create(int32_t n, int64_t nnz, const int32_t *in_offsets,
                          const int32_t *in_sources, const int32_t *out_degree,
                          pr_graph **out);

/* Release a graph and its device memory. NULL is accepted. */
pr_status pr_graph_destroy(pr_graph *g);

/* Vertex, edge and dangling-vertex counts of a graph (any pointer may be NULL). */
pr_status pr_graph_info(const pr_graph *g, int32_t *n, int64_t *nnz, int32_t *n_dangling);

/*
 * Solve one instance (Sections 2-4).
 *   alpha     : damping factor in [0, 1] (1 allowed: the paper sweeps to 1.00)
 *   tol       : tau > 0, finite
 *   norm      : pr_norm
 *   max_iter  : >= 1
 *   opt       : NULL for defaults
 *   ranks_out : n doubles, caller order (host, or device if
 *               opt->outputs_on_device); the iterate at the stopping iteration
 *   iters_out, err_out, converged_out : host, may be NULL
 */
pr_status pr_solve(const pr_graph *g, double alpha, double tol, int32_t norm, int32_t max_iter,
                   const pr_options *opt, double *ranks_out, int32_t *iters_out, double *err_out,
                   int32_t *converged_out);

/*
 * pr_solve_noalloc — the same solve as pr_solve (DF64, uniform start), for
 * callers that cannot let the library allocate device memory. The paper has
 * no counterpart; this is a deployment variant.
 *
 * Who needs it: a process whose device memory belongs to its own pool or
 * caching allocator (a cudaMalloc behind its back can fail or fragment the
 * pool), a service held to a fixed device-memory budget, or a latency-bound
 * loop that cannot take the implicit device synchronisation of
 * cudaMalloc/cudaFree. This call makes no cudaMalloc, cudaFree or other
 * allocating call: the iterates, contributions, per-CTA partials and loop
 * state live in one file-scope device array of 40 MiB that every GPU loading
 * the library holds until the process exits.
 *
 * Arguments as pr_solve, except:
 *   d_ranks_out : device pointer, n doubles, caller order
 *   stream      : cudaStream_t or NULL; the call returns after the stream
 *                 has finished the solve
 * Limits and behaviour:
 *   - the working set is about 32 bytes per vertex plus small tables; a graph
 *     that does not fit (about n > 1.2 million) is rejected with PR_EINVAL
 *     and a message stating the bytes needed;
 *   - the graph must live on the current device, and d_ranks_out must be
 *     device memory of that device (checked with cudaPointerGetAttributes;
 *     PR_EINVAL otherwise);
 *   - the first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and keeps it for the
 *     life of the process;
 *   - the call reads the device's stop flag back after every pass and
 *     synchronises the stream each time, so it must not be called on a stream
 *     that is being captured into a CUDA graph;
 *   - every call shares the one array and overwrites what the previous call
 *     left there: calls that overlap on the GPU (other streams, other host
 *     threads) race and corrupt each other; serialise them.
 */
pr_status pr_solve_noalloc(const pr_graph *g, double alpha, double tol, int32_t norm, int32_t max_iter,
                           double *d_ranks_out, void *stream, int32_t *iters_out, double *err_out,
                           int32_t *converged_out);

/* One instance of a batch. Inputs: g .. init_vec. Outputs: iters .. status. */
typedef struct pr_instance {
    const pr_graph *g;
    double alpha;
    double tol;
    int32_t norm;
    int32_t max_iter;
    double *ranks_out;          /* n doubles (host, or device if outputs_on_device) */
    const double *init_vec;     /* PR_INIT_USER: this instance's start (NULL: opt->init_vec) */
    int32_t iters;
    int32_t converged;
    double err;                 /* the chosen norm at the stopping iteration */
    double err_l1;              /* the L1 norm of the same step (error bound:
                                   ||r - r*||_1 <= alpha/(1-alpha) * err_l1) */
    int32_t status;             /* pr_status of this instance */
    int32_t reserved;
} pr_instance;

/*
 * Solve many (graph, alpha, tau, norm, max_iter) instances together: the
 * alpha sweep of Section 2, the norm comparison of Section 3 and the tau sweep
 * of Section 4 as one batched device loop. Instances on the same graph become
 * columns of an N x k vertex-major rank matrix so that one index read serves
 * k gathers; different graphs run side by side in the same launches. Every
 * column stops and is retired on its own. Returns the first failing
 * instance's status (others are still filled in).
 */
pr_status pr_solve_batch(pr_instance *inst, int32_t count, const pr_options *opt);

/*
 * Learned warm start (no counterpart in the paper). A 5-64-64-1 MLP with
 * GELU activations on per-vertex features
 *   [log(1+indeg), log(1+outdeg), mean and max of log(1+outdeg(u)) over
 *    in-neighbours u, alpha]
 * predicts log(N * r); the start is exp(prediction) renormalised to sum 1.
 * Weights are held in FP32 (master) and BF16 (inference/training operands).
 * Training differentiates the exact (erf) GELU; inference evaluates GELU by
 * its tanh approximation (Hendrycks and Gimpel) on the hardware tanh, within
 * 5e-4 of the exact form (below the BF16 rounding of the hidden layer).
 * params layout (host, 4609 floats): W1[64][5], b1[64], W2[64][64], b2[64],
 * W3[1][64], b3[1].
 */
pr_status pr_mlp_create(const float *params, pr_mlp **out);
pr_status pr_mlp_destroy(pr_mlp *m);
pr_status pr_mlp_get_params(const pr_mlp *m, float *params_out);

/* Features (n x 5 floats, caller order, device pointer) of graph g at alpha.
 * Returns after the features are written (the stream is synchronised). */
pr_status pr_features(const pr_graph *g, double alpha, float *d_feat_out, void *stream);

/* Warm-start vector (n doubles, caller order; device pointer) for (g, alpha).
 * Returns after the vector is written (the stream is synchronised). Errors:
 * PR_ESTATE for a stale handle, PR_EINVAL for a NULL output or alpha outside
 * [0, 1]. */
pr_status pr_mlp_warm_start(const pr_mlp *m, const pr_graph *g, double alpha, double *d_r0_out,
                            void *stream);

/*
 * Mean squared error of the network on one set, L = mean over vertices of
 * (y - log(N r*))^2, and its gradient with respect to every parameter (host
 * outputs: loss_out one float, grad_out 4609 floats in the params layout;
 * either may be NULL). d_target_r: device, n doubles r* in caller order.
 */
pr_status pr_mlp_loss_grad(const pr_mlp *m, const pr_graph *g, double alpha, const double *d_target_r,
                           float *loss_out, float *grad_out, void *stream);

/*
 * Train the MLP on the device with the library's own forward, backward and
 * Adam kernels: minimise mean((y - log(N r*))^2) over all vertices of the
 * given (graph, alpha, target) sets. targets[i] is a device pointer to n_i
 * doubles r* in caller order. Runs `epochs` full-batch steps per set,
 * round-robin, with learning rate lr. loss_out (host, may be NULL) receives
 * the last epoch's mean loss over the sets.
 */
pr_status pr_mlp_train(pr_mlp *m, const pr_graph *const *graphs, const double *alphas,
                       const double *const *targets, int32_t nsets, int32_t epochs, float lr,
                       float *loss_out, void *stream);

/*
 * The network's gain: the mean over its training sets of
 * ln(||1/N - r*||_1 / ||r0 - r*||_1), r0 its start and r* the set's target,
 * measured at the end of pr_mlp_train (epochs > 0); known_out (may be NULL)
 * is 1 once measured or set. pr_mlp_set_gain sets it for a network created
 * from saved parameters (finite; PR_INIT_AUTO uses the network only for a
 * positive gain). No counterpart in the paper.
 */
pr_status pr_mlp_gain(const pr_mlp *m, double *gain_out, int32_t *known_out);
pr_status pr_mlp_set_gain(pr_mlp *m, double gain);

/*
 * Autotuning of the column width (no counterpart in the paper, which solves
 * one instance at a time): times the iteration kernel on graph g for the
 * widths W = 1, 2, 4, ..., max_width (a power of two, 1..32) in `precision`
 * (PR_PREC_DF64, PR_PREC_FP64 or PR_PREC_FP32; PR_PREC_MIXED tunes FP32 and
 * DF64 and reports DF64), by solving W synthetic columns (alpha 0.85, uniform
 * start) for a few iterations with one launch per iteration on `stream`.
 *   us_out : NULL or 6 doubles: microseconds per launch for W = 1 .. 32;
 *            0 for widths not measured (above max_width, or skipped because
 *            the W-column workspace would exceed a quarter of the free device
 *            memory)
 * Results are cached per process and device by graph signature; widths
 * already measured are not timed again. Errors: PR_ESTATE for a bad handle,
 * PR_EINVAL for a bad precision or width, PR_ENOMEM / PR_ECUDA from the
 * timing solves.
 */
pr_status pr_graph_tune(pr_graph *g, int32_t precision, int32_t max_width, void *stream, double *us_out);

/*
 * The planner behind PR_GROUP_AUTO, on host data only (no device work):
 * given `count` columns of one graph with estimated iteration counts
 * iters[c] > 0 and launch times us_per_launch[k] for width 2^k (k = 0..5;
 * <= 0 marks a width as unavailable, and width 1 must be available), cuts
 * the columns, sorted by decreasing iters (ties by index), into contiguous
 * jobs of at most 32 minimising sum over jobs of max(iters) x us_per_launch at
 * the smallest available width holding the job. Writes job_of[c] (jobs
 * numbered 0.. in sorted order) and width_of[c] (the job's width); *cost_out
 * (may be NULL) receives the minimum. PR_EINVAL on a bad argument.
 */
pr_status pr_plan_columns(int32_t count, const double *iters, const double *us_per_launch, int32_t *job_of,
                          int32_t *width_of, double *cost_out);

/*
 * The same grouping when jobs of one width share each launch and with it the
 * launch's latency (latency_us, measured by pr_graph_tune with four
 * single-column jobs in one launch). Candidates: the pr_plan_columns
 * partition, the partition for the launch times less the latency, and one job
 * per column; kept: the cheapest under
 *     sum over widths used  latency_us x max(iters)
 *   + sum over jobs         max(iters in the job) x max(t(W) - latency_us, 0.05 t(W)).
 * cost_out (optional) receives that cost. Errors as pr_plan_columns, and
 * PR_EINVAL for a negative or non-finite latency. Host only.
 */
pr_status pr_plan_columns_shared(int32_t count, const double *iters, const double *us_per_launch, double latency_us,
                                 int32_t *job_of, int32_t *width_of, double *cost_out);

/*
 * Resident CTAs per SM of the iteration kernel for `precision` (PR_PREC_DF64,
 * PR_PREC_FP64 or PR_PREC_FP32) and column width `width` (1, 2, 4, .., 32) on
 * the current device, as the CUDA occupancy calculator reports it for the
 * kernel's 256 threads and shared memory (for width 1, whose passes run as a
 * gather kernel and an update kernel, the gather kernel's); solves size the
 * gather grids as this times the SM count. PR_EINVAL for a bad argument,
 * PR_ECUDA on failure.
 */
pr_status pr_kernel_occupancy(int32_t precision, int32_t width, int32_t *ctas_per_sm);

/*
 * Counters of the last solve on any thread (host pointers, each may be NULL):
 *   launches  : kernel launches of the solve loop (init passes included; a
 *               one-column pass is two kernels, a gather and an update)
 *   passes    : iteration passes executed on the device
 *   kernel_ms : PR_LOOP_HOST only: sum over iteration passes of the CUDA-event
 *               time between the events recorded just before and just after
 *               each pass's launches on the solve's stream; 0 for the device
 *               loops (PR_LOOP_GRAPH, PR_LOOP_PERSISTENT)
 *   total_ms  : CUDA-event time of the whole device loop (all phases)
 */
pr_status pr_last_solve_stats(int32_t *launches, int32_t *passes, double *kernel_ms, double *total_ms);

/*
 * The last solve's kernel_ms (PR_LOOP_HOST) split by kernel for one-column
 * passes, which run as a gather kernel (row sums) and an update kernel (new
 * ranks, norms, stopping rules): the CUDA-event time from the start of each
 * pass to the end of its gather kernel, and from there to the end of the
 * pass, summed over passes. Both 0 when the passes were single kernels or the
 * loop was PR_LOOP_GRAPH. Host pointers, each may be NULL.
 */
pr_status pr_last_solve_kernel_ms(double *gather_ms, double *update_ms);

/*
 * The workspace pool of the current device (no counterpart in the paper):
 * bytes it has reserved from the device, bytes lent out to calls in flight
 * now, and the most ever lent out at once (host pointers, each may be NULL).
 * All zero before the first call that used the pool on this device.
 */
pr_status pr_workspace_info(int64_t *reserved_bytes, int64_t *used_bytes, int64_t *used_high_bytes);

/*
 * Return the pool's reserved but unused memory on the current device to the
 * device (after synchronising the device); later calls reserve again as
 * needed. PR_ECUDA on failure.
 */
pr_status pr_workspace_release(void);

/*
 * Columns (iterate sequences) of the last pr_solve / pr_solve_batch and, of
 * those, the ones solved in mixed precision (FP32 then DF64; with
 * PR_PREC_AUTO, what the planner chose) and the ones started from the learned
 * start (with PR_INIT_AUTO, what the cost model chose). Host pointers, each
 * may be NULL.
 */
pr_status pr_last_solve_columns(int32_t *columns, int32_t *mixed_columns, int32_t *learned_columns);

/*
 * How the last solve on any thread looped: the number of its phases (one per
 * precision phase and sub-solve) that ran as a CUDA graph while-loop, as a
 * host loop and as persistent passes (pr_loop). Host pointers, each may be
 * NULL.
 */
pr_status pr_last_solve_loops(int32_t *graph_phases, int32_t *host_phases, int32_t *persistent_phases);

/*
 * Test hook for the bounded waits of persistent passes: while `on` is nonzero,
 * the CTAs of solves that run persistent passes never announce the end of
 * their pass, so every CTA's wait for its job's other CTAs runs out after
 * persist_wait_us and the solve returns PR_ETIMEOUT (no GPU fault is
 * involved; the context stays usable). Process-wide; always PR_OK.
 */
pr_status pr_test_hold_decisions(int32_t on);

/* Message for the last error on this thread ("" if none). */
const char *pr_last_error(void);

/* Static name of a status code. */
const char *pr_status_string(pr_status s);

/* ABI version: major * 10000 + minor * 100 + patch. */
int32_t pr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PAGERANK_H */
