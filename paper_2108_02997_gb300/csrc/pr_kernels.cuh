// pr_kernels.cuh — the PageRank iteration kernels and the init pass.
//
// One pass updates every active column of every job once (Section 2) and
// decides, on the device, which columns stop (Sections 3-4). A pass is either
// two kernels, the gather kernel (pr_iter_kernel in its gather form: row sums
// only) followed by the streaming update kernel (pr_update_kernel), or, for
// small solves, one fused pr_iter_kernel that does both.
//
// Gather work is cut into warp tiles; every warp runs its tiles independently
// (no block-wide barrier until the end of the pass):
//   rows tile, one column (a run of rows of one in-degree class, at most 224
//   in-edges): coalesced loads of the tile's in-edge indices and of its row
//   offsets (kept in registers, read by shuffles), seven independent gathers
//   contrib[u] = r[u]/d_u per lane into a per-warp shared buffer, then lane
//   groups add each row's values in a fixed order;
//   rows tile, W columns: the same with one 8- or 16-byte vector gather per
//   in-edge and column group;
//   chunk tile (part of a long row): the warp strides over the chunk with the
//   next step's indices in flight; the last chunk of a row to finish adds the
//   chunk sums in chunk order.
// The update of a row (fused kernel, or update kernel from the row sums):
//     r'[v]  = c0 + alpha * sum                                    (SpMV)
//     accumulate |r'-r|, (r'-r)^2, max|r'-r|                         (norms)
//     contrib'[v] = r'[v]/d_v, or add r'[v] to the dangling sum when d_v = 0
//
// At the end of the pass the last CTA of a job reduces the CTA partials in a
// fixed order (FP64), forms L1, L2 = sqrt(sum of squares) and Linf, applies
// every pending stopping rule of each column, and computes
// c0 = (1-alpha)/N + alpha*D/N for the next update; the last job decides
// whether another pass is needed and, inside a CUDA graph, ends the graph's
// while-loop through its conditional handle.
#pragma once
#include "df64.cuh"
#include "pr_internal.cuh"

enum PassMode { kPassInit = 0, kPassIterate = 1 };
// Iteration kernel forms: the whole pass in one kernel, the gather half of a
// split pass that only writes row sums, or the whole pass repeated inside one
// cooperative launch until the stopping decision (persistent passes).
enum KernelMode { kModeFused = 0, kModeGather = 1, kModePersist = 2 };

// ---------------------------------------------------------------- small helpers
template <typename V>
__device__ __forceinline__ V load_raw(const double *p) {
    V v;
    memcpy(&v, p, sizeof(V));
    return v;
}
template <typename V>
__device__ __forceinline__ void store_raw(double *p, V v) {
    memcpy(p, &v, sizeof(V));
}
__device__ __forceinline__ double ld_cg(const double *p) { return __ldcg(p); }
template <typename V> __device__ __forceinline__ V ld_cg_v(const V *p);
template <> __device__ __forceinline__ double ld_cg_v<double>(const double *p) { return __ldcg(p); }
template <> __device__ __forceinline__ float ld_cg_v<float>(const float *p) { return __ldcg(p); }
template <> __device__ __forceinline__ df64 ld_cg_v<df64>(const df64 *p) {
    float2 f = __ldcg(reinterpret_cast<const float2 *>(p));
    return {f.x, f.y};
}

// Arrival counters of persistent passes (gpu-scope acquire loads).
__device__ __forceinline__ void red_release_gpu_add(uint32_t *p, uint32_t v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_gpu_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// An in-edge index of the one-column kernels (read once per pass: with
// kStreamIndex, marked evict-first so that it does not displace contributions
// from L1).
__device__ __forceinline__ int32_t ld_idx(const int32_t *p) {
    if constexpr (kStreamIndex) return __ldcs(p);
    else return *p;
}

// A work tile's descriptor: two 16-byte loads.
__device__ __forceinline__ Tile load_tile(const Tile *p) {
    const int4 a = __ldg(reinterpret_cast<const int4 *>(p));
    const int4 b = __ldg(reinterpret_cast<const int4 *>(p) + 1);
    return Tile{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
}

// CP adjacent column values of one vertex, read with one vector load.
template <typename V, int CP>
struct alignas(sizeof(V) * CP) VecV {
    V v[CP];
};
template <typename V, int CP>
__device__ __forceinline__ VecV<V, CP> load_vec(const V *p) {
    static_assert(sizeof(VecV<V, CP>) == 16 || sizeof(VecV<V, CP>) == 8, "vector loads are 8 or 16 bytes");
    VecV<V, CP> r;
    if constexpr (sizeof(VecV<V, CP>) == 16) {
        const float4 f = *reinterpret_cast<const float4 *>(p);
        memcpy(&r, &f, 16);
    } else {
        const float2 f = *reinterpret_cast<const float2 *>(p);
        memcpy(&r, &f, 8);
    }
    return r;
}

template <typename V>
struct RowAcc {
    using N = Num<V>;
    typename N::Acc l1, l2, linf, dsum, rsum;
    __device__ void init() {
        l1 = N::acc_zero(); l2 = N::acc_zero(); linf = N::acc_zero();
        dsum = N::acc_zero(); rsum = N::acc_zero();
    }
};

// Per-thread view of the column the thread serves (threads serve column tid % W).
template <typename V>
struct ColView {
    bool has;         // column exists in this job
    bool active;      // column updates this pass
    V alpha, c0;
    const V *r_prev;  // the column's current iterate (its own buffer parity)
    V *r_new;
    const V *c_prev;
    V *c_new;
    double *copy_dst;
};

// cs: the column's state (null when the thread's column is past the job's)
template <typename V>
__device__ __forceinline__ ColView<V> col_view_cs(const JobDev &job, const ColState *csp) {
    ColView<V> cv;
    cv.has = csp != nullptr;
    cv.active = false;
    cv.copy_dst = nullptr;
    cv.r_prev = cv.c_prev = nullptr;
    cv.r_new = cv.c_new = nullptr;
    if (cv.has) {
        const ColState &cs = *csp;
        const int cur = cs.cur;
        cv.active = cs.active;
        cv.alpha = load_raw<V>(cs.v_alpha);
        cv.c0 = load_raw<V>(cs.v_c0);
        cv.r_prev = reinterpret_cast<const V *>(job.r[cur]);
        cv.r_new = reinterpret_cast<V *>(job.r[cur ^ 1]);
        cv.c_prev = reinterpret_cast<const V *>(job.contrib[cur]);
        cv.c_new = reinterpret_cast<V *>(job.contrib[cur ^ 1]);
        cv.copy_dst = cs.copy_dst;
    }
    return cv;
}
template <typename V>
__device__ __forceinline__ ColView<V> col_view(const JobDev &job, int col) {
    return col_view_cs<V>(job, col < job.ncols ? &job.cols[col] : nullptr);
}

// New rank of row v in the thread's column: norms, contribution or dangling
// sum; and the copy of the column's current iterate into a stopping rule's
// output when one fired in the previous pass.
template <typename V, int W>
__device__ __forceinline__ void row_update_pd(const int32_t *__restrict__ perm, const ColView<V> &cv, RowAcc<V> &acc,
                                              int32_t v, int col, V s, V prev, int32_t d) {
    using N = Num<V>;
    const size_t idx = (size_t)v * W + col;
    if (cv.active) {
        V rn = N::axpy(cv.alpha, s, cv.c0);
        V dlt = N::sub(rn, prev);
        auto ad = N::acc_abs(dlt);
        acc.l1 = N::acc_add(acc.l1, ad);
        acc.l2 = N::acc_add(acc.l2, N::acc_sqr(ad));
        acc.linf = N::acc_max(acc.linf, ad);
        if (d == 0) acc.dsum = N::acc_add(acc.dsum, N::acc_of(rn));
        else cv.c_new[idx] = N::div_int(rn, d);
        acc.rsum = N::acc_add(acc.rsum, N::acc_of(rn));
        cv.r_new[idx] = rn;
    }
    if (cv.copy_dst) cv.copy_dst[perm[v]] = N::to_double(prev);
}

template <typename V, int W>
__device__ __forceinline__ void row_update(const int32_t *__restrict__ outdeg, const int32_t *__restrict__ perm,
                                           const ColView<V> &cv, RowAcc<V> &acc, int32_t v, int col, V s) {
    using N = Num<V>;
    const size_t idx = (size_t)v * W + col;
    if (!cv.active && !cv.copy_dst) return;
    const V prev = cv.r_prev[idx];
    if (cv.active) {
        V rn = N::axpy(cv.alpha, s, cv.c0);
        V dlt = N::sub(rn, prev);
        auto ad = N::acc_abs(dlt);
        acc.l1 = N::acc_add(acc.l1, ad);
        acc.l2 = N::acc_add(acc.l2, N::acc_sqr(ad));
        acc.linf = N::acc_max(acc.linf, ad);
        const int32_t d = outdeg[v];
        if (d == 0) acc.dsum = N::acc_add(acc.dsum, N::acc_of(rn));
        else cv.c_new[idx] = N::div_int(rn, d);
        acc.rsum = N::acc_add(acc.rsum, N::acc_of(rn));
        cv.r_new[idx] = rn;
    }
    if (cv.copy_dst) cv.copy_dst[perm[v]] = N::to_double(prev);
}

// ---------------------------------------------------------------- pass bookkeeping
// CTA partials of the thread accumulators, then the job finalizer (last CTA of
// the job) and the global decision (last job). Shared by both kernels.
// The CTA's partials of the thread accumulators (L1, sum of squares, Linf,
// dangling sum, sum of ranks per column, in a fixed order over warps) written
// to dst[c * kPartials + k]; with kFence the writers fence them for the CTA
// that reads them (otherwise the caller releases all the CTA's stores at once).
template <typename V, int W, bool kFence = true>
__device__ __forceinline__ void cta_partials(RowAcc<V> &acc, double *dst) {
    using N = Num<V>;
    using Acc = typename N::Acc;
    const int tid = threadIdx.x;
    const int col = tid % W;
    __shared__ Acc s_red[kWarps][W][kPartials];
    Acc a[kPartials] = {acc.l1, acc.l2, acc.linf, acc.dsum, acc.rsum};
    for (int m = W; m < 32; m <<= 1) {
#pragma unroll
        for (int k = 0; k < kPartials; k++) {
            Acc o = N::acc_shfl_xor(a[k], m);
            a[k] = (k == 2) ? N::acc_max(a[k], o) : N::acc_add(a[k], o);
        }
    }
    if ((tid & 31) < W) {
#pragma unroll
        for (int k = 0; k < kPartials; k++) s_red[tid >> 5][col][k] = a[k];
    }
    __syncthreads();
    if (tid < W * kPartials) {
        const int c = tid / kPartials, k = tid % kPartials;
        Acc t = s_red[0][c][k];
        for (int w = 1; w < kWarps; w++) t = (k == 2) ? N::acc_max(t, s_red[w][c][k]) : N::acc_add(t, s_red[w][c][k]);
        dst[c * kPartials + k] = N::acc_to_double(t);
        if constexpr (kFence) __threadfence();
    }
    __syncthreads();
}

// Fixed-order FP64 reduction of a job's CTA partials (cta_count x W x
// kPartials) into s_fin: partial p by warp p mod kWarps, lane l adding CTAs
// l, l + 32, ... (four loads in flight), then a fixed butterfly over the
// lanes; short dependent chains, since every FP64 operation on this GPU has a
// long latency. Every caller gets the same bits from the same partials.
template <int W>
__device__ __forceinline__ void reduce_partials(const double *cta_part, int cta_count, double *s_fin) {
    constexpr int P = W * kPartials;
    const int tid = threadIdx.x;
    const int rl = tid & 31, rw = tid >> 5;
    for (int p = rw; p < P; p += kWarps) {
        const bool is_max = (p % kPartials) == 2;
        double t = 0.0;
        for (int c = rl; c < cta_count; c += 4 * 32) {
            double x[4];
#pragma unroll
            for (int u = 0; u < 4; u++)
                x[u] = c + 32 * u < cta_count ? ld_cg(cta_part + (size_t)(c + 32 * u) * P + p) : 0.0;
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (c + 32 * u < cta_count) t = is_max ? fmax(t, x[u]) : t + x[u];
        }
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) {
            const double o = __shfl_xor_sync(0xffffffffu, t, m);
            t = is_max ? fmax(t, o) : t + o;
        }
        if (rl == 0) s_fin[p] = t;
    }
    __syncthreads();
}

template <typename V, int W>
__device__ __noinline__ void finish_pass(JobDev *jobs, JobDev &job, GlobalDev *glob, RowAcc<V> &acc, int local, int mode) {
    using N = Num<V>;
    const int tid = threadIdx.x;
    __shared__ int s_flag;
    __shared__ double s_fin[W * kPartials];
    // only the partials are read by another CTA of this launch (the job's
    // last); the other stores need not drain before arriving
    cta_partials<V, W>(acc, job.cta_part + (size_t)local * W * kPartials);
    if (tid == 0) {
        unsigned int old = atomicAdd(&job.arrive, 1u);
        s_flag = (old == (unsigned int)(job.cta_count - 1));
    }
    __syncthreads();
    if (!s_flag) return;
    __threadfence();
    // ---- last CTA of the job. Its work is a chain of dependent memory round
    // trips, which sets the latency of every pass: the job's fields, the
    // column states and the stopping rules are read once, with independent
    // loads, into registers and shared memory, changed there, and written back.
    const int ncols = job.ncols, cta_count = job.cta_count, job_cur = job.cur;
    // the pass bookkeeping the last job needs, requested now (only the last
    // job of a pass changes it)
    int g_njobs = 0, g_pass = 0, g_cap = 0;
    if (tid == 0) {
        g_njobs = glob->njobs;
        g_pass = glob->pass;
        g_cap = glob->pass_cap;
    }
    const int32_t n_rows = job.n;
    ColState *const cols = job.cols;
    Tap *const taps = job.taps;
    const double *const cta_part = job.cta_part;
    reduce_partials<W>(cta_part, cta_count, s_fin);
    // ---- column decisions: one warp per column, its lanes over the column's
    // stopping rules (taps, in order); the column state is staged in shared memory
    static_assert(sizeof(ColState) % 8 == 0, "ColState is copied in 8-byte words");
    constexpr int kCsWords = (int)(sizeof(ColState) / 8);
    __shared__ int s_colalive[W];
    __shared__ __align__(16) ColState s_cs[kWarps];
    const int lane = tid & 31, warp = tid >> 5;
    for (int c = warp; c < ncols; c += kWarps) {
        {
            const unsigned long long *src = reinterpret_cast<const unsigned long long *>(cols + c);
            unsigned long long *dst = reinterpret_cast<unsigned long long *>(&s_cs[warp]);
            for (int i = lane; i < kCsWords; i += 32) dst[i] = src[i];
        }
        __syncwarp();
        ColState &cs = s_cs[warp];
        const double l1 = s_fin[c * kPartials + 0];
        const double l2 = sqrt(s_fin[c * kPartials + 1]);
        const double li = s_fin[c * kPartials + 2];
        const double D = s_fin[c * kPartials + 3];
        const double S = s_fin[c * kPartials + 4];
        int col_alive = 0;
        if (mode == kPassInit) {
            col_alive = cs.active;
            __syncwarp();
            if (lane == 0) {
                cs.c0 = fma(cs.c0_coef, D, cs.c0_base);
                store_raw<V>(cs.v_c0, N::from_double(cs.c0));
                cs.last_sum = S;
                cs.copy_dst = nullptr;
            }
        } else if (cs.active) {
            const int it = cs.iters + 1;
            const double errs[3] = {l1, l2, li};
            const int tb = cs.tap_begin, te = cs.tap_end;
            int primary = -1;
            double *copy = nullptr;
            bool pending = false;
            for (int q0 = tb; q0 < te; q0 += 32) {
                const int q = q0 + lane;
                bool fires = false, pend = false;
                double e = 0.0;
                double *out = nullptr;
                if (q < te) {
                    const Tap tp = taps[q];
                    out = tp.out;
                    if (!tp.fired) {
                        e = errs[tp.norm - 1];
                        if (e < tp.tau || it >= tp.max_iter) fires = true;
                        else pend = true;
                    }
                    if (fires) {
                        // the rule's result fields (the rest of the tap is unchanged)
                        taps[q].fired = 1;
                        taps[q].iters = it;
                        taps[q].err = e;
                        taps[q].err_l1 = l1;
                        taps[q].converged = e < tp.tau;
                    }
                }
                const unsigned int fm = __ballot_sync(0xffffffffu, fires);
                if (__any_sync(0xffffffffu, pend)) pending = true;
                if (fm) {
                    const int first = __ffs(fm) - 1;
                    double *first_out = reinterpret_cast<double *>(
                        __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(out), first));
                    if (primary < 0) {
                        primary = q0 + first;
                        copy = first_out;
                    }
                    if (fires) taps[q].alias_of = q == primary ? -1 : primary;
                }
            }
            bool active = pending;
            if (cs.switch_norm && !cs.switched && errs[cs.switch_norm - 1] <= cs.switch_tol) active = false;
            col_alive = active || copy != nullptr;
            __syncwarp();
            if (lane == 0) {
                cs.iters = it;
                cs.cur ^= 1;
                cs.last_err[0] = l1; cs.last_err[1] = l2; cs.last_err[2] = li;
                cs.last_sum = S;
                if (cs.hist && it <= cs.hist_cap) {
                    cs.hist[3 * (it - 1) + 0] = l1;
                    cs.hist[3 * (it - 1) + 1] = l2;
                    cs.hist[3 * (it - 1) + 2] = li;
                }
                cs.copy_dst = copy;
                if (cs.switch_norm && !cs.switched && errs[cs.switch_norm - 1] <= cs.switch_tol)
                    cs.switched = 1;   // hand over to the refinement phase
                cs.active = active ? 1 : 0;
                cs.c0 = fma(cs.c0_coef, D, cs.c0_base);
                store_raw<V>(cs.v_c0, N::from_double(cs.c0));
            }
        } else {
            __syncwarp();
            if (lane == 0) cs.copy_dst = nullptr;
        }
        if (lane == 0) s_colalive[c] = col_alive;
        __syncwarp();
        {
            const unsigned long long *src = reinterpret_cast<const unsigned long long *>(&s_cs[warp]);
            unsigned long long *dst = reinterpret_cast<unsigned long long *>(cols + c);
            for (int i = lane; i < kCsWords; i += 32) dst[i] = src[i];
        }
        __syncwarp();
    }
    __syncthreads();
    if (tid == 0) {
        int alive = 0;
        for (int c = 0; c < ncols; c++) alive |= s_colalive[c];
        job.alive = alive;
        if (mode == kPassIterate) job.cur = job_cur ^ 1;   // parity shared by the columns still active
        job.arrive = 0;
        __threadfence();
        // one atomic: this job's arrival (high word) and whether it is alive (low word)
        const unsigned long long old =
            atomicAdd(&glob->arrive_alive, (1ull << 32) | (unsigned long long)(alive ? 1u : 0u));
        if ((unsigned int)(old >> 32) == (unsigned int)(g_njobs - 1)) {
            __threadfence();
            int any = (unsigned int)(old & 0xffffffffull) + (alive ? 1u : 0u) > 0u;
            glob->arrive_alive = 0ull;
            if (mode == kPassIterate) {
                if (*(volatile int32_t *)&glob->error) any = 0;
                if (any && g_pass + 1 >= g_cap) {
                    glob->error = kErrPassCap;
                    any = 0;
                }
                glob->alive = any;
                glob->pass = g_pass + 1;
                if (!any && glob->cond) cudaGraphSetConditional((cudaGraphConditionalHandle)glob->cond, 0u);
            } else {
                glob->alive = any;
            }
        }
    }
}

// ---------------------------------------------------------------- init pass
// r^0 (uniform, a caller vector, or an FP32 iterate being promoted), its
// contributions r/d and the dangling sum that gives c0 for the first update.
// Writes buffer cur of every column (all columns of a job start at cur = 0).
template <typename V, int W>
__global__ void __launch_bounds__(kBlock) pr_init_kernel(JobDev *jobs, GlobalDev *glob, const int32_t *cta_job) {
    using N = Num<V>;
    const int tid = threadIdx.x;
    const int col = tid % W;
    JobDev &job = jobs[cta_job[blockIdx.x]];
    const int local = blockIdx.x - job.cta_begin;
    RowAcc<V> acc;
    acc.init();
    if (col < job.ncols) {
        const ColState &cs = job.cols[col];
        V *r = reinterpret_cast<V *>(job.r[cs.cur]);
        V *c = reinterpret_cast<V *>(job.contrib[cs.cur]);
        const V uni = load_raw<V>(cs.v_c0);
        const long long total = (long long)job.n * W;
        for (long long i = (long long)local * kBlock + tid; i < total; i += (long long)job.cta_count * kBlock) {
            const int32_t v = (int32_t)(i / W);
            V x;
            if (cs.init_src == nullptr) {
                x = uni;
            } else if (cs.init_float) {
                const float *f = reinterpret_cast<const float *>(cs.init_src);
                x = N::from_double((double)f[(size_t)v * cs.init_col_stride + cs.init_col]);
            } else {
                const int32_t s = cs.init_order == 0 ? job.perm[v] : v;
                x = N::from_double(cs.init_src[(size_t)s * cs.init_col_stride + cs.init_col]);
            }
            r[i] = x;
            const int32_t d = job.outdeg[v];
            if (d == 0) acc.dsum = N::acc_add(acc.dsum, N::acc_of(x));
            else c[i] = N::div_int(x, d);
            acc.rsum = N::acc_add(acc.rsum, N::acc_of(x));
        }
    }
    finish_pass<V, W>(jobs, job, glob, acc, local, kPassInit);
}

// ---------------------------------------------------------------- persistent passes
// Every iteration pass of a job in one cooperative launch. Each CTA keeps a
// copy of the job's column states and stopping rules in shared memory and, at
// the end of a pass, takes the job's decisions itself: it publishes its
// partials, arrives on the job's counter, waits until all the job's CTAs have
// arrived, reduces all partials in the same fixed order as the job finalizer
// of the other loops, and applies the same stopping rules to its copy. Every
// CTA of the job therefore computes the same bits, no CTA waits for another to
// decide, and jobs do not wait for one another. The job's first CTA (the
// writer) also stores what the host reads back: fired rules, histories, and
// the column states when the job ends.
constexpr int kPersistTaps = 256;   // stopping rules per job that persistent passes hold in shared memory

struct PersistTap {
    double tau;
    double *out;
    int32_t norm, max_iter;
};
template <int W>
struct PersistState {
    ColState cols[W];
    PersistTap taps[kPersistTaps];
    uint32_t fired[kPersistTaps / 32];
    int32_t alive, cur, go, pad;
};
struct NoPersistState {
    int32_t unused;
};
template <int W, bool P>
struct PersistSel {
    using type = NoPersistState;
};
template <int W>
struct PersistSel<W, true> {
    using type = PersistState<W>;
};

// The job's state into shared memory, once per launch (all threads).
template <int W>
__device__ __forceinline__ void persist_load(const JobDev &job, PersistState<W> &ps) {
    static_assert(sizeof(ColState) % 8 == 0, "ColState is copied in 8-byte words");
    constexpr int kCsWords = (int)(sizeof(ColState) / 8);
    const int tid = threadIdx.x;
    const int ncols = min(job.ncols, W);
    const unsigned long long *src = reinterpret_cast<const unsigned long long *>(job.cols);
    unsigned long long *dst = reinterpret_cast<unsigned long long *>(ps.cols);
    for (int i = tid; i < ncols * kCsWords; i += kBlock) dst[i] = src[i];
    __syncthreads();
    int ntaps = 0;
    for (int c = 0; c < ncols; c++) ntaps = max(ntaps, ps.cols[c].tap_end);
    ntaps = min(ntaps, kPersistTaps);   // the host admits jobs of at most kPersistTaps rules
    for (int q = tid; q < ntaps; q += kBlock) {
        const Tap &t = job.taps[q];
        ps.taps[q] = PersistTap{t.tau, t.out, t.norm, t.max_iter};
    }
    for (int w = tid; w < kPersistTaps / 32; w += kBlock) {
        uint32_t bits = 0;
        for (int b = 0; b < 32; b++)
            if (w * 32 + b < ntaps && job.taps[w * 32 + b].fired) bits |= 1u << b;
        ps.fired[w] = bits;
    }
    if (tid == 0) {
        ps.alive = job.alive;
        ps.cur = job.cur;
        ps.go = 1;
    }
    __syncthreads();
}

// End of persistent pass `pass` (counted from 0 in this launch); returns
// whether the job runs another pass. The wait for the job's arrivals is
// bounded: after wait_ns of the global timer the CTA records kErrWait and
// stops, and every CTA that sees an error stops too, so that a CTA that never
// arrives ends the launch with an error the host reports.
template <typename V, int W>
__device__ __noinline__ bool persist_pass(JobDev &job, GlobalDev *glob, RowAcc<V> &acc, int local, PersistState<W> &ps,
                                          int32_t pass, unsigned long long wait_ns) {
    using N = Num<V>;
    constexpr int P = W * kPartials;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cta_count = job.cta_count, ncols = min(job.ncols, W);
    const bool writer = local == 0;
    // partials double-buffered by pass parity: a CTA may publish pass p + 1's
    // while another still reads pass p's
    double *part = job.cta_part + (size_t)(pass & 1) * cta_count * P;
    cta_partials<V, W, false>(acc, part + (size_t)local * P);
    __shared__ int s_ok;
    if (tid == 0) {
        // a release at gpu scope after the CTA barrier: every store of this
        // pass (iterates, contributions, partials) is visible to the CTA that
        // sees the arrival
        if (!*(volatile int32_t *)&glob->hold) red_release_gpu_add(&job.arrive, 1u);
        const uint32_t target = (uint32_t)(pass + 1) * (uint32_t)cta_count;
        int ok = 0;
        const unsigned long long t0 = global_ns();
        for (unsigned int spin = 0;; spin++) {
            if (ld_acquire_gpu_u32(&job.arrive) >= target) {
                ok = 1;
                break;
            }
            if (*(volatile int32_t *)&glob->error) break;
            if ((spin & 15u) == 15u && global_ns() - t0 > wait_ns) {
                atomicCAS(&glob->error, kErrNone, kErrWait);
                break;
            }
            __nanosleep(32);
        }
        // the acquire load above orders this CTA's later reads (the barrier
        // below extends it to the other threads)
        s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return false;
    __shared__ double s_fin[P];
    reduce_partials<W>(part, cta_count, s_fin);
    // ---- column decisions, as in finish_pass: one warp per column, its lanes
    // over the column's stopping rules in order
    __shared__ int s_colalive[W];
    Tap *const taps = job.taps;
    for (int c = warp; c < ncols; c += kWarps) {
        ColState &cs = ps.cols[c];
        const double l1 = s_fin[c * kPartials + 0];
        const double l2 = sqrt(s_fin[c * kPartials + 1]);
        const double li = s_fin[c * kPartials + 2];
        const double D = s_fin[c * kPartials + 3];
        const double S = s_fin[c * kPartials + 4];
        int col_alive = 0;
        if (cs.active) {
            const int it = cs.iters + 1;
            const double errs[3] = {l1, l2, li};
            const int tb = cs.tap_begin, te = min(cs.tap_end, kPersistTaps);
            int primary = -1;
            double *copy = nullptr;
            bool pending = false;
            for (int q0 = tb; q0 < te; q0 += 32) {
                const int q = q0 + lane;
                bool fires = false, pend = false;
                double e = 0.0;
                double *out = nullptr;
                if (q < te) {
                    const PersistTap tp = ps.taps[q];
                    out = tp.out;
                    if (!((ps.fired[q >> 5] >> (q & 31)) & 1u)) {
                        e = errs[tp.norm - 1];
                        if (e < tp.tau || it >= tp.max_iter) fires = true;
                        else pend = true;
                    }
                    if (fires) {
                        atomicOr(&ps.fired[q >> 5], 1u << (q & 31));
                        if (writer) {
                            taps[q].fired = 1;
                            taps[q].iters = it;
                            taps[q].err = e;
                            taps[q].err_l1 = l1;
                            taps[q].converged = e < tp.tau;
                        }
                    }
                }
                const unsigned int fm = __ballot_sync(0xffffffffu, fires);
                if (__any_sync(0xffffffffu, pend)) pending = true;
                if (fm) {
                    const int first = __ffs(fm) - 1;
                    double *first_out = reinterpret_cast<double *>(
                        __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(out), first));
                    if (primary < 0) {
                        primary = q0 + first;
                        copy = first_out;
                    }
                    if (fires && writer) taps[q].alias_of = q == primary ? -1 : primary;
                }
            }
            bool active = pending;
            if (cs.switch_norm && !cs.switched && errs[cs.switch_norm - 1] <= cs.switch_tol) active = false;
            col_alive = active || copy != nullptr;
            __syncwarp();
            if (lane == 0) {
                cs.iters = it;
                cs.cur ^= 1;
                cs.last_err[0] = l1; cs.last_err[1] = l2; cs.last_err[2] = li;
                cs.last_sum = S;
                if (writer && cs.hist && it <= cs.hist_cap) {
                    cs.hist[3 * (it - 1) + 0] = l1;
                    cs.hist[3 * (it - 1) + 1] = l2;
                    cs.hist[3 * (it - 1) + 2] = li;
                }
                cs.copy_dst = copy;
                if (cs.switch_norm && !cs.switched && errs[cs.switch_norm - 1] <= cs.switch_tol)
                    cs.switched = 1;   // hand over to the refinement phase
                cs.active = active ? 1 : 0;
                cs.c0 = fma(cs.c0_coef, D, cs.c0_base);
                store_raw<V>(cs.v_c0, N::from_double(cs.c0));
            }
        } else {
            __syncwarp();
            if (lane == 0) cs.copy_dst = nullptr;
        }
        if (lane == 0) s_colalive[c] = col_alive;
        __syncwarp();
    }
    __syncthreads();
    if (tid == 0) {
        int alive = 0;
        for (int c = 0; c < ncols; c++) alive |= s_colalive[c];
        ps.cur ^= 1;   // parity shared by the columns still active
        if (*(volatile int32_t *)&glob->error) alive = 0;
        if (alive && pass + 1 >= glob->pass_cap) {
            // the same pass budget as the other loops (every CTA of the job
            // stops here; the writer records why)
            if (writer) atomicCAS(&glob->error, kErrNone, kErrPassCap);
            alive = 0;
        }
        ps.alive = alive;
        ps.go = alive;
    }
    __syncthreads();
    if (ps.go) return true;
    if (writer) {
        // what the host reads back: the column states, the job's flags and
        // the passes run (the launch's pass count is the longest job's)
        constexpr int kCsWords = (int)(sizeof(ColState) / 8);
        const unsigned long long *src = reinterpret_cast<const unsigned long long *>(ps.cols);
        unsigned long long *dst = reinterpret_cast<unsigned long long *>(job.cols);
        for (int i = tid; i < ncols * kCsWords; i += kBlock) dst[i] = src[i];
        if (tid == 0) {
            job.alive = ps.alive;
            job.cur = ps.cur;
            atomicMax(&glob->pass, pass + 1);
        }
    }
    return false;
}

// ---------------------------------------------------------------- the iteration kernel
template <typename V, int W, int Mode = kModeFused>
__global__ void __launch_bounds__(kBlock, W == 1 ? (Mode == kModeGather ? kGatherMinBlocks : kMinBlocks)
                                                 : (Mode == kModeGather ? kVecGatherMinBlocks : vec_min_blocks((int)sizeof(V))))
    pr_iter_kernel(JobDev *jobs, GlobalDev *glob, const int32_t *cta_job) {
    using N = Num<V>;
    constexpr bool kGather = Mode == kModeGather;
    constexpr bool kPersist = Mode == kModePersist;
    static_assert(32 % W == 0, "W must divide the warp");
    constexpr bool kStaged = (W == 1);       // one column: values staged in shared memory
    constexpr int VT = kStaged ? kTileValues : 32;   // gathered values per warp step
    constexpr int TR = kStaged ? tile_rows(W) : 1;
    constexpr int PER = VT / 32;             // gathers in flight per lane (staged path)
    constexpr bool kTU = kTileUpdate && sizeof(V) == 8;   // all-lane row updates (8-byte values)
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int col = tid % W;                 // equals lane % W
    JobDev &job = jobs[cta_job[blockIdx.x]];
    // The job's fields are read once into registers: reads through `job` would
    // be repeated after every global store, which the compiler must assume
    // could alias the descriptor.
    const int local = blockIdx.x - (kGather ? job.gcta_begin : job.cta_begin);
    V *rowsum = reinterpret_cast<V *>(job.rowsum);
    const int32_t *__restrict__ src = job.src;
    const int32_t *__restrict__ off = job.off;
    const int32_t *__restrict__ outdeg = job.outdeg;
    const int32_t *__restrict__ perm = job.perm;
    const Tile *__restrict__ tiles = job.tiles;
    const int32_t *__restrict__ slot_base = job.slot_base;
    V *chunk_part = reinterpret_cast<V *>(job.chunk_part);
    uint32_t *chunk_cnt = job.chunk_cnt;
    const int ntiles = job.ntiles, cta_count = kGather ? job.gcta_count : job.cta_count;
    __shared__ V s_vals[kWarps][kStaged ? VT : 1];
    __shared__ V s_prev[kWarps][kStaged && !kGather ? TR * W : 1];
    constexpr int kOffRegs = kStaged ? TR / 32 + 1 : 1;   // one column: row offsets held in registers
    __shared__ int32_t s_od[kWarps][kStaged && !kGather ? TR : 1];
    __shared__ V s_sum[kWarps][kStaged && kTU && !kGather ? TR : 1];
    // several columns: per-warp buffers in dynamic shared memory
    constexpr int CP = vec_cols((int)sizeof(V), W);   // columns per vector load
    constexpr int NG = W / CP;                          // column groups (passes over a tile)
    constexpr int VTR = tile_rows(W);
    using VV = VecV<V, CP>;
    extern __shared__ __align__(16) unsigned char pr_dyn_smem[];
    unsigned char *wbase = pr_dyn_smem + (size_t)warp * vec_warp_bytes((int)sizeof(V), W, kGather);
    VV *v_vals = reinterpret_cast<VV *>(wbase);
    V *v_rsum = reinterpret_cast<V *>(wbase + vec_vals_bytes((int)sizeof(V), W));
    int32_t *v_src = reinterpret_cast<int32_t *>(wbase + vec_vals_bytes((int)sizeof(V), W) +
                                                 vec_rows_bytes((int)sizeof(V), W));
    int32_t *v_off = v_src + kVecTileEdges;
    V *v_prev = reinterpret_cast<V *>(v_off + round16((VTR + 1) * 4) / 4);   // not in the gather-only kernel
    int32_t *v_od = reinterpret_cast<int32_t *>(reinterpret_cast<unsigned char *>(v_prev) +
                                                vec_rows_bytes((int)sizeof(V), W));

    // Loop guard independent of the pass bookkeeping: should the job
    // finalizers ever fail to stop the graph's while-loop, the launch after the
    // cap ends it (no other thread sets the condition in that case).
    if (!kGather && blockIdx.x == 0 && tid == 0) {
        unsigned int nb = atomicAdd(&glob->body_count, 1u) + 1u;
        if (nb > (unsigned int)glob->pass_cap + 8u) {
            glob->error = kErrLoopGuard;
            if (glob->cond) cudaGraphSetConditional((cudaGraphConditionalHandle)glob->cond, 0u);
        }
    }
    // persistent passes: the pass below repeats in this launch until the
    // job's stopping decision (the CTA's tiles stay the same in every pass)
    __shared__ typename PersistSel<W, kPersist>::type ps;
    unsigned long long wait_ns = kPersistWaitNs;
    if constexpr (kPersist) {
        if (glob->wait_us) wait_ns = 1000ull * glob->wait_us;
        persist_load<W>(job, ps);
    }
    for (int32_t pass = 0;; pass++) {
        ColView<V> cv;
        if constexpr (kPersist) cv = col_view_cs<V>(job, col < job.ncols ? &ps.cols[col] : nullptr);
        else cv = col_view<V>(job, col);
        const bool need_prev = cv.has && (cv.active || cv.copy_dst);
        RowAcc<V> acc;
        acc.init();
        bool job_alive;
        int32_t job_cur;
        if constexpr (kPersist) {
            job_alive = ps.alive;
            job_cur = ps.cur;
        } else {
            job_alive = job.alive;
            job_cur = job.cur;
        }
        const bool work = job_alive && !*(volatile int32_t *)&glob->error;
        // several columns: the active columns read the job's shared buffer parity
        const unsigned int act_mask = __ballot_sync(0xffffffffu, cv.active);
        const V *c_all = reinterpret_cast<const V *>(job.contrib[job_cur]);
        auto gather1 = [&](int32_t u) -> V { return cv.c_prev[(size_t)u * W + col]; };

        if (work) {
            const int wstride = cta_count * kWarps;
            // ---------------- rows tile, several columns. Sources, offsets,
            // out-degrees and previous ranks are staged first; then per column
            // group: one vector gather per in-edge into shared memory, and lane
            // groups add each row's vectors; last, lane (row, column) pairs update rows.
            auto rows_tile_vec = [&](const Tile &T) {
                if constexpr (!kStaged) {
                    const int ne = T.e1 - T.e0, nr = T.r1 - T.r0;
#pragma unroll
                    for (int k = 0; k < kVecTileEdges / 32; k++) {
                        const int i = lane + 32 * k;
                        if (i < ne) v_src[i] = src[T.e0 + i];
                    }
                    for (int i = lane; i <= nr; i += 32) v_off[i] = off[T.r0 + i] - T.e0;
                    if constexpr (!kGather) {
                        for (int i = lane; i < nr; i += 32) v_od[i] = outdeg[T.r0 + i];
                        if (need_prev)
                            for (int i = lane; i < nr * W; i += 32) v_prev[i] = cv.r_prev[(size_t)T.r0 * W + i];
                    }
                    __syncwarp();
                    const int g = 1 << T.glog;
                    const int es = lane & (g - 1);
                    const int rpp = 32 >> T.glog;
#pragma unroll 1
                    for (int cg = 0; cg < NG; cg++) {
                        if (!((act_mask >> (cg * CP)) & ((1u << CP) - 1u))) continue;
#pragma unroll
                        for (int k0 = 0; k0 < kVecTileEdges / 32; k0 += kVecGatherBatch) {
                            VV x[kVecGatherBatch];
#pragma unroll
                            for (int k = 0; k < kVecGatherBatch; k++) {
                                const int i = lane + 32 * (k0 + k);
                                if (i < ne) x[k] = load_vec<V, CP>(c_all + (size_t)v_src[i] * W + cg * CP);
                            }
#pragma unroll
                            for (int k = 0; k < kVecGatherBatch; k++) {
                                const int i = lane + 32 * (k0 + k);
                                if (i < ne) v_vals[i] = x[k];
                            }
                        }
                        __syncwarp();
                        for (int rb = 0; rb < nr; rb += rpp) {
                            const int r = rb + (lane >> T.glog);
                            const bool valid = r < nr;
                            EdgeSum<V> sum[CP];
#pragma unroll
                            for (int j = 0; j < CP; j++) sum[j].init();
                            if (valid) {
                                const int lo = v_off[r], hi = v_off[r + 1];
                                for (int e = lo + es; e < hi; e += g) {
                                    const VV y = v_vals[e];
#pragma unroll
                                    for (int j = 0; j < CP; j++) sum[j].add(y.v[j]);
                                }
                            }
#pragma unroll
                            for (int j = 0; j < CP; j++) {
                                V sv = sum[j].get();
                                for (int m = 1; m < g; m <<= 1) sv = N::add_pos(sv, N::shfl_xor(sv, m));
                                if (valid && es == 0) v_rsum[r * W + cg * CP + j] = sv;
                            }
                        }
                        __syncwarp();
                    }
                    if constexpr (kGather) {
                        // element i of the rows belongs to column i % W == lane % W
                        if (cv.active)
                            for (int i = lane; i < nr * W; i += 32) rowsum[(size_t)T.r0 * W + i] = v_rsum[i];
                    } else {
                        if (need_prev)
                            for (int i = lane; i < nr * W; i += 32)
                                row_update_pd<V, W>(perm, cv, acc, T.r0 + i / W, col, v_rsum[i], v_prev[i], v_od[i / W]);
                    }
                    __syncwarp();
                }
            };
            // ---------------- rows tile, one column: indices, offsets, previous
            // ranks and out-degrees are all requested before any gather waits
            auto rows_tile_w1 = [&](const Tile &T) {
                if constexpr (kStaged) {
                    const int ne = T.e1 - T.e0, nr = T.r1 - T.r0;
                    int32_t u[PER];
#pragma unroll
                    for (int k = 0; k < PER; k++) {
                        const int idx = lane + 32 * k;
                        u[k] = (cv.active && idx < ne * W) ? ld_idx(src + T.e0 + idx / W) : -1;
                    }
                    // row offsets relative to e0 in registers: lane l holds rows l, l + 32, ...
                    int32_t o[kOffRegs];
#pragma unroll
                    for (int j = 0; j < kOffRegs; j++) {
                        const int i = lane + 32 * j;
                        o[j] = i <= nr ? off[T.r0 + i] - T.e0 : 0;
                    }
                    // element i of the rows belongs to column i % W == lane % W
                    if constexpr (!kGather) {
                        if (need_prev)
                            for (int i = lane; i < nr * W; i += 32) s_prev[warp][i] = cv.r_prev[(size_t)T.r0 * W + i];
                        for (int i = lane; i < nr; i += 32) s_od[warp][i] = outdeg[T.r0 + i];
                    }
                    {
                        V x[PER];
#pragma unroll
                        for (int k = 0; k < PER; k++) x[k] = u[k] >= 0 ? gather1(u[k]) : N::zero();
#pragma unroll
                        for (int k = 0; k < PER; k++)
                            if (u[k] >= 0) s_vals[warp][lane + 32 * k] = x[k];
                    }
                    __syncwarp();
                    const int g = 1 << T.glog;
                    const int es = (lane & (g - 1)) / W;
                    const int ES = g / W;
                    const int rpp = 32 >> T.glog;
                    for (int rb = 0; rb < nr; rb += rpp) {
                        const int r = rb + (lane >> T.glog);
                        const bool valid = r < nr;
                        // rows r and r + 1 lie in [rb, rb + 32]: registers j0 and j0 + 1 of their lanes
                        const int j0 = rb >> 5;
                        int32_t oa = o[0], ob = o[kOffRegs > 1 ? 1 : 0];
#pragma unroll
                        for (int j = 1; j + 1 < kOffRegs; j++) {
                            if (j0 == j) {
                                oa = o[j];
                                ob = o[j + 1];
                            }
                        }
                        const int32_t la = __shfl_sync(0xffffffffu, oa, r & 31), lb = __shfl_sync(0xffffffffu, ob, r & 31);
                        const int32_t ha = __shfl_sync(0xffffffffu, oa, (r + 1) & 31),
                                      hb = __shfl_sync(0xffffffffu, ob, (r + 1) & 31);
                        EdgeSum<V> sum;
                        sum.init();
                        if (valid && cv.active) {
                            const int lo = (r >> 5) == j0 ? la : lb, hi = ((r + 1) >> 5) == j0 ? ha : hb;
                            for (int e = lo + es; e < hi; e += ES) sum.add(s_vals[warp][e * W + col]);
                        }
                        V sv = sum.get();
                        for (int m = W; m < g; m <<= 1) sv = N::add_pos(sv, N::shfl_xor(sv, m));
                        if constexpr (kGather) {
                            if (valid && es == 0 && cv.active) rowsum[T.r0 + r] = sv;
                        } else if constexpr (kTU) {
                            if (valid && es == 0) s_sum[warp][r] = sv;
                        } else {
                            if (valid && es == 0 && need_prev)
                                row_update_pd<V, W>(perm, cv, acc, T.r0 + r, col, sv, s_prev[warp][r * W + col],
                                                    s_od[warp][r]);
                        }
                    }
                    __syncwarp();
                    if constexpr (kTU && !kGather) {
                        // every lane updates rows: consecutive rows on consecutive lanes
                        if (need_prev)
                            for (int r = lane; r < nr; r += 32)
                                row_update_pd<V, W>(perm, cv, acc, T.r0 + r, col, s_sum[warp][r], s_prev[warp][r],
                                                    s_od[warp][r]);
                        __syncwarp();
                    }
                }
            };
            // ---------------- one chunk of a long row
            auto chunk_tile = [&](const Tile &T) {
                // ---------------- one chunk of a long row, VT values per step
                const int32_t v = T.r0;
                const int nv = (T.e1 - T.e0) * W;
                EdgeSum<V> sum;
                sum.init();
                if constexpr (!kStaged) {
                    // several columns: per column group, lanes stride over the
                    // chunk's in-edges with vector loads, four in flight
                    const int ne = T.e1 - T.e0;
#pragma unroll 1
                    for (int cg = 0; cg < NG; cg++) {
                        if (!((act_mask >> (cg * CP)) & ((1u << CP) - 1u))) continue;
                        EdgeSum<V> vs[CP];
#pragma unroll
                        for (int j = 0; j < CP; j++) vs[j].init();
                        const V *cb = c_all + cg * CP;
                        int i = lane;
                        for (; i + 96 < ne; i += 128) {
                            const int32_t u0 = src[T.e0 + i], u1 = src[T.e0 + i + 32];
                            const int32_t u2 = src[T.e0 + i + 64], u3 = src[T.e0 + i + 96];
                            const VV x0 = load_vec<V, CP>(cb + (size_t)u0 * W), x1 = load_vec<V, CP>(cb + (size_t)u1 * W);
                            const VV x2 = load_vec<V, CP>(cb + (size_t)u2 * W), x3 = load_vec<V, CP>(cb + (size_t)u3 * W);
#pragma unroll
                            for (int j = 0; j < CP; j++) {
                                vs[j].add(x0.v[j]); vs[j].add(x1.v[j]); vs[j].add(x2.v[j]); vs[j].add(x3.v[j]);
                            }
                        }
                        for (; i < ne; i += 32) {
                            const VV x0 = load_vec<V, CP>(cb + (size_t)src[T.e0 + i] * W);
#pragma unroll
                            for (int j = 0; j < CP; j++) vs[j].add(x0.v[j]);
                        }
#pragma unroll
                        for (int j = 0; j < CP; j++) {
                            V sv = vs[j].get();
                            for (int m = 1; m < 32; m <<= 1) sv = N::add_pos(sv, N::shfl_xor(sv, m));
                            if (lane == 0) v_rsum[cg * CP + j] = sv;
                        }
                    }
                    __syncwarp();
                }
                if (kStaged && cv.active) {
                    // the next step's indices are requested while this step's
                    // gathers are in flight
                    int32_t u[PER];
#pragma unroll
                    for (int k = 0; k < PER; k++) {
                        const int idx = lane + 32 * k;
                        u[k] = idx < nv ? ld_idx(src + T.e0 + idx) : -1;
                    }
                    for (int base = lane; base < nv; base += VT) {
                        V x[PER];
#pragma unroll
                        for (int k = 0; k < PER; k++) x[k] = u[k] >= 0 ? gather1(u[k]) : N::zero();
                        int32_t un[PER];
#pragma unroll
                        for (int k = 0; k < PER; k++) {
                            const int idx = base + VT + 32 * k;
                            un[k] = idx < nv ? ld_idx(src + T.e0 + idx) : -1;
                        }
#pragma unroll
                        for (int k = 0; k < PER; k++)
                            if (u[k] >= 0) sum.add(x[k]);
#pragma unroll
                        for (int k = 0; k < PER; k++) u[k] = un[k];
                    }
                }
                V sv = sum.get();
                if constexpr (kStaged) {
                    for (int m = W; m < 32; m <<= 1) sv = N::add_pos(sv, N::shfl_xor(sv, m));
                } else {
                    if (lane < W) sv = v_rsum[lane];
                    __syncwarp();
                }
                if (T.slot < 0) {
                    if constexpr (kGather) {
                        if (lane < W && cv.active) rowsum[(size_t)v * W + lane] = sv;
                    } else {
                        if (lane < W && cv.has) row_update<V, W>(outdeg, perm, cv, acc, v, col, sv);
                    }
                } else {
                    const int32_t base = slot_base[T.slot];
                    if (lane < W) chunk_part[(size_t)(base + T.k) * W + lane] = sv;
                    __threadfence();
                    __syncwarp();
                    int last = 0;
                    if (lane == 0) last = atomicAdd(&chunk_cnt[T.slot], 1u) == (unsigned int)(T.nch - 1);
                    last = __shfl_sync(0xffffffffu, last, 0);
                    if (last) {
                        // the row's chunk sums, lane-parallel in a fixed order:
                        // lane slot q0 adds chunks q0, q0 + 32/W, ... then a fixed tree
                        __threadfence();
                        constexpr int QS = 32 / W;
                        V t = N::zero();
                        for (int32_t q = lane / W; q < T.nch; q += QS)
                            t = N::add_pos(t, ld_cg_v<V>(chunk_part + (size_t)(base + q) * W + col));
                        for (int m = W; m < 32; m <<= 1) t = N::add_pos(t, N::shfl_xor(t, m));
                        if constexpr (kGather) {
                            if (lane < W && cv.active) rowsum[(size_t)v * W + lane] = t;
                        } else {
                            if (lane < W && cv.has) row_update<V, W>(outdeg, perm, cv, acc, v, col, t);
                        }
                        if (lane == 0) chunk_cnt[T.slot] = 0;
                    }
                    __syncwarp();
                }
            };

            // the next tile's descriptor is requested while this tile is worked on
            Tile T_next{};
            if (local * kWarps + warp < ntiles) T_next = load_tile(tiles + local * kWarps + warp);
            for (int t = local * kWarps + warp; t < ntiles; t += wstride) {
                const Tile T = T_next;
                if (t + wstride < ntiles) T_next = load_tile(tiles + t + wstride);
                if (T.glog >= 0) {
                    if constexpr (kStaged) rows_tile_w1(T);
                    else rows_tile_vec(T);
                } else {
                    chunk_tile(T);
                }
            }
        }
        if constexpr (kPersist) {
            if (!persist_pass<V, W>(job, glob, acc, local, ps, pass, wait_ns)) break;
        } else {
            if constexpr (!kGather) finish_pass<V, W>(jobs, job, glob, acc, local, kPassIterate);
            break;
        }
    }
}

// ---------------------------------------------------------------- the update kernel (split passes)
// Second half of a split pass: streams the rows, turns each row sum into the
// new rank (r' = c0 + alpha * s), its contribution or dangling share and the
// norm terms, copies iterates into stopping-rule outputs, and ends the pass
// like the fused kernel (CTA partials, last-CTA decisions, c0 for the next pass).
template <typename V, int W>
__global__ void __launch_bounds__(kBlock, kUpdateMinBlocks) pr_update_kernel(JobDev *jobs, GlobalDev *glob, const int32_t *cta_job) {
    using N = Num<V>;
    const int tid = threadIdx.x;
    const int col = tid % W;
    JobDev &job = jobs[cta_job[blockIdx.x]];
    const int local = blockIdx.x - job.cta_begin;
    if (blockIdx.x == 0 && tid == 0) {
        unsigned int nb = atomicAdd(&glob->body_count, 1u) + 1u;
        if (nb > (unsigned int)glob->pass_cap + 8u) {
            glob->error = kErrLoopGuard;
            if (glob->cond) cudaGraphSetConditional((cudaGraphConditionalHandle)glob->cond, 0u);
        }
    }
    const ColView<V> cv = col_view<V>(job, col);
    RowAcc<V> acc;
    acc.init();
    const bool work = job.alive && !*(volatile int32_t *)&glob->error;
    if (work && cv.has && (cv.active || cv.copy_dst)) {
        const V *__restrict__ rowsum = reinterpret_cast<const V *>(job.rowsum);
        const int32_t *__restrict__ outdeg = job.outdeg;
        const int32_t *__restrict__ perm = job.perm;
        const V *__restrict__ r_prev = cv.r_prev;
        const long long total = (long long)job.n * W;
        const long long stride = (long long)job.cta_count * kBlock;
        long long i = (long long)local * kBlock + tid;
        if constexpr (W == 1) {
            // one column: pairs of consecutive rows, their row sums and previous
            // ranks read with one vector load each and their out-degrees with one
            // 8-byte load; kPairs pairs per step, all loads issued before any update
            using V2 = VecV<V, 2>;
            const long long npairs = total >> 1;
            const V2 *__restrict__ rs2 = reinterpret_cast<const V2 *>(rowsum);
            const V2 *__restrict__ rp2 = reinterpret_cast<const V2 *>(r_prev);
            const int2 *__restrict__ od2 = reinterpret_cast<const int2 *>(outdeg);
            constexpr int kPairs = PR_UPDATE_PAIRS;
            long long q = i;
            for (; q + (kPairs - 1) * stride < npairs; q += kPairs * stride) {
                V2 sv[kPairs], pv[kPairs];
                int2 dv[kPairs];
#pragma unroll
                for (int k = 0; k < kPairs; k++) {
                    const long long j = q + k * stride;
                    if (cv.active) sv[k] = load_vec<V, 2>(reinterpret_cast<const V *>(rs2 + j));
                    else sv[k].v[0] = sv[k].v[1] = N::zero();
                    pv[k] = load_vec<V, 2>(reinterpret_cast<const V *>(rp2 + j));
                    dv[k] = od2[j];
                }
#pragma unroll
                for (int k = 0; k < kPairs; k++) {
                    const int32_t v = (int32_t)(2 * (q + k * stride));
                    row_update_pd<V, 1>(perm, cv, acc, v, 0, sv[k].v[0], pv[k].v[0], dv[k].x);
                    row_update_pd<V, 1>(perm, cv, acc, v + 1, 0, sv[k].v[1], pv[k].v[1], dv[k].y);
                }
            }
            for (; q < npairs; q += stride) {
                row_update<V, 1>(outdeg, perm, cv, acc, (int32_t)(2 * q), 0, cv.active ? rowsum[2 * q] : N::zero());
                row_update<V, 1>(outdeg, perm, cv, acc, (int32_t)(2 * q + 1), 0,
                                 cv.active ? rowsum[2 * q + 1] : N::zero());
            }
            // an odd last row
            if ((total & 1) && local == 0 && tid == 0)
                row_update<V, 1>(outdeg, perm, cv, acc, (int32_t)(total - 1), 0,
                                 cv.active ? rowsum[total - 1] : N::zero());
            i = total;   // nothing left for the general loops below
        }
        // four rows per step, their loads issued before any update
        for (; i + 3 * stride < total; i += 4 * stride) {
            V sv[4], pv[4];
            int32_t dv[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const long long j = i + k * stride;
                sv[k] = cv.active ? rowsum[j] : N::zero();
                pv[k] = r_prev[j];
                dv[k] = outdeg[j / W];
            }
#pragma unroll
            for (int k = 0; k < 4; k++)
                row_update_pd<V, W>(perm, cv, acc, (int32_t)((i + k * stride) / W), col, sv[k], pv[k], dv[k]);
        }
        for (; i < total; i += stride) {
            const V sv = cv.active ? rowsum[i] : N::zero();
            row_update<V, W>(outdeg, perm, cv, acc, (int32_t)(i / W), col, sv);
        }
    }
    finish_pass<V, W>(jobs, job, glob, acc, local, kPassIterate);
}

// ---------------------------------------------------------------- the update kernel, bulk-copy form
// The one-column update of a split pass (pr_update_kernel<V, 1>'s work) with
// the rows' inputs (row sums, previous ranks, out-degrees) streamed into shared
// memory by 1-D bulk copies: each CTA takes tiles of kUpdRows consecutive rows
// (tile t = local, local + CTAs, ...), keeps kUpdStages tiles in flight behind
// one mbarrier each, and its threads update the rows of a tile from shared
// memory (thread t: rows t, t + 256, ...), so that the bytes in flight per SM do
// not depend on the threads' registers. A copy starts at a multiple of
// kUpdRows rows (16-byte aligned) and covers the tile's rows rounded up to four
// (the arrays are padded). Every wait is bounded: a wait that runs out records
// kErrWait, waits (bounded) for the CTA's copies still in flight and ends the
// CTA's row work.
constexpr unsigned int kUpdSpinLimit = 1u << 22;   // mbarrier polls before a wait is abandoned

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase) {
    for (unsigned int spin = 0; spin < kUpdSpinLimit; spin++)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}
__device__ __forceinline__ void bulk_to_shared(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

template <typename V>
__global__ void __launch_bounds__(kBlock, kUpdateMinBlocks) pr_update_bulk_kernel(JobDev *jobs, GlobalDev *glob,
                                                                                   const int32_t *cta_job) {
    using N = Num<V>;
    constexpr int kSB = upd_stage_bytes((int)sizeof(V));
    const int tid = threadIdx.x;
    JobDev &job = jobs[cta_job[blockIdx.x]];
    const int local = blockIdx.x - job.cta_begin;
    if (blockIdx.x == 0 && tid == 0) {
        unsigned int nb = atomicAdd(&glob->body_count, 1u) + 1u;
        if (nb > (unsigned int)glob->pass_cap + 8u) {
            glob->error = kErrLoopGuard;
            if (glob->cond) cudaGraphSetConditional((cudaGraphConditionalHandle)glob->cond, 0u);
        }
    }
    const ColView<V> cv = col_view<V>(job, 0);
    RowAcc<V> acc;
    acc.init();
    extern __shared__ __align__(128) unsigned char upd_smem[];
    __shared__ __align__(8) uint64_t s_bar[kUpdStages];
    const bool work = job.alive && !*(volatile int32_t *)&glob->error;
    if (work && cv.has && (cv.active || cv.copy_dst)) {
        const int32_t n = job.n;
        const int cta_count = job.cta_count;
        const int ntiles = (int)(((int64_t)n + kUpdRows - 1) / kUpdRows);
        const int my_tiles = local < ntiles ? (ntiles - 1 - local) / cta_count + 1 : 0;
        const V *rowsum = reinterpret_cast<const V *>(job.rowsum);
        const V *r_prev = cv.r_prev;
        const int32_t *outdeg = job.outdeg;
        const int32_t *__restrict__ perm = job.perm;
        if (tid == 0) {
            for (int st = 0; st < kUpdStages; st++) mbar_init(&s_bar[st], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        // thread 0: the k-th tile of this CTA into stage k mod kUpdStages
        auto issue = [&](int k) {
            const int32_t r0 = (local + k * cta_count) * kUpdRows;
            const int rows = min(kUpdRows, n - r0);
            const uint32_t rows4 = (uint32_t)((rows + 3) & ~3);
            unsigned char *stg = upd_smem + (size_t)(k % kUpdStages) * kSB;
            uint64_t *bar = &s_bar[k % kUpdStages];
            // the stage's previous contents were read by the threads (generic
            // proxy) before this copy (async proxy) overwrites them
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(bar, rows4 * (2u * (uint32_t)sizeof(V) + 4u));
            bulk_to_shared(stg, rowsum + r0, rows4 * (uint32_t)sizeof(V), bar);
            bulk_to_shared(stg + kUpdRows * sizeof(V), r_prev + r0, rows4 * (uint32_t)sizeof(V), bar);
            bulk_to_shared(stg + 2 * kUpdRows * sizeof(V), outdeg + r0, rows4 * 4u, bar);
        };
        if (tid == 0)
            for (int k = 0; k < min(kUpdStages, my_tiles); k++) issue(k);
        for (int k = 0; k < my_tiles; k++) {
            const int sidx = k % kUpdStages;
            const uint32_t phase = (uint32_t)(k / kUpdStages) & 1u;
            const bool ok = mbar_wait_bounded(&s_bar[sidx], phase);
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    atomicCAS(&glob->error, kErrNone, kErrWait);
                    // the copies issued and not yet consumed may still be in flight
                    for (int k2 = k; k2 < min(k + kUpdStages, my_tiles); k2++)
                        mbar_wait_bounded(&s_bar[k2 % kUpdStages], (uint32_t)(k2 / kUpdStages) & 1u);
                }
                __syncthreads();
                break;
            }
            const unsigned char *stg = upd_smem + (size_t)sidx * kSB;
            const V *s_rs = reinterpret_cast<const V *>(stg);
            const V *s_pv = reinterpret_cast<const V *>(stg + kUpdRows * sizeof(V));
            const int32_t *s_od = reinterpret_cast<const int32_t *>(stg + 2 * kUpdRows * sizeof(V));
            const int32_t r0 = (local + k * cta_count) * kUpdRows;
            const int rows = min(kUpdRows, n - r0);
            for (int i = tid; i < rows; i += kBlock) {
                const V sv = cv.active ? s_rs[i] : N::zero();
                row_update_pd<V, 1>(perm, cv, acc, r0 + i, 0, sv, s_pv[i], s_od[i]);
            }
            __syncthreads();   // every thread is done with this stage
            if (tid == 0 && k + kUpdStages < my_tiles) issue(k + kUpdStages);
        }
    }
    finish_pass<V, 1>(jobs, job, glob, acc, local, kPassIterate);
}

// ---------------------------------------------------------------- the hub gather kernel (split passes)
// The gather half of a pass (row sums only) for jobs of W columns whose W
// values of a vertex fill at most one 32-byte L2 sector (one, two or four
// columns; four df64/FP64 columns are read with two 16-byte loads; one column
// runs pr_gather_hub1_kernel below, the same code for a single value), with one CTA
// of kHubBlock threads per SM. The CTA first copies the contribution vectors
// of vertices [0, hub_n) into shared memory: after the relabelling these are
// the highest in-/out-degree classes, the sources most often gathered (R-MAT
// scale 22: the first 12,288 ids originate 37 % of the in-edges). A gather of
// a source below hub_n then reads shared memory, the others the global
// contribution array through L1/L2, whose random-sector rate bounds the
// kernel; a vector of W columns costs one sector like a single value, so the
// W columns share the index stream and the random reads.
template <typename V, int W>
__device__ __forceinline__ VecV<V, W> ld_gather_vec(const V *p) {
    static_assert(sizeof(VecV<V, W>) == 4 || sizeof(VecV<V, W>) == 8 || sizeof(VecV<V, W>) == 16 ||
                      sizeof(VecV<V, W>) == 32, "vector size");
    VecV<V, W> r;
    if constexpr (sizeof(VecV<V, W>) == 32) {
        if constexpr (kGatherV8) {
            // one 32-byte sector in one 256-bit load
            uint32_t w[8];
            asm("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
                : "l"(p));
            memcpy(&r, w, 32);
        } else {
            // one 32-byte sector: two 16-byte loads of the same sector
            const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
            const float4 b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
            memcpy(&r, &a, 16);
            memcpy(reinterpret_cast<unsigned char *>(&r) + 16, &b, 16);
        }
    } else if constexpr (sizeof(VecV<V, W>) == 16) {
        const float4 f = __ldg(reinterpret_cast<const float4 *>(p));
        memcpy(&r, &f, 16);
    } else if constexpr (sizeof(VecV<V, W>) == 8) {
        const float2 f = __ldg(reinterpret_cast<const float2 *>(p));
        memcpy(&r, &f, 8);
    } else {
        const float f = __ldg(reinterpret_cast<const float *>(p));
        memcpy(&r, &f, 4);
    }
    return r;
}

template <typename V, int W>
__global__ void __launch_bounds__(kHubBlock, 1) pr_gather_hub_kernel(JobDev *jobs, GlobalDev *glob, const int32_t *cta_job) {
    using N = Num<V>;
    using VV = VecV<V, W>;
    constexpr int TV = hub_tile_edges(W);   // staged vectors per warp (rows tiles)
    constexpr int PER = TV / 32;            // staged gathers per lane
    constexpr int TR = tile_rows(1);
    constexpr int kOffRegs = TR / 32 + 1;   // row offsets of a rows tile, in registers
    constexpr int CPER = kHubChunkPer / W;  // vector gathers per lane in flight (chunk tiles)
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    JobDev &job = jobs[cta_job[blockIdx.x]];
    // CTA-uniform: nothing to gather when the job or all its columns have stopped
    bool any_active = job.cols[0].active != 0;
    if constexpr (W > 1)
        for (int c = 1; c < job.ncols; c++) any_active |= job.cols[c].active != 0;
    if (!job.alive || !any_active || *(volatile int32_t *)&glob->error) return;
    const int local = blockIdx.x - job.gcta_begin;
    const int cta_count = job.gcta_count;
    // the contributions of the active columns, vertex-major (W values per vertex)
    const V *__restrict__ c_prev = reinterpret_cast<const V *>(job.contrib[W == 1 ? job.cols[0].cur : job.cur]);
    V *__restrict__ rowsum = reinterpret_cast<V *>(job.rowsum);
    const int32_t *__restrict__ src = job.src;
    const int32_t *__restrict__ off = job.off;
    const Tile *__restrict__ tiles = job.tiles;
    const int32_t *__restrict__ slot_base = job.slot_base;
    V *chunk_part = reinterpret_cast<V *>(job.chunk_part);
    uint32_t *chunk_cnt = job.chunk_cnt;
    const int ntiles = job.ntiles;
    // at most what the launch's shared memory holds for this vector type
    const int hub_n = min(job.hub_n, hub_bytes(W) / (int)sizeof(VV));
    extern __shared__ __align__(16) unsigned char pr_hub_smem[];
    VV *s_vals = reinterpret_cast<VV *>(pr_hub_smem) + warp * TV;   // this warp's staged vectors
    VV *s_hub = reinterpret_cast<VV *>(pr_hub_smem) + kHubWarps * TV;
    for (int i = tid; i < hub_n; i += kHubBlock) {
        VV x;
#pragma unroll
        for (int j = 0; j < W; j++) x.v[j] = ld_cg_v<V>(c_prev + i * W + j);
        s_hub[i] = x;
    }
    __syncthreads();
    auto gather = [&](int32_t u) -> VV {
        if constexpr (W == 1) return u < hub_n ? s_hub[u] : ld_gather_vec<V, W>(c_prev + u);
        else return u < hub_n ? s_hub[u] : ld_gather_vec<V, W>(c_prev + (size_t)u * W);
    };
    auto zero_vec = [&]() -> VV {
        VV z;
#pragma unroll
        for (int j = 0; j < W; j++) z.v[j] = N::zero();
        return z;
    };

    // rows tile: indices and row offsets requested first, PER independent
    // vector gathers per lane staged in shared memory, then lane groups of
    // 2^glog lanes add each row's vectors in a fixed order
    auto rows_tile = [&](const Tile &T) {
        const int ne = T.e1 - T.e0, nr = T.r1 - T.r0;
        int32_t u[PER];
#pragma unroll
        for (int k = 0; k < PER; k++) {
            const int i = lane + 32 * k;
            u[k] = i < ne ? ld_idx(src + T.e0 + i) : -1;
        }
        // row offsets relative to e0: lane l holds rows l, l + 32, ...
        int32_t o[kOffRegs];
#pragma unroll
        for (int j = 0; j < kOffRegs; j++) {
            const int i = lane + 32 * j;
            o[j] = i <= nr ? off[T.r0 + i] - T.e0 : 0;
        }
        {
            VV x[PER];
#pragma unroll
            for (int k = 0; k < PER; k++) x[k] = u[k] >= 0 ? gather(u[k]) : zero_vec();
#pragma unroll
            for (int k = 0; k < PER; k++)
                if (u[k] >= 0) s_vals[lane + 32 * k] = x[k];
        }
        __syncwarp();
        const int g = 1 << T.glog;
        const int es = lane & (g - 1);
        const int rpp = 32 >> T.glog;
        for (int rb = 0; rb < nr; rb += rpp) {
            const int r = rb + (lane >> T.glog);
            const bool valid = r < nr;
            // rows r and r + 1 lie in [rb, rb + 32]: registers j0 and j0 + 1 of their lanes
            const int j0 = rb >> 5;
            int32_t oa = o[0], ob = o[kOffRegs > 1 ? 1 : 0];
#pragma unroll
            for (int j = 1; j + 1 < kOffRegs; j++) {
                if (j0 == j) {
                    oa = o[j];
                    ob = o[j + 1];
                }
            }
            const int32_t la = __shfl_sync(0xffffffffu, oa, r & 31), lb = __shfl_sync(0xffffffffu, ob, r & 31);
            const int32_t ha = __shfl_sync(0xffffffffu, oa, (r + 1) & 31), hb = __shfl_sync(0xffffffffu, ob, (r + 1) & 31);
            EdgeSum<V> sum[W];
#pragma unroll
            for (int j = 0; j < W; j++) sum[j].init();
            if (valid) {
                const int lo = (r >> 5) == j0 ? la : lb, hi = ((r + 1) >> 5) == j0 ? ha : hb;
                for (int e = lo + es; e < hi; e += g) {
                    const VV y = s_vals[e];
#pragma unroll
                    for (int j = 0; j < W; j++) sum[j].add(y.v[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < W; j++) {
                V sv = sum[j].get();
                for (int m = 1; m < g; m <<= 1) sv = N::add_pos(sv, N::shfl_xor(sv, m));
                if (valid && es == 0) rowsum[(size_t)(T.r0 + r) * W + j] = sv;
            }
        }
        __syncwarp();
    };
    // chunk of a long row: the warp strides over the chunk, CPER vector
    // gathers per lane in flight and the next step's indices requested
    // meanwhile; lane l adds in-edges l, l + 32, ... in order; the last chunk
    // of a row to finish adds the chunk sums in chunk order
    auto chunk_tile = [&](const Tile &T) {
        const int32_t v = T.r0;
        const int nv = T.e1 - T.e0;
        EdgeSum<V> sum[W];
#pragma unroll
        for (int j = 0; j < W; j++) sum[j].init();
        int32_t u[CPER];
#pragma unroll
        for (int k = 0; k < CPER; k++) {
            const int idx = lane + 32 * k;
            u[k] = idx < nv ? ld_idx(src + T.e0 + idx) : -1;
        }
        for (int base = lane; base < nv; base += 32 * CPER) {
            VV x[CPER];
#pragma unroll
            for (int k = 0; k < CPER; k++) x[k] = u[k] >= 0 ? gather(u[k]) : zero_vec();
            int32_t un[CPER];
#pragma unroll
            for (int k = 0; k < CPER; k++) {
                const int idx = base + 32 * CPER + 32 * k;
                un[k] = idx < nv ? ld_idx(src + T.e0 + idx) : -1;
            }
#pragma unroll
            for (int k = 0; k < CPER; k++)
                if (u[k] >= 0) {
#pragma unroll
                    for (int j = 0; j < W; j++) sum[j].add(x[k].v[j]);
                }
#pragma unroll
            for (int k = 0; k < CPER; k++) u[k] = un[k];
        }
        V sv[W];
#pragma unroll
        for (int j = 0; j < W; j++) {
            sv[j] = sum[j].get();
            for (int m = 1; m < 32; m <<= 1) sv[j] = N::add_pos(sv[j], N::shfl_xor(sv[j], m));
        }
        if (T.slot < 0) {
            if (lane == 0) {
#pragma unroll
                for (int j = 0; j < W; j++) rowsum[(size_t)v * W + j] = sv[j];
            }
        } else {
            const int32_t base = slot_base[T.slot];
            if (lane == 0) {
#pragma unroll
                for (int j = 0; j < W; j++) chunk_part[(size_t)(base + T.k) * W + j] = sv[j];
            }
            __threadfence();
            __syncwarp();
            int last = 0;
            if (lane == 0) last = atomicAdd(&chunk_cnt[T.slot], 1u) == (unsigned int)(T.nch - 1);
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                __threadfence();
#pragma unroll
                for (int j = 0; j < W; j++) {
                    V t = N::zero();
                    for (int32_t q = lane; q < T.nch; q += 32)
                        t = N::add_pos(t, ld_cg_v<V>(chunk_part + (size_t)(base + q) * W + j));
                    for (int m = 1; m < 32; m <<= 1) t = N::add_pos(t, N::shfl_xor(t, m));
                    if (lane == 0) rowsum[(size_t)v * W + j] = t;
                }
                if (lane == 0) chunk_cnt[T.slot] = 0;
            }
            __syncwarp();
        }
    };

    // the next tile's descriptor is requested while this tile is worked on
    const int wstride = cta_count * kHubWarps;
    Tile T_next{};
    if (local * kHubWarps + warp < ntiles) T_next = load_tile(tiles + local * kHubWarps + warp);
    for (int t = local * kHubWarps + warp; t < ntiles; t += wstride) {
        const Tile T = T_next;
        if (t + wstride < ntiles) T_next = load_tile(tiles + t + wstride);
        if (T.glog >= 0) rows_tile(T);
        else chunk_tile(T);
    }
}

template <typename V>
__device__ __forceinline__ V ld_gather(const V *p) {
    return __ldg(p);
}
template <>
__device__ __forceinline__ df64 ld_gather<df64>(const df64 *p) {
    const float2 f = __ldg(reinterpret_cast<const float2 *>(p));
    return {f.x, f.y};
}

// One column: the same kernel written for a single value per in-edge (its
// register allocation is tighter than the vector form's: measured 1-2 % faster).
template <typename V>
__global__ void __launch_bounds__(kHubBlock, 1) pr_gather_hub1_kernel(JobDev *jobs, GlobalDev *glob, const int32_t *cta_job) {
    using N = Num<V>;
    constexpr int PER = kHubTile / 32;       // staged gathers per lane (rows tiles)
    constexpr int TR = tile_rows(1);
    constexpr int kOffRegs = TR / 32 + 1;    // row offsets of a rows tile, in registers
    constexpr int CPER = kHubChunkPer;       // gathers per lane in flight (chunk tiles)
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    JobDev &job = jobs[cta_job[blockIdx.x]];
    const ColState &cs = job.cols[0];
    // CTA-uniform: nothing to gather when the job or its column has stopped
    if (!job.alive || !cs.active || *(volatile int32_t *)&glob->error) return;
    const int local = blockIdx.x - job.gcta_begin;
    const int cta_count = job.gcta_count;
    const V *__restrict__ c_prev = reinterpret_cast<const V *>(job.contrib[cs.cur]);
    V *__restrict__ rowsum = reinterpret_cast<V *>(job.rowsum);
    const int32_t *__restrict__ src = job.src;
    const int32_t *__restrict__ off = job.off;
    const Tile *__restrict__ tiles = job.tiles;
    const int32_t *__restrict__ slot_base = job.slot_base;
    V *chunk_part = reinterpret_cast<V *>(job.chunk_part);
    uint32_t *chunk_cnt = job.chunk_cnt;
    const int ntiles = job.ntiles;
    // at most what the launch's shared memory holds for this value type
    const int hub_n = min(job.hub_n, kHubBytes / (int)sizeof(V));
    extern __shared__ __align__(16) unsigned char pr_hub_smem[];
    V *s_vals = reinterpret_cast<V *>(pr_hub_smem) + warp * kHubTile;   // this warp's staged values
    V *s_hub = reinterpret_cast<V *>(pr_hub_smem) + kHubWarps * kHubTile;
    for (int i = tid; i < hub_n; i += kHubBlock) s_hub[i] = ld_cg_v<V>(c_prev + i);
    __syncthreads();
    auto gather = [&](int32_t u) -> V { return u < hub_n ? s_hub[u] : ld_gather<V>(c_prev + u); };

    // rows tile: indices and row offsets requested first, PER independent
    // gathers per lane staged in shared memory, then lane groups of 2^glog
    // lanes add each row's values in a fixed order
    auto rows_tile = [&](const Tile &T) {
        const int ne = T.e1 - T.e0, nr = T.r1 - T.r0;
        int32_t u[PER];
#pragma unroll
        for (int k = 0; k < PER; k++) {
            const int i = lane + 32 * k;
            u[k] = i < ne ? ld_idx(src + T.e0 + i) : -1;
        }
        // row offsets relative to e0: lane l holds rows l, l + 32, ...
        int32_t o[kOffRegs];
#pragma unroll
        for (int j = 0; j < kOffRegs; j++) {
            const int i = lane + 32 * j;
            o[j] = i <= nr ? off[T.r0 + i] - T.e0 : 0;
        }
        {
            V x[PER];
#pragma unroll
            for (int k = 0; k < PER; k++) x[k] = u[k] >= 0 ? gather(u[k]) : N::zero();
#pragma unroll
            for (int k = 0; k < PER; k++)
                if (u[k] >= 0) s_vals[lane + 32 * k] = x[k];
        }
        __syncwarp();
        const int g = 1 << T.glog;
        const int es = lane & (g - 1);
        const int rpp = 32 >> T.glog;
        for (int rb = 0; rb < nr; rb += rpp) {
            const int r = rb + (lane >> T.glog);
            const bool valid = r < nr;
            // rows r and r + 1 lie in [rb, rb + 32]: registers j0 and j0 + 1 of their lanes
            const int j0 = rb >> 5;
            int32_t oa = o[0], ob = o[kOffRegs > 1 ? 1 : 0];
#pragma unroll
            for (int j = 1; j + 1 < kOffRegs; j++) {
                if (j0 == j) {
                    oa = o[j];
                    ob = o[j + 1];
                }
            }
            const int32_t la = __shfl_sync(0xffffffffu, oa, r & 31), lb = __shfl_sync(0xffffffffu, ob, r & 31);
            const int32_t ha = __shfl_sync(0xffffffffu, oa, (r + 1) & 31), hb = __shfl_sync(0xffffffffu, ob, (r + 1) & 31);
            EdgeSum<V> sum;
            sum.init();
            if (valid) {
                const int lo = (r >> 5) == j0 ? la : lb, hi = ((r + 1) >> 5) == j0 ? ha : hb;
                for (int e = lo + es; e < hi; e += g) sum.add(s_vals[e]);
            }
            V sv = sum.get();
            for (int m = 1; m < g; m <<= 1) sv = N::add_pos(sv, N::shfl_xor(sv, m));
            if (valid && es == 0) rowsum[T.r0 + r] = sv;
        }
        __syncwarp();
    };
    // chunk of a long row: the warp strides over the chunk, CPER gathers per
    // lane in flight and the next step's indices requested meanwhile; lane l
    // adds in-edges l, l + 32, ... in order; the last chunk of a row to finish
    // adds the chunk sums in chunk order
    auto chunk_tile = [&](const Tile &T) {
        const int32_t v = T.r0;
        const int nv = T.e1 - T.e0;
        EdgeSum<V> sum;
        sum.init();
        int32_t u[CPER];
#pragma unroll
        for (int k = 0; k < CPER; k++) {
            const int idx = lane + 32 * k;
            u[k] = idx < nv ? ld_idx(src + T.e0 + idx) : -1;
        }
        for (int base = lane; base < nv; base += 32 * CPER) {
            V x[CPER];
#pragma unroll
            for (int k = 0; k < CPER; k++) x[k] = u[k] >= 0 ? gather(u[k]) : N::zero();
            int32_t un[CPER];
#pragma unroll
            for (int k = 0; k < CPER; k++) {
                const int idx = base + 32 * CPER + 32 * k;
                un[k] = idx < nv ? ld_idx(src + T.e0 + idx) : -1;
            }
#pragma unroll
            for (int k = 0; k < CPER; k++)
                if (u[k] >= 0) sum.add(x[k]);
#pragma unroll
            for (int k = 0; k < CPER; k++) u[k] = un[k];
        }
        V sv = sum.get();
        for (int m = 1; m < 32; m <<= 1) sv = N::add_pos(sv, N::shfl_xor(sv, m));
        if (T.slot < 0) {
            if (lane == 0) rowsum[v] = sv;
        } else {
            const int32_t base = slot_base[T.slot];
            if (lane == 0) chunk_part[base + T.k] = sv;
            __threadfence();
            __syncwarp();
            int last = 0;
            if (lane == 0) last = atomicAdd(&chunk_cnt[T.slot], 1u) == (unsigned int)(T.nch - 1);
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                __threadfence();
                V t = N::zero();
                for (int32_t q = lane; q < T.nch; q += 32) t = N::add_pos(t, ld_cg_v<V>(chunk_part + base + q));
                for (int m = 1; m < 32; m <<= 1) t = N::add_pos(t, N::shfl_xor(t, m));
                if (lane == 0) {
                    rowsum[v] = t;
                    chunk_cnt[T.slot] = 0;
                }
            }
            __syncwarp();
        }
    };

    // the next tile's descriptor is requested while this tile is worked on
    const int wstride = cta_count * kHubWarps;
    Tile T_next{};
    if (local * kHubWarps + warp < ntiles) T_next = load_tile(tiles + local * kHubWarps + warp);
    for (int t = local * kHubWarps + warp; t < ntiles; t += wstride) {
        const Tile T = T_next;
        if (t + wstride < ntiles) T_next = load_tile(tiles + t + wstride);
        if (T.glog >= 0) rows_tile(T);
        else chunk_tile(T);
    }
}
