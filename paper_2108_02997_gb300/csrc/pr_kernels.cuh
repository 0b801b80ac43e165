// pr_kernels.cuh — the fused PageRank iteration kernel and its init pass.
//
// One launch of pr_iter_kernel performs one update of every active column of
// every job (Section 2) and decides, on the device, which columns stop
// (Sections 3-4):
//
//   for each tile of rows (grid-stride over the job's tiles):
//     stage the tile's in-edge indices, row offsets, out-degrees and previous
//       ranks in shared memory with bulk asynchronous copies (cp.async.bulk,
//       completion counted on an mbarrier), the next tile's copies in flight
//       while this one is computed;
//     gather contrib[u] = r[u]/d_u for every in-edge of the tile (a batch of
//       gathers issued before any is consumed);
//     s      = sum of the gathered values of each row               (SpMV)
//     r'[v]  = c0 + alpha * s                                        (new rank)
//     accumulate |r'-r|, (r'-r)^2, max|r'-r|                         (norms)
//     contrib'[v] = r'[v]/d_v, or add r'[v] to the dangling sum when d_v = 0
//   the last CTA of a job reduces the CTA partials in a fixed order (FP64),
//   forms L1, L2 = sqrt(sum of squares) and Linf, applies every pending
//   stopping rule of each column, and computes c0 = (1-alpha)/N + alpha*D/N
//   for the next update;
//   the last job to finish decides whether another pass is needed and, inside
//   a CUDA graph, ends the graph's while-loop through its conditional handle.
//
// Every wait on an mbarrier is bounded: past kWaitNs the CTA records
// kErrCopyTimeout, drops its remaining tiles and still reports to the pass
// bookkeeping, so the host gets PR_ETIMEOUT instead of a hung device.
#pragma once
#include "df64.cuh"
#include "pr_internal.cuh"

enum PassMode { kPassInit = 0, kPassIterate = 1 };

constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s per staged tile

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

// ---------------------------------------------------------------- bulk copies and mbarriers (PTX)
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// One 1-D bulk copy global -> shared; both addresses 16-byte aligned, bytes a
// non-zero multiple of 16. Completion is counted on the mbarrier.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Element-wise asynchronous copies global -> shared (LDGSTS): the random
// gathers of a tile are issued this way so that a whole tile's worth stays in
// flight without occupying registers. .ca keeps the lines in L1.
template <int BYTES>
__device__ __forceinline__ void cp_async_ca(void *dst, const void *src) {
    static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async size");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst)), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait: true when the phase completed, false after kWaitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > kWaitNs) return false;
    }
    return true;
}

// ---------------------------------------------------------------- shared-memory layout
// per stage:
//   src : tile_edges + 8 int32   (in-edge indices from a 16-byte-aligned start)
//   off : tile_rows + 8 int32    (offsets r0..r1)
//   od  : tile_rows + 8 int32    (out-degrees)
//   rp  : tile_rows * W + 8 values (previous ranks)
// then vals (tile_edges * W gathered values) and the stage mbarriers.
template <typename V, int W>
struct StageLayout {
    static constexpr int TE = tile_edges(W);
    static constexpr int TR = tile_rows(W);
    static constexpr size_t bytes_src = (size_t)(TE + 8) * 4;
    static constexpr size_t bytes_off = (size_t)(TR + 8) * 4;
    static constexpr size_t bytes_od = (size_t)(TR + 8) * 4;
    static constexpr size_t bytes_rp = ((size_t)(TR * W + 8) * sizeof(V) + 15) / 16 * 16;
    static constexpr size_t stage_bytes = bytes_src + bytes_off + bytes_od + bytes_rp;
    static constexpr size_t vals_bytes = (size_t)TE * W * sizeof(V);
    static constexpr size_t total = kStages * stage_bytes + 2 * vals_bytes + 8 * kStages;
};

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

template <typename V>
__device__ __forceinline__ ColView<V> col_view(const JobDev &job, int col) {
    ColView<V> cv;
    cv.has = col < job.ncols;
    cv.active = false;
    cv.copy_dst = nullptr;
    cv.r_prev = cv.c_prev = nullptr;
    cv.r_new = cv.c_new = nullptr;
    if (cv.has) {
        const ColState &cs = job.cols[col];
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

// New rank of row v in the thread's column: norms, contribution or dangling
// sum; and the copy of the current iterate into a stopping rule's output.
// `prev` is the staged previous rank (valid for active columns, whose buffer
// parity is the job's).
template <typename V, int W>
__device__ __forceinline__ void row_update(const JobDev &job, const ColView<V> &cv, RowAcc<V> &acc, int32_t v,
                                           int col, V s, V prev, int32_t d) {
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
    if (cv.copy_dst) cv.copy_dst[job.perm[v]] = N::to_double(cv.active ? prev : cv.r_prev[idx]);
}

// ---------------------------------------------------------------- pass bookkeeping
// CTA partials of the thread accumulators, then the job finalizer (last CTA of
// the job) and the global decision (last job). Shared by both kernels.
template <typename V, int W>
__device__ void finish_pass(JobDev *jobs, JobDev &job, GlobalDev *glob, RowAcc<V> &acc, int local, int mode) {
    using N = Num<V>;
    using Acc = typename N::Acc;
    const int tid = threadIdx.x;
    const int col = tid % W;
    __shared__ Acc s_red[kWarps][W][kPartials];
    __shared__ int s_flag;
    __shared__ double s_tot[kBlock];
    __shared__ double s_fin[W * kPartials];
    {
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
            job.cta_part[((size_t)local * W + c) * kPartials + k] = N::acc_to_double(t);
        }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        unsigned int old = atomicAdd(&job.arrive, 1u);
        s_flag = (old == (unsigned int)(job.cta_count - 1));
    }
    __syncthreads();
    if (!s_flag) return;
    __threadfence();
    // ---- last CTA of the job: fixed-order FP64 reduction over its CTAs
    {
        constexpr int P = W * kPartials;
        constexpr int S = kBlock / P;
        const int p = tid % P, sl = tid / P;
        const int k = p % kPartials;
        double t = 0.0;
        if (sl < S) {
            for (int c = sl; c < job.cta_count; c += S) {
                double x = ld_cg(job.cta_part + (size_t)c * P + p);
                t = (k == 2) ? fmax(t, x) : t + x;
            }
        }
        s_tot[tid] = t;
        __syncthreads();
        if (tid < P) {
            double r = s_tot[tid];
            for (int q = 1; q < S; q++) {
                double x = s_tot[q * P + tid];
                r = (k == 2) ? fmax(r, x) : r + x;
            }
            s_fin[tid] = r;
        }
        __syncthreads();
    }
    // ---- column decisions (one thread per column)
    if (tid < job.ncols) {
        ColState &cs = job.cols[tid];
        const double l1 = s_fin[tid * kPartials + 0];
        const double l2 = sqrt(s_fin[tid * kPartials + 1]);
        const double li = s_fin[tid * kPartials + 2];
        const double D = s_fin[tid * kPartials + 3];
        const double S = s_fin[tid * kPartials + 4];
        const double Nn = (double)job.n;
        if (mode == kPassInit) {
            cs.c0 = (1.0 - cs.alpha) / Nn + cs.alpha * D / Nn;
            store_raw<V>(cs.v_c0, N::from_double(cs.c0));
            cs.last_sum = S;
            cs.copy_dst = nullptr;
        } else if (cs.active) {
            const int it = ++cs.iters;
            cs.cur ^= 1;
            cs.last_err[0] = l1; cs.last_err[1] = l2; cs.last_err[2] = li;
            cs.last_sum = S;
            if (cs.hist && it <= cs.hist_cap) {
                cs.hist[3 * (it - 1) + 0] = l1;
                cs.hist[3 * (it - 1) + 1] = l2;
                cs.hist[3 * (it - 1) + 2] = li;
            }
            const double errs[3] = {l1, l2, li};
            int primary = -1;
            bool pending = false;
            for (int q = cs.tap_begin; q < cs.tap_end; q++) {
                Tap &tp = job.taps[q];
                if (tp.fired) continue;
                const double e = errs[tp.norm - 1];
                if (e < tp.tau || it >= tp.max_iter) {
                    tp.fired = 1;
                    tp.iters = it;
                    tp.err = e;
                    tp.err_l1 = l1;
                    tp.converged = e < tp.tau;
                    tp.alias_of = primary;
                    if (primary < 0) primary = q;
                } else {
                    pending = true;
                }
            }
            cs.copy_dst = primary >= 0 ? job.taps[primary].out : nullptr;
            if (!pending) cs.active = 0;
            if (cs.switch_norm && !cs.switched && errs[cs.switch_norm - 1] <= cs.switch_tol) {
                cs.switched = 1;
                cs.active = 0;   // hand over to the refinement phase
            }
            cs.c0 = (1.0 - cs.alpha) / Nn + cs.alpha * D / Nn;
            store_raw<V>(cs.v_c0, N::from_double(cs.c0));
        } else {
            cs.copy_dst = nullptr;
        }
    }
    __syncthreads();
    if (tid == 0) {
        int alive = 0;
        for (int c = 0; c < job.ncols; c++) {
            const volatile ColState &cs = job.cols[c];
            if (cs.active || cs.copy_dst) alive = 1;
        }
        job.alive = alive;
        if (mode == kPassIterate) job.cur ^= 1;   // parity shared by the columns still active
        job.arrive = 0;
        __threadfence();
        unsigned int old = atomicAdd(&glob->jobs_arrive, 1u);
        if (old == (unsigned int)(glob->njobs - 1)) {
            __threadfence();
            glob->jobs_arrive = 0;
            int any = 0;
            for (int q = 0; q < glob->njobs; q++)
                if (*(volatile int32_t *)&jobs[q].alive) any = 1;
            if (mode == kPassIterate) {
                glob->pass += 1;
                if (*(volatile int32_t *)&glob->error) any = 0;
                if (any && glob->pass >= glob->pass_cap) {
                    glob->error = kErrPassCap;
                    any = 0;
                }
                glob->alive = any;
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

// ---------------------------------------------------------------- the iteration kernel
// Per CTA, tiles flow through three steps, each one tile ahead of the next:
//   k+2 : bulk copy of indices/offsets/out-degrees/previous ranks (TMA engine)
//   k+1 : random gathers contrib[src] -> vals[(k+1) % 2] with cp.async
//   k   : row sums from vals[k % 2], new ranks, norms (this tile)
template <typename V, int W>
__global__ void __launch_bounds__(kBlock, 4) pr_iter_kernel(JobDev *jobs, GlobalDev *glob, const int32_t *cta_job) {
    using N = Num<V>;
    using L = StageLayout<V, W>;
    static_assert(32 % W == 0, "W must divide the warp");
    constexpr int E16 = 16 / (int)sizeof(V);   // values per 16 bytes
    const int tid = threadIdx.x;
    const int col = tid % W;
    JobDev &job = jobs[cta_job[blockIdx.x]];
    const int local = blockIdx.x - job.cta_begin;

    extern __shared__ __align__(128) unsigned char smem[];
    V *vals0 = reinterpret_cast<V *>(smem + kStages * L::stage_bytes);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kStages * L::stage_bytes + 2 * L::vals_bytes);
    __shared__ Tile s_tile[kStages];
    __shared__ int s_fail;
    __shared__ V s_chunk[kWarps][W];
    __shared__ int s_last;

    // Loop guard independent of the pass bookkeeping: should the job
    // finalizers ever fail to stop the graph's while-loop, the launch after the
    // cap ends it (no other thread sets the condition in that case).
    if (blockIdx.x == 0 && tid == 0) {
        unsigned int nb = atomicAdd(&glob->body_count, 1u) + 1u;
        if (nb > (unsigned int)glob->pass_cap + 8u) {
            glob->error = kErrLoopGuard;
            if (glob->cond) cudaGraphSetConditional((cudaGraphConditionalHandle)glob->cond, 0u);
        }
    }
    const ColView<V> cv = col_view<V>(job, col);
    const V *rp_base = reinterpret_cast<const V *>(job.r[job.cur]);
    RowAcc<V> acc;
    acc.init();
    const bool work = job.alive && !*(volatile int32_t *)&glob->error;
    int ntl = 0;
    if (work && local < job.ntiles) ntl = (job.ntiles - 1 - local) / job.cta_count + 1;

    if (tid == 0) {
        s_fail = 0;
        for (int s = 0; s < kStages; s++) mbar_init(&bars[s], 1);
        mbar_fence_init();
    }
    __syncthreads();

    // Thread 0 stages the CTA's k-th tile into stage k % kStages.
    auto stage_tile = [&](int k) {
        const int s = k % kStages;
        const Tile T = job.tiles[local + (size_t)k * job.cta_count];
        s_tile[s] = T;
        unsigned char *st = smem + s * L::stage_bytes;
        const int32_t ea = T.e0 & ~3, eb = (T.e1 + 3) & ~3;
        const int32_t oa = T.r0 & ~3, ob = (T.r1 + 1 + 3) & ~3;
        const int32_t da = T.r0 & ~3, db = (T.r1 + 3) & ~3;
        const long long ra = ((long long)T.r0 * W) / E16 * E16;
        const long long rb = (((long long)T.r1 * W) + E16 - 1) / E16 * E16;
        const uint32_t b_src = (uint32_t)(eb - ea) * 4u, b_off = (uint32_t)(ob - oa) * 4u;
        const uint32_t b_od = (uint32_t)(db - da) * 4u, b_rp = (uint32_t)(rb - ra) * (uint32_t)sizeof(V);
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bars[s], b_src + b_off + b_od + b_rp);
        if (b_src) bulk_copy_g2s(st, job.src + ea, b_src, &bars[s]);
        bulk_copy_g2s(st + L::bytes_src, job.off + oa, b_off, &bars[s]);
        bulk_copy_g2s(st + L::bytes_src + L::bytes_off, job.outdeg + da, b_od, &bars[s]);
        bulk_copy_g2s(st + L::bytes_src + L::bytes_off + L::bytes_od, rp_base + ra, b_rp, &bars[s]);
    };
    // All threads: wait for tile k's staged data, then issue its gathers.
    auto gather_tile = [&](int k) -> bool {
        const int s = k % kStages;
        if (!mbar_wait_bounded(&bars[s], (uint32_t)((k / kStages) & 1))) return false;
        const Tile &T = s_tile[s];
        const int32_t *s_src = reinterpret_cast<const int32_t *>(smem + s * L::stage_bytes) + (T.e0 & 3);
        V *vals = vals0 + (size_t)(k & 1) * (L::vals_bytes / sizeof(V));
        const int nv = (T.e1 - T.e0) * W;
        if (cv.active) {
            const V *cp = cv.c_prev;
            for (int idx = tid; idx < nv; idx += kBlock)
                cp_async_ca<sizeof(V)>(vals + idx, cp + (size_t)s_src[idx / W] * W + col);
        }
        cp_async_commit();
        return true;
    };

    if (tid == 0)
        for (int k = 0; k < 2 && k < ntl; k++) stage_tile(k);
    if (ntl > 0 && !gather_tile(0)) s_fail = 1;

    int k = 0;
    for (; k < ntl; k++) {
        if (tid == 0 && k + 2 < ntl) stage_tile(k + 2);
        if (k + 1 < ntl) {
            if (!gather_tile(k + 1)) s_fail = 1;
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        if (s_fail) break;
        const int s = k % kStages;
        const Tile T = s_tile[s];
        const unsigned char *st = smem + s * L::stage_bytes;
        const int32_t *s_off = reinterpret_cast<const int32_t *>(st + L::bytes_src) + (T.r0 & 3);
        const int32_t *s_od = reinterpret_cast<const int32_t *>(st + L::bytes_src + L::bytes_off) + (T.r0 & 3);
        const V *s_rp = reinterpret_cast<const V *>(st + L::bytes_src + L::bytes_off + L::bytes_od) +
                        ((long long)T.r0 * W - ((long long)T.r0 * W) / E16 * E16);
        const V *vals = vals0 + (size_t)(k & 1) * (L::vals_bytes / sizeof(V));
        const int nv = (T.e1 - T.e0) * W;
        if (T.glog >= 0) {
            // ---- rows: g lanes per row add the row's values from shared memory
            const int g = 1 << T.glog;
            const int lg = tid & (g - 1);
            const int es = lg / W;
            const int ES = g / W;
            const int rows_per_pass = kBlock >> T.glog;
            for (int32_t rb = T.r0; rb < T.r1; rb += rows_per_pass) {
                const int32_t v = rb + (tid >> T.glog);
                const bool valid = v < T.r1;
                EdgeSum<V> sum;
                sum.init();
                if (valid && cv.active) {
                    const int lo = s_off[v - T.r0] - T.e0, hi = s_off[v - T.r0 + 1] - T.e0;
                    for (int e = lo + es; e < hi; e += ES) sum.add(vals[e * W + col]);
                }
                V sv = sum.get();
                for (int m = W; m < g; m <<= 1) sv = N::add_pos(sv, N::shfl_xor(sv, m));
                if (valid && es == 0 && cv.has)
                    row_update<V, W>(job, cv, acc, v, col, sv, s_rp[(v - T.r0) * W + col], s_od[v - T.r0]);
            }
        } else {
            // ---- chunk of a long row: the whole CTA adds it per column
            EdgeSum<V> sum;
            sum.init();
            if (cv.active)
                for (int idx = tid; idx < nv; idx += kBlock) sum.add(vals[idx]);
            V sv = sum.get();
            for (int m = W; m < 32; m <<= 1) sv = N::add_pos(sv, N::shfl_xor(sv, m));
            if ((tid & 31) < W) s_chunk[tid >> 5][col] = sv;
            __syncthreads();
            V tot = N::zero();
            if (tid < W)
                for (int w = 0; w < kWarps; w++) tot = N::add_pos(tot, s_chunk[w][tid]);
            const int32_t v = T.r0;
            if (T.slot < 0) {
                if (tid < W && cv.has) row_update<V, W>(job, cv, acc, v, col, tot, s_rp[col], s_od[0]);
            } else {
                V *part = reinterpret_cast<V *>(job.chunk_part);
                const int32_t base = job.slot_base[T.slot];
                if (tid < W) part[(size_t)(base + T.k) * W + tid] = tot;
                __threadfence();
                __syncthreads();
                if (tid == 0) {
                    unsigned int old = atomicAdd(&job.chunk_cnt[T.slot], 1u);
                    s_last = (old == (unsigned int)(T.nch - 1));
                }
                __syncthreads();
                if (s_last) {
                    __threadfence();
                    if (tid < W && cv.has) {
                        V t = N::zero();
                        for (int32_t q = 0; q < T.nch; q++) t = N::add_pos(t, ld_cg_v<V>(part + (size_t)(base + q) * W + tid));
                        row_update<V, W>(job, cv, acc, v, col, t, s_rp[col], s_od[0]);
                    }
                    if (tid == 0) job.chunk_cnt[T.slot] = 0;
                }
            }
        }
        __syncthreads();   // stage k % kStages and vals[k % 2] are free again
    }
    if (s_fail) {
        // a staged copy did not arrive in time: let this CTA's element copies
        // land, wait (bounded) for its bulk copies in flight, record the error,
        // skip the remaining tiles and still take part in the pass bookkeeping
        cp_async_wait<0>();
        if (tid == 0) {
            for (int j = k + 1; j < ntl && j < k + 3; j++)
                mbar_wait_bounded(&bars[j % kStages], (uint32_t)((j / kStages) & 1));
            glob->error = kErrCopyTimeout;
        }
        __syncthreads();
    }
    finish_pass<V, W>(jobs, job, glob, acc, local, kPassIterate);
}
