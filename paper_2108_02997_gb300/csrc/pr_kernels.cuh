// pr_kernels.cuh — the fused PageRank iteration kernel.
//
// One launch performs one update of every active column of every job
// (Section 2) and decides, on the device, which columns stop (Sections 3-4):
//
//   for each row v of the job (grid-stride over work units):
//     s      = sum over in-edges u -> v of contrib[u]          (gather-SpMV)
//     r'[v]  = c0 + alpha * s                                    (new rank)
//     accumulate |r'-r|, (r'-r)^2, max|r'-r|                     (norm partials)
//     contrib'[v] = r'[v] / d_v, or add r'[v] to the dangling sum when d_v = 0
//   the last CTA of a job reduces the CTA partials in a fixed order (FP64),
//   forms L1, L2 = sqrt(sum of squares), Linf, applies every pending stopping
//   rule of each column, and computes c0 = (1-alpha)/N + alpha*D/N for the
//   next update;
//   the last job to finish decides whether another pass is needed and, inside
//   a CUDA graph, ends the graph's while-loop through its conditional handle.
//
// The in-edge sum for row v uses contrib = r/d of the previous iterate, which
// this kernel's previous launch wrote in its epilogue, so one launch per
// iteration reads the index stream once and every vector once.
#pragma once
#include "df64.cuh"
#include "pr_internal.cuh"

enum PassMode { kPassInit = 0, kPassIterate = 1 };

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

template <typename V>
__device__ __forceinline__ V ld_cg_v(const V *p);
template <>
__device__ __forceinline__ double ld_cg_v<double>(const double *p) { return __ldcg(p); }
template <>
__device__ __forceinline__ float ld_cg_v<float>(const float *p) { return __ldcg(p); }
template <>
__device__ __forceinline__ df64 ld_cg_v<df64>(const df64 *p) {
    float2 f = __ldcg(reinterpret_cast<const float2 *>(p));
    return {f.x, f.y};
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
    const V *r_prev;
    V *r_new;
    const V *c_prev;
    V *c_new;
    double *copy_dst;
    // init pass
    const double *init_src;
    int init_order, init_float, init_stride, init_col;
    V init_uniform;
};

template <typename V, int W>
__device__ __forceinline__ void row_epilogue(const JobDev &job, const ColView<V> &cv, RowAcc<V> &acc,
                                             int32_t v, V s, int mode, int col) {
    using N = Num<V>;
    size_t idx = (size_t)v * W + col;
    if (mode == kPassInit) {
        if (!cv.has) return;
        V x;
        if (cv.init_src == nullptr) {
            x = cv.init_uniform;
        } else if (cv.init_float) {
            const float *f = reinterpret_cast<const float *>(cv.init_src);
            x = N::from_double((double)f[(size_t)v * cv.init_stride + cv.init_col]);
        } else {
            int32_t src_idx = cv.init_order == 0 ? job.perm[v] : v;
            x = N::from_double(cv.init_src[(size_t)src_idx * cv.init_stride + cv.init_col]);
        }
        const_cast<V *>(cv.r_prev)[idx] = x;
        int32_t d = job.outdeg[v];
        if (d == 0) acc.dsum = N::acc_add(acc.dsum, N::acc_of(x));
        else const_cast<V *>(cv.c_prev)[idx] = N::div_int(x, d);
        acc.rsum = N::acc_add(acc.rsum, N::acc_of(x));
        return;
    }
    if (!cv.has) return;
    if (cv.active) {
        V prev = cv.r_prev[idx];
        V rn = N::axpy(cv.alpha, s, cv.c0);
        V dlt = N::sub(rn, prev);
        auto ad = N::acc_abs(dlt);
        acc.l1 = N::acc_add(acc.l1, ad);
        acc.l2 = N::acc_add(acc.l2, N::acc_sqr(ad));
        acc.linf = N::acc_max(acc.linf, ad);
        int32_t d = job.outdeg[v];
        if (d == 0) acc.dsum = N::acc_add(acc.dsum, N::acc_of(rn));
        else cv.c_new[idx] = N::div_int(rn, d);
        acc.rsum = N::acc_add(acc.rsum, N::acc_of(rn));
        cv.r_new[idx] = rn;
    }
    if (cv.copy_dst) cv.copy_dst[job.perm[v]] = N::to_double(cv.r_prev[idx]);
}

template <typename V, int W>
__global__ void __launch_bounds__(kBlock) pr_iter_kernel(JobDev *jobs, GlobalDev *glob,
                                                         const int32_t *cta_job, int mode) {
    using N = Num<V>;
    using Acc = typename N::Acc;
    static_assert(32 % W == 0, "W must divide the warp");
    const int tid = threadIdx.x;
    const int col = tid % W;
    const int jid = cta_job[blockIdx.x];
    JobDev &job = jobs[jid];
    const int local = blockIdx.x - job.cta_begin;

    __shared__ Acc s_red[kWarps][W][kPartials];
    __shared__ V s_chunk[kWarps][W];
    __shared__ int s_flag;
    __shared__ double s_tot[kBlock];
    __shared__ double s_fin[W * kPartials];

    // ---- this thread's column
    ColView<V> cv;
    cv.has = col < job.ncols;
    cv.active = false;
    cv.copy_dst = nullptr;
    cv.init_src = nullptr;
    if (cv.has) {
        const ColState &cs = job.cols[col];
        int cur = cs.cur;
        cv.active = (mode == kPassIterate) && cs.active;
        cv.alpha = load_raw<V>(cs.v_alpha);
        cv.c0 = load_raw<V>(cs.v_c0);
        cv.r_prev = reinterpret_cast<const V *>(job.r[cur]);
        cv.r_new = reinterpret_cast<V *>(job.r[cur ^ 1]);
        cv.c_prev = reinterpret_cast<const V *>(job.contrib[cur]);
        cv.c_new = reinterpret_cast<V *>(job.contrib[cur ^ 1]);
        cv.copy_dst = mode == kPassIterate ? cs.copy_dst : nullptr;
        cv.init_src = cs.init_src;
        cv.init_order = cs.init_order;
        cv.init_float = cs.init_float;
        cv.init_stride = cs.init_col_stride;
        cv.init_col = cs.init_col;
        cv.init_uniform = load_raw<V>(cs.v_c0);   // init pass: host stores 1/N here
    }
    // Loop guard independent of the pass bookkeeping below: should the job
    // finalizers ever fail to stop the graph's while-loop, the launch after the
    // cap ends it (no other thread sets the condition in that case).
    if (mode == kPassIterate && blockIdx.x == 0 && tid == 0) {
        unsigned int nb = atomicAdd(&glob->body_count, 1u) + 1u;
        if (nb > (unsigned int)glob->pass_cap + 8u) {
            glob->error = 3;
            if (glob->cond) cudaGraphSetConditional((cudaGraphConditionalHandle)glob->cond, 0u);
        }
    }
    const bool work = (mode == kPassInit) || job.alive;
    RowAcc<V> acc;
    acc.init();
    const int32_t *__restrict__ off = job.off;
    const int32_t *__restrict__ src = job.src;

    if (work) {
        for (int u = local; u < job.nunits; u += job.cta_count) {
            const Unit U = job.units[u];
            if (U.c < 0) {
                // ---------------- rows of one in-degree class, g lanes per row
                const int glog = U.d;
                const int g = 1 << glog;
                const int grp = tid >> glog;
                const int lg = tid & (g - 1);
                const int es = lg / W;
                const int ES = g / W;
                const int32_t v = U.a + grp;
                const bool valid = v < U.b;
                EdgeSum<V> sum;
                sum.init();
                if (valid && cv.active) {
                    const int32_t e0 = off[v], e1 = off[v + 1];
                    const V *cp = cv.c_prev;
                    int32_t e = e0 + es;
                    for (; e + 3 * ES < e1; e += 4 * ES) {
                        int32_t u0 = src[e], u1 = src[e + ES], u2 = src[e + 2 * ES], u3 = src[e + 3 * ES];
                        V x0 = cp[(size_t)u0 * W + col], x1 = cp[(size_t)u1 * W + col];
                        V x2 = cp[(size_t)u2 * W + col], x3 = cp[(size_t)u3 * W + col];
                        sum.add(x0); sum.add(x1); sum.add(x2); sum.add(x3);
                    }
                    for (; e < e1; e += ES) sum.add(cp[(size_t)src[e] * W + col]);
                }
                V s = sum.get();
                for (int m = W; m < g; m <<= 1) s = N::add_pos(s, N::shfl_xor(s, m));
                if (valid && es == 0) row_epilogue<V, W>(job, cv, acc, v, s, mode, col);
            } else {
                // ---------------- one chunk of a long row, whole CTA
                const int32_t v = U.a;
                const int es = tid / W;
                constexpr int ES = kBlock / W;
                EdgeSum<V> sum;
                sum.init();
                if (cv.active) {
                    const V *cp = cv.c_prev;
                    int32_t e = U.b + es;
                    for (; e + 3 * ES < U.c; e += 4 * ES) {
                        int32_t u0 = src[e], u1 = src[e + ES], u2 = src[e + 2 * ES], u3 = src[e + 3 * ES];
                        V x0 = cp[(size_t)u0 * W + col], x1 = cp[(size_t)u1 * W + col];
                        V x2 = cp[(size_t)u2 * W + col], x3 = cp[(size_t)u3 * W + col];
                        sum.add(x0); sum.add(x1); sum.add(x2); sum.add(x3);
                    }
                    for (; e < U.c; e += ES) sum.add(cp[(size_t)src[e] * W + col]);
                }
                V s = sum.get();
                for (int m = W; m < 32; m <<= 1) s = N::add_pos(s, N::shfl_xor(s, m));
                if ((tid & 31) < W) s_chunk[tid >> 5][col] = s;
                __syncthreads();
                V tot = N::zero();
                if (tid < W) {
                    for (int w = 0; w < kWarps; w++) tot = N::add_pos(tot, s_chunk[w][tid]);
                }
                if (U.d < 0) {
                    if (tid < W) row_epilogue<V, W>(job, cv, acc, v, tot, mode, col);
                } else {
                    const int32_t deg = off[v + 1] - off[v];
                    constexpr int32_t kChunk = (kBlock / W) * 8;
                    const int32_t nch = (deg + kChunk - 1) / kChunk;
                    const int32_t k = (U.b - off[v]) / kChunk;
                    V *part = reinterpret_cast<V *>(job.chunk_part);
                    const int32_t base = job.slot_base[U.d];
                    if (tid < W) part[(size_t)(base + k) * W + tid] = tot;
                    __threadfence();
                    __syncthreads();
                    if (tid == 0) {
                        unsigned int old = atomicAdd(&job.chunk_cnt[U.d], 1u);
                        s_flag = (old == (unsigned int)(nch - 1));
                    }
                    __syncthreads();
                    if (s_flag) {
                        __threadfence();
                        if (tid < W) {
                            V t = N::zero();
                            for (int32_t q = 0; q < nch; q++) t = N::add_pos(t, ld_cg_v<V>(part + (size_t)(base + q) * W + tid));
                            row_epilogue<V, W>(job, cv, acc, v, t, mode, col);
                        }
                        if (tid == 0) job.chunk_cnt[U.d] = 0;
                    }
                }
                __syncthreads();
            }
        }
    }

    // ---- CTA partials per column: lanes of the same column, then warps
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
                if (any && glob->pass >= glob->pass_cap) {
                    glob->error = 2;
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
