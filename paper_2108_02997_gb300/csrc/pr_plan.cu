// pr_plan.cu — how pr_solve_batch groups its columns into jobs.
//
// A job holds W columns of one graph (W = 1, 2, 4, .., 32) and costs one
// launch-time share t(W) per iteration until its slowest column stops. The
// planner measures t(W) once per graph signature (pr_graph_tune), together
// with the error decay of a few uniform-start iterations, from which it
// estimates each column's iterations; it then cuts the columns of each graph,
// sorted by estimated iterations, into the contiguous jobs that minimise
//     sum over jobs  max(iterations in the job) x t(W of the job)
// by dynamic programming. Jobs of one width share the launches of a
// sub-solve, and with them each launch's latency (measured once per signature
// as well, with four single-column jobs in one launch), so the planner also
// forms the partition for the launch times less that latency and one job per
// column, and keeps the cheapest of the three under
//     sum over widths  latency x max(iterations)
//   + sum over jobs    max(iterations in the job) x (t(W) - latency).
// Jobs run as sub-solves (one kernel launch per
// iteration for all jobs of a sub-solve): jobs of one width share a sub-solve
// while their gathered vectors together fit in half of the L2 cache, since
// jobs sharing launches also share the cache, and a job larger than that runs
// alone (it fills the GPU by itself).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <tuple>

#include "pr_internal.cuh"

namespace {

constexpr int kWidths = 6;          // W = 1, 2, 4, 8, 16, 32
constexpr int kTuneIters = 8;       // timed iterations per width
constexpr double kTuneAlpha = 0.85;

// L1 size of the rounding noise an FP32 iterate carries into the refinement
// phase of mixed precision (measured on R-MAT graphs: 1e-8 to 4e-8); unlike
// the start's error it decays only at the rate alpha.
constexpr double kMixedNoise = 3e-8;

using Table = std::array<double, kWidths>;   // microseconds per launch; 0 unknown, < 0 skipped

// Error decay of the uniform start at alpha = kTuneAlpha, per norm: the first
// difference e1 and the per-iteration ratio rho (0 = not measured).
struct Decay {
    double e1[3] = {0.0, 0.0, 0.0};
    double rho[3] = {0.0, 0.0, 0.0};
};

struct TuneEntry {
    Table us{};
    Decay decay;
    double lat = -1.0;   // per-launch latency shared by concurrent jobs (us; < 0 unknown)
};

std::mutex g_tune_mu;
std::map<std::tuple<int, int, uint64_t>, TuneEntry> g_tune;   // (device, precision, signature)

// Updates until the norm-`norm` error falls below tau, within [1, max_iter].
// Without a measured decay: the error shrinks like alpha^k from about 1
// (Section 1's estimate log(tau)/log(alpha)). With one: the error starts at
// e1 * alpha / kTuneAlpha and shrinks by alpha * (rho / kTuneAlpha) per
// iteration (the graph's subdominant behaviour scaled by alpha), never slower
// than alpha.
double estimate_iterations(double alpha, double tau, int norm, int max_iter, const Decay *d) {
    double k;
    if (alpha <= 0.0) {
        k = 2.0;
    } else if (alpha >= 1.0) {
        k = (double)max_iter;
    } else if (d && d->rho[norm - 1] > 0.0 && d->e1[norm - 1] > 0.0) {
        const double rate = std::max(1e-3, std::min(alpha, alpha * d->rho[norm - 1] / kTuneAlpha));
        const double e1 = d->e1[norm - 1] * alpha / kTuneAlpha;
        k = tau >= e1 ? 1.0 : 1.0 + std::ceil(std::log(tau / e1) / std::log(rate));
    } else {
        k = std::ceil(std::log(tau) / std::log(alpha));
    }
    return std::min<double>(std::max(k, 1.0), (double)max_iter);
}

// Estimated iterations of a column per phase: {FP32 phase, DF64 refinement}
// for mixed precision, {all, 0} otherwise. A column runs until its last tap.
// d0: decay measured in the (first) phase's precision.
std::array<double, 2> column_iterations(const SolveColumn &c, int precision, double switch_tol, const Decay *d0) {
    if (precision != PR_PREC_MIXED) {
        double k = 1.0;
        for (const Tap &t : c.taps) k = std::max(k, estimate_iterations(c.alpha, t.tau, t.norm, t.max_iter, d0));
        return {k, 0.0};
    }
    // the FP32 phase ends at switch_tol in the strictest norm of the taps; the
    // refinement damps the FP32 rounding noise at the rate alpha
    int sn = 3, max_iter = 1;
    double k_all = 1.0;
    for (const Tap &t : c.taps) {
        sn = std::min(sn, (int)t.norm);
        max_iter = std::max(max_iter, (int)t.max_iter);
    }
    const double k1 = estimate_iterations(c.alpha, switch_tol, sn, max_iter, d0);
    for (const Tap &t : c.taps) {
        double k2 = 0.0;
        if (t.tau < kMixedNoise && c.alpha > 0.0 && c.alpha < 1.0)
            k2 = std::ceil(std::log(t.tau / kMixedNoise) / std::log(c.alpha));
        else if (c.alpha >= 1.0)
            k2 = (double)t.max_iter;
        k_all = std::max(k_all, std::min(k1 + k2 + 1.0, (double)t.max_iter));
    }
    return {std::min(k1, k_all), std::max(0.0, k_all - k1)};
}

int smallest_width_index(int m, const double *const *t, int nphase) {
    for (int w = 0; w < kWidths; w++) {
        if ((1 << w) < m) continue;
        bool ok = true;
        for (int p = 0; p < nphase; p++) ok = ok && t[p][w] > 0.0;
        if (ok) return w;
    }
    return -1;
}

// The partition planner. it[c][p]: iterations of column c in phase p;
// t[p][w]: launch time of phase p at width 2^w. Fills job_of / width_of per
// column (jobs numbered in sorted order). Returns false if no plan exists.
bool plan_partition(const std::vector<std::array<double, 2>> &it, const double *const *t, int nphase,
                    std::vector<int> &job_of, std::vector<int> &width_of, double *cost_out) {
    const int n = (int)it.size();
    std::vector<int> order(n);
    for (int c = 0; c < n; c++) order[c] = c;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return it[a][0] + it[a][1] > it[b][0] + it[b][1];
    });
    const double inf = std::numeric_limits<double>::infinity();
    std::vector<double> f(n + 1, inf);
    std::vector<int> take(n + 1, 0), wsel(n + 1, -1);
    f[0] = 0.0;
    for (int i = 1; i <= n; i++) {
        double mx[2] = {0.0, 0.0};
        for (int m = 1; m <= std::min(32, i); m++) {
            const int c = order[i - m];
            for (int p = 0; p < nphase; p++) mx[p] = std::max(mx[p], it[c][p]);
            const int w = smallest_width_index(m, t, nphase);
            if (w < 0 || f[i - m] == inf) continue;
            double cost = f[i - m];
            for (int p = 0; p < nphase; p++) cost += mx[p] * t[p][w];
            if (cost < f[i]) {
                f[i] = cost;
                take[i] = m;
                wsel[i] = w;
            }
        }
    }
    if (n > 0 && f[n] == inf) return false;
    job_of.assign(n, -1);
    width_of.assign(n, 0);
    std::vector<std::pair<int, int>> cuts;   // (end, size) from the back
    for (int i = n; i > 0; i -= take[i]) cuts.push_back({i, take[i]});
    std::reverse(cuts.begin(), cuts.end());
    for (size_t j = 0; j < cuts.size(); j++) {
        const int end = cuts[j].first, m = cuts[j].second;
        for (int q = end - m; q < end; q++) {
            job_of[order[q]] = (int)j;
            width_of[order[q]] = 1 << wsel[end];
        }
    }
    if (cost_out) *cost_out = f[n];
    return true;
}

// Cost of a grouping when jobs of one width share each launch, and with it
// the launch's latency lat: sum over widths lat x max(iterations) plus sum
// over jobs max(iterations in the job) x (t(W) - lat), per phase.
double shared_cost(const std::vector<std::array<double, 2>> &it, const double *const *t, int nphase,
                   const double *lat, const std::vector<int> &job_of, const std::vector<int> &width_of) {
    std::map<int, std::array<double, 2>> job_it;
    std::map<int, int> job_w;
    for (size_t k = 0; k < job_of.size(); k++) {
        auto &m = job_it[job_of[k]];
        for (int p = 0; p < nphase; p++) m[p] = std::max(m[p], it[k][p]);
        job_w[job_of[k]] = width_of[k];
    }
    std::map<int, std::array<double, 2>> width_it;
    double cost = 0.0;
    for (auto &kv : job_it) {
        int wi = 0;
        while ((1 << wi) < job_w[kv.first]) wi++;
        auto &m = width_it[wi];
        for (int p = 0; p < nphase; p++) {
            m[p] = std::max(m[p], kv.second[p]);
            cost += kv.second[p] * std::max(t[p][wi] - lat[p], 0.05 * t[p][wi]);
        }
    }
    for (auto &kv : width_it)
        for (int p = 0; p < nphase; p++) cost += kv.second[p] * lat[p];
    return cost;
}

// Given the partition for whole launch times in job_of / width_of, keeps the
// cheapest under shared_cost of: that partition, the partition for the
// launch times less the latency, and one job per column. Returns its cost.
double choose_shared_plan(const std::vector<std::array<double, 2>> &it, const double *const *t, int nphase,
                          const double *lat, std::vector<int> &job_of, std::vector<int> &width_of) {
    double best = shared_cost(it, t, nphase, lat, job_of, width_of);
    if (!(lat[0] > 0.0)) return best;
    Table vt[2];
    for (int p = 0; p < nphase; p++)
        for (int w = 0; w < kWidths; w++) vt[p][w] = t[p][w] > 0.0 ? std::max(t[p][w] - lat[p], 0.05 * t[p][w]) : t[p][w];
    const double *vp[2] = {vt[0].data(), vt[1].data()};
    std::vector<int> jo2, wo2;
    if (plan_partition(it, vp, nphase, jo2, wo2, nullptr)) {
        const double c2 = shared_cost(it, t, nphase, lat, jo2, wo2);
        if (c2 < best) {
            best = c2;
            job_of = jo2;
            width_of = wo2;
        }
    }
    std::vector<int> jo3(it.size()), wo3(it.size(), 1);
    for (size_t k = 0; k < it.size(); k++) jo3[k] = (int)k;
    const double c3 = shared_cost(it, t, nphase, lat, jo3, wo3);
    if (c3 < best) {
        best = c3;
        job_of = jo3;
        width_of = wo3;
    }
    return best;
}

// Bytes of device workspace a W-column timing solve needs (two rank and two
// contribution buffers of 8-byte slots, plus the staged answers), with slack.
double tune_bytes(const pr_graph *g, int W) { return 48.0 * (double)g->n * W + (64 << 20); }

pr_status time_width(const pr_graph *g, int precision, int W, cudaStream_t st, double *us, Decay *decay) {
    SolveRequest r;
    r.precision = precision;
    r.loop = PR_LOOP_HOST;
    r.stream = st;
    std::vector<int> job;
    for (int c = 0; c < W; c++) {
        SolveColumn sc;
        sc.g = g;
        sc.alpha = kTuneAlpha;
        Tap t{};
        t.tau = 1e-300;
        t.norm = PR_NORM_L1;
        t.max_iter = kTuneIters;
        t.alias_of = -1;
        t.out = nullptr;
        sc.taps.push_back(t);
        sc.inst.push_back(c);
        sc.host_dst.push_back(nullptr);
        r.cols.push_back(sc);
        job.push_back(c);
    }
    r.jobs.push_back(job);
    double hist[3 * kTuneIters];
    std::memset(hist, 0, sizeof(hist));
    if (decay) {
        r.cols[0].hist_host = hist;
        r.cols[0].hist_cap = kTuneIters;
    }
    std::vector<std::vector<Tap>> taps;
    pr_status s = pr_run_solve(r, taps);
    if (s != PR_OK) return s;
    *us = r.stats.kernel_ms * 1000.0 / std::max(r.stats.passes, 1);
    if (decay) {
        // e_k = e1 rho^(k-1): rho from the last four differences, where the
        // start's fastest components have died out
        for (int q = 0; q < 3; q++) {
            const double e1 = hist[q], ea = hist[3 * (kTuneIters - 5) + q], eb = hist[3 * (kTuneIters - 1) + q];
            decay->e1[q] = e1 > 0.0 && std::isfinite(e1) ? e1 : 0.0;
            decay->rho[q] = (ea > 0.0 && eb > 0.0 && eb < ea) ? std::pow(eb / ea, 0.25) : 0.0;
        }
    }
    return PR_OK;
}

// Latency share of a launch: one solve of kMultiJobs single-column jobs in
// the same launches against one job alone. The jobs' work adds, the pass's
// latency (launch, finalizer, loop) does not: t(k jobs) = lat + k v.
constexpr int kMultiJobs = 4;
pr_status time_latency(const pr_graph *g, int precision, double us1, cudaStream_t st, double *lat) {
    SolveRequest r;
    r.precision = precision;
    r.loop = PR_LOOP_HOST;
    r.stream = st;
    // the kernel form one job alone gets, so that both timings use the same kernels
    r.kernels = kSplitPasses && (double)g->nnz >= kSplitMinWork ? PR_KERNELS_SPLIT : PR_KERNELS_FUSED;
    for (int c = 0; c < kMultiJobs; c++) {
        SolveColumn sc;
        sc.g = g;
        sc.alpha = kTuneAlpha - 0.01 * c;
        Tap t{};
        t.tau = 1e-300;
        t.norm = PR_NORM_L1;
        t.max_iter = kTuneIters;
        t.alias_of = -1;
        t.out = nullptr;
        sc.taps.push_back(t);
        sc.inst.push_back(c);
        sc.host_dst.push_back(nullptr);
        r.cols.push_back(sc);
        r.jobs.push_back({c});
    }
    std::vector<std::vector<Tap>> taps;
    pr_status s = pr_run_solve(r, taps);
    if (s != PR_OK) return s;
    const double usk = r.stats.kernel_ms * 1000.0 / std::max(r.stats.passes, 1);
    const double v = std::max(0.0, (usk - us1) / (kMultiJobs - 1));
    *lat = std::max(0.0, us1 - v);
    return PR_OK;
}

size_t free_device_bytes() {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return free_b;
}

// Fills `out` with the launch times of `precision` on g for widths up to
// max_width, timing those not yet known for g's signature.
pr_status tune(const pr_graph *g, int precision, int max_width, cudaStream_t st, TuneEntry &out) {
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    const auto key = std::make_tuple(dev, precision, g->signature);
    TuneEntry te;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) te = it->second;
    }
    bool changed = false;
    for (int w = 0; w < kWidths && (1 << w) <= max_width; w++) {
        if (te.us[w] != 0.0) continue;
        size_t free_b = 0, total_b = 0;
        PR_CUDA(cudaMemGetInfo(&free_b, &total_b));
        if (w > 0 && tune_bytes(g, 1 << w) > 0.25 * (double)free_b) {
            te.us[w] = -1.0;
        } else {
            double us = 0.0;
            pr_status s = time_width(g, precision, 1 << w, st, &us, w == 0 ? &te.decay : nullptr);
            if (s != PR_OK) return s;
            te.us[w] = std::max(us, 1e-3);
        }
        changed = true;
    }
    if (te.lat < 0.0 && te.us[0] > 0.0 && tune_bytes(g, kMultiJobs) <= 0.25 * (double)free_device_bytes()) {
        pr_status s = time_latency(g, precision, te.us[0], st, &te.lat);
        if (s != PR_OK) return s;
        changed = true;
    }
    if (changed) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        TuneEntry &dst = g_tune[key];
        for (int w = 0; w < kWidths; w++)
            if (dst.us[w] == 0.0) dst.us[w] = te.us[w];
        if (dst.decay.rho[0] == 0.0) dst.decay = te.decay;
        if (dst.lat < 0.0) dst.lat = te.lat;
    }
    out = te;
    return PR_OK;
}

// Bytes of the gathered vector of a job (the part of its working set that is
// read at random and so wants to stay in L2).
double gather_bytes(const pr_graph *g, int W, int precision) {
    return (double)g->n * W * (precision == PR_PREC_FP32 ? 4.0 : 8.0);
}

int pow2_ceil(int k) {
    int w = 1;
    while (w < k) w <<= 1;
    return w;
}

}  // namespace

// Persistent passes run every job on its own CTAs and decide per job, so a
// small graph's columns finish their passes soonest as one-column jobs, as
// long as each job still gets at least half of the CTAs that give every warp
// one tile (measured on the 330-instance ER-10k sweep: 0.38 ms of device time
// as eleven one-column jobs, 0.44 ms as the graph-loop cost model's jobs). True
// when the graph's columns are few and small enough for that: the fused
// pass's work stays below the split threshold and the CTAs fit the device.
bool prefer_single_persistent(const pr_graph *g, int ncols, const SolveRequest &req) {
    if (req.loop != PR_LOOP_AUTO && req.loop != PR_LOOP_PERSISTENT) return false;
    if (req.kernels == PR_KERNELS_SPLIT) return false;
    if ((double)g->nnz * ncols >= kSplitMinWork) return false;
    const TileTable &t1 = g->tables[0];
    if (!t1.d_tiles) return false;
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (pr_kernel_setup(PR_PREC_DF64, 1, &occ) != PR_OK) return false;
    const int64_t half = (tile_ctas(t1.ntiles) + 1) / 2;
    return (int64_t)ncols * half <= (int64_t)sms * occ;
}

pr_status pr_plan_request(const SolveRequest &req, int group, std::vector<SubSolve> &plan) {
    plan.clear();
    const int ncols = (int)req.cols.size();
    std::vector<const pr_graph *> order;
    std::map<const pr_graph *, std::vector<int>> by_graph;
    for (int c = 0; c < ncols; c++) {
        if (!by_graph.count(req.cols[c].g)) order.push_back(req.cols[c].g);
        by_graph[req.cols[c].g].push_back(c);
    }
    if (group == PR_GROUP_PACK) {
        SubSolve sp;
        sp.precision = req.precision == PR_PREC_AUTO ? PR_PREC_DF64 : req.precision;
        for (const pr_graph *g : order) {
            const auto &v = by_graph[g];
            for (size_t i = 0; i < v.size(); i += 32) {
                sp.jobs.emplace_back(v.begin() + i, v.begin() + std::min(v.size(), i + 32));
                sp.W = std::max(sp.W, pow2_ceil((int)sp.jobs.back().size()));
            }
        }
        if (!sp.jobs.empty()) plan.push_back(sp);
        return PR_OK;
    }
    // ---- jobs per graph: (precision, width, request columns). PR_PREC_AUTO
    // takes, per graph, mixed precision when the cost model (measured launch
    // times of both value types, estimated iterations of both phases) predicts
    // it cheaper than DF64 throughout, else DF64; single-column graphs, which
    // are not tuned, run DF64.
    struct JobSpec {
        int precision, W;
        std::vector<int> cols;
    };
    std::vector<JobSpec> jobs_all;
    const bool auto_prec = req.precision == PR_PREC_AUTO;
    for (const pr_graph *g : order) {
        const auto &v = by_graph[g];
        if (group == PR_GROUP_SINGLE || v.size() == 1 ||
            (group == PR_GROUP_AUTO && prefer_single_persistent(g, (int)v.size(), req))) {
            const int pg = auto_prec ? PR_PREC_DF64 : req.precision;
            for (int c : v) jobs_all.push_back({pg, 1, {c}});
            continue;
        }
        const int maxw = pow2_ceil(std::min<int>((int)v.size(), 32));
        // candidate precisions for this graph, each with its plan and cost
        std::vector<int> cands;
        if (auto_prec) cands = {PR_PREC_DF64, PR_PREC_MIXED};
        else cands = {req.precision};
        double best_cost = std::numeric_limits<double>::infinity();
        int best_prec = cands[0];
        std::vector<int> best_job, best_width;
        for (int prec : cands) {
            const bool mixed = prec == PR_PREC_MIXED;
            TuneEntry t0, t1;
            pr_status s = tune(g, mixed ? PR_PREC_FP32 : prec, maxw, req.stream, t0);
            if (s != PR_OK) return s;
            if (mixed && (s = tune(g, PR_PREC_DF64, maxw, req.stream, t1)) != PR_OK) return s;
            std::vector<std::array<double, 2>> it;
            for (int c : v) it.push_back(column_iterations(req.cols[c], prec, req.switch_tol, &t0.decay));
            const int np = mixed ? 2 : 1;
            const double *tp[2] = {t0.us.data(), t1.us.data()};
            std::vector<int> job_of, width_of;
            if (!plan_partition(it, tp, np, job_of, width_of, nullptr))
                return pr_fail(PR_ECUDA, "internal: no column plan (width 1 untimed)");
            const double lat[2] = {std::max(0.0, t0.lat), std::max(0.0, mixed ? t1.lat : 0.0)};
            const double cost = choose_shared_plan(it, tp, np, lat, job_of, width_of);
            if (cost < best_cost) {
                best_cost = cost;
                best_prec = prec;
                best_job = job_of;
                best_width = width_of;
            }
        }
        std::map<int, std::pair<int, std::vector<int>>> jobs;   // job index -> (width, request columns)
        for (size_t k = 0; k < v.size(); k++) {
            jobs[best_job[k]].first = best_width[k];
            jobs[best_job[k]].second.push_back(v[k]);
        }
        for (auto &kv : jobs) jobs_all.push_back({best_prec, kv.second.first, kv.second.second});
    }
    // ---- sub-solves: jobs of one precision and width together while their
    // gathered vectors fit in half of L2; a job larger than that alone
    int dev = 0, l2 = 0;
    PR_CUDA(cudaGetDevice(&dev));
    PR_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    const double budget = 0.5 * (double)std::max(l2, 1 << 20);
    std::stable_sort(jobs_all.begin(), jobs_all.end(), [](const JobSpec &a, const JobSpec &b) {
        return a.precision != b.precision ? a.precision < b.precision : a.W < b.W;
    });
    SubSolve cur;
    double cur_bytes = 0.0;
    for (auto &jb : jobs_all) {
        const int vprec = jb.precision == PR_PREC_MIXED ? PR_PREC_DF64 : jb.precision;
        const double b = gather_bytes(req.cols[jb.cols[0]].g, jb.W, vprec);
        if (!cur.jobs.empty() && (cur.W != jb.W || cur.precision != jb.precision || cur_bytes + b > budget)) {
            plan.push_back(cur);
            cur = SubSolve();
            cur_bytes = 0.0;
        }
        cur.W = jb.W;
        cur.precision = jb.precision;
        cur.jobs.push_back(jb.cols);
        cur_bytes += b;
    }
    if (!cur.jobs.empty()) plan.push_back(cur);
    return PR_OK;
}

pr_status pr_graph_pass_model(pr_graph *g, cudaStream_t st, double *t1_us, double *lat_us, double *rho_l1) {
    TuneEntry t;
    pr_status s = tune(g, PR_PREC_DF64, 1, st, t);
    if (s != PR_OK) return s;
    *t1_us = t.us[0] > 0.0 ? t.us[0] : 0.0;
    *lat_us = t.lat > 0.0 ? t.lat : 0.0;
    *rho_l1 = t.decay.rho[0];
    return PR_OK;
}

extern "C" pr_status pr_plan_columns(int32_t count, const double *iters, const double *us_per_launch, int32_t *job_of,
                                     int32_t *width_of, double *cost_out) {
    pr_clear_error();
    if (count < 0) return pr_fail(PR_EINVAL, "count must be >= 0");
    if (count > 0 && (!iters || !us_per_launch || !job_of || !width_of)) return pr_fail(PR_EINVAL, "NULL argument");
    if (count == 0) {
        if (cost_out) *cost_out = 0.0;
        return PR_OK;
    }
    for (int32_t c = 0; c < count; c++)
        if (!(iters[c] > 0.0) || !std::isfinite(iters[c])) return pr_fail(PR_EINVAL, "iters must be positive and finite");
    for (int w = 0; w < kWidths; w++)
        if (!std::isfinite(us_per_launch[w])) return pr_fail(PR_EINVAL, "launch times must be finite");
    if (!(us_per_launch[0] > 0.0)) return pr_fail(PR_EINVAL, "width 1 must be available");
    std::vector<std::array<double, 2>> it(count);
    for (int32_t c = 0; c < count; c++) it[c] = {iters[c], 0.0};
    const double *tp[1] = {us_per_launch};
    std::vector<int> jo, wo;
    if (!plan_partition(it, tp, 1, jo, wo, cost_out)) return pr_fail(PR_EINVAL, "no plan");
    for (int32_t c = 0; c < count; c++) {
        job_of[c] = jo[c];
        width_of[c] = wo[c];
    }
    return PR_OK;
}

extern "C" pr_status pr_plan_columns_shared(int32_t count, const double *iters, const double *us_per_launch,
                                            double latency_us, int32_t *job_of, int32_t *width_of,
                                            double *cost_out) {
    pr_clear_error();
    if (!(latency_us >= 0.0) || !std::isfinite(latency_us)) return pr_fail(PR_EINVAL, "latency must be >= 0 and finite");
    double base_cost = 0.0;
    pr_status s = pr_plan_columns(count, iters, us_per_launch, job_of, width_of, &base_cost);
    if (s != PR_OK || count == 0) {
        if (s == PR_OK && cost_out) *cost_out = 0.0;
        return s;
    }
    std::vector<std::array<double, 2>> it(count);
    for (int32_t c = 0; c < count; c++) it[c] = {iters[c], 0.0};
    std::vector<int> jo(job_of, job_of + count), wo(width_of, width_of + count);
    const double *tp[1] = {us_per_launch};
    const double lat[2] = {latency_us, 0.0};
    const double cost = choose_shared_plan(it, tp, 1, lat, jo, wo);
    for (int32_t c = 0; c < count; c++) {
        job_of[c] = jo[c];
        width_of[c] = wo[c];
    }
    if (cost_out) *cost_out = cost;
    return PR_OK;
}

extern "C" pr_status pr_graph_tune(pr_graph *g, int32_t precision, int32_t max_width, void *stream, double *us_out) {
    pr_clear_error();
    if (!pr_graph_valid(g)) return pr_fail(PR_ESTATE, "not a live graph handle");
    if (precision < PR_PREC_DF64 || precision > PR_PREC_FP32) return pr_fail(PR_EINVAL, "unknown precision");
    if (max_width < 1 || max_width > 32 || (max_width & (max_width - 1)))
        return pr_fail(PR_EINVAL, "max_width must be 1, 2, 4, 8, 16 or 32");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    TuneEntry t;
    pr_status s;
    if (precision == PR_PREC_MIXED) {
        if ((s = tune(g, PR_PREC_FP32, max_width, st, t)) != PR_OK) return s;
        if ((s = tune(g, PR_PREC_DF64, max_width, st, t)) != PR_OK) return s;
    } else if ((s = tune(g, precision, max_width, st, t)) != PR_OK) {
        return s;
    }
    if (us_out)
        for (int w = 0; w < kWidths; w++) us_out[w] = t.us[w] > 0.0 && (1 << w) <= max_width ? t.us[w] : 0.0;
    return PR_OK;
}
