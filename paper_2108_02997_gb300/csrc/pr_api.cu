// pr_api.cu — C-ABI entry points: argument checks, batching, error reporting.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <unordered_set>
#include <memory>
#include <mutex>
#include <set>
#include <tuple>

#include "pr_internal.cuh"

// ------------------------------------------------------------------ errors
namespace {
thread_local std::string t_last_error;
std::mutex g_reg_mu;
std::set<const void *> g_registry;
}  // namespace

void pr_set_error(const std::string &msg) { t_last_error = msg; }
void pr_clear_error() { t_last_error.clear(); }
pr_status pr_fail(pr_status s, const std::string &msg) {
    t_last_error = msg;
    return s;
}
pr_status pr_cuda_fail(cudaError_t e, const char *what) {
    t_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return PR_ENOMEM;
    }
    return PR_ECUDA;
}

void registry_add(const void *p) {
    std::lock_guard<std::mutex> lk(g_reg_mu);
    g_registry.insert(p);
}
void registry_remove(const void *p) {
    std::lock_guard<std::mutex> lk(g_reg_mu);
    g_registry.erase(p);
}
bool registry_has(const void *p) {
    std::lock_guard<std::mutex> lk(g_reg_mu);
    return g_registry.count(p) != 0;
}

extern "C" const char *pr_last_error(void) { return t_last_error.c_str(); }

extern "C" const char *pr_status_string(pr_status s) {
    switch (s) {
        case PR_OK: return "PR_OK";
        case PR_EINVAL: return "PR_EINVAL";
        case PR_ENOMEM: return "PR_ENOMEM";
        case PR_ECUDA: return "PR_ECUDA";
        case PR_ETIMEOUT: return "PR_ETIMEOUT";
        case PR_ESTATE: return "PR_ESTATE";
        case PR_ENOTSUP: return "PR_ENOTSUP";
        default: return "PR_UNKNOWN";
    }
}

extern "C" int32_t pr_version(void) { return 10000; }

extern "C" void pr_options_default(pr_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = PR_PREC_DF64;
    opt->init = PR_INIT_UNIFORM;
    opt->switch_tol = 1e-6;
    opt->share_trajectories = 1;
    opt->loop = PR_LOOP_AUTO;
    opt->group = PR_GROUP_AUTO;
}

// Implemented in pr_learn.cu.

namespace {

pr_status check_options(const pr_options &o) {
    if (o.precision < PR_PREC_DF64 || o.precision > PR_PREC_AUTO) return pr_fail(PR_EINVAL, "unknown precision");
    if (o.init < PR_INIT_UNIFORM || o.init > PR_INIT_AUTO) return pr_fail(PR_EINVAL, "unknown init mode");
    if (o.loop < PR_LOOP_GRAPH || o.loop > PR_LOOP_AUTO) return pr_fail(PR_EINVAL, "unknown loop mode");
    if (o.group < PR_GROUP_AUTO || o.group > PR_GROUP_SINGLE) return pr_fail(PR_EINVAL, "unknown group mode");
    if (o.max_passes < 0) return pr_fail(PR_EINVAL, "max_passes must be >= 0");
    if (o.kernels < PR_KERNELS_AUTO || o.kernels > PR_KERNELS_SPLIT) return pr_fail(PR_EINVAL, "unknown kernels mode");
    if (o.persist_wait_us < 0) return pr_fail(PR_EINVAL, "persist_wait_us must be >= 0");
    if ((o.precision == PR_PREC_MIXED || o.precision == PR_PREC_AUTO) && !(o.switch_tol > 0.0 && std::isfinite(o.switch_tol)))
        return pr_fail(PR_EINVAL, "switch_tol must be positive and finite");
    if ((o.init == PR_INIT_LEARNED || o.init == PR_INIT_AUTO) && !pr_mlp_valid(o.mlp))
        return pr_fail(PR_EINVAL, "PR_INIT_LEARNED and PR_INIT_AUTO need a live pr_mlp");
    return PR_OK;
}

// `seen`: graphs of this call already found live (each handle is looked up in
// the registry once per call); `dev`: the current device, asked for once a
// live handle has been seen (-1 before).
pr_status check_instance(const pr_instance &in, int &dev, std::unordered_set<const pr_graph *> &seen) {
    if (!seen.count(in.g)) {
        if (!pr_graph_valid(in.g)) return pr_fail(PR_ESTATE, "not a live graph handle");
        seen.insert(in.g);
    }
    if (dev < 0) PR_CUDA(cudaGetDevice(&dev));
    if (in.g->device != dev)
        return pr_fail(PR_EINVAL, "the graph lives on device " + std::to_string(in.g->device) + " but device " +
                                      std::to_string(dev) + " is current");
    if (!(in.alpha >= 0.0 && in.alpha <= 1.0)) return pr_fail(PR_EINVAL, "alpha must be in [0, 1]");
    if (!(in.tol > 0.0) || !std::isfinite(in.tol)) return pr_fail(PR_EINVAL, "tol must be positive and finite");
    if (in.norm < PR_NORM_L1 || in.norm > PR_NORM_LINF) return pr_fail(PR_EINVAL, "norm must be 1 (L1), 2 (L2) or 3 (Linf)");
    if (in.max_iter < 1) return pr_fail(PR_EINVAL, "max_iter must be >= 1");
    if (!in.ranks_out) return pr_fail(PR_EINVAL, "ranks_out is NULL");
    return PR_OK;
}


}  // namespace

static pr_status pr_solve_batch_ex(pr_instance *inst, int32_t count, const pr_options *opt_in, double *hist_host,
                                       int32_t hist_cap) {
    pr_clear_error();
    if (count < 0) return pr_fail(PR_EINVAL, "count must be >= 0");
    if (count > 0 && !inst) return pr_fail(PR_EINVAL, "inst is NULL");
    pr_options opt;
    if (opt_in) opt = *opt_in; else pr_options_default(&opt);
    pr_status s = check_options(opt);
    if (s != PR_OK) return s;
    if (count == 0) return PR_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(opt.stream);
    pr_status first = PR_OK;
    std::string first_msg;
    std::vector<int> ok;
    int dev = -1;
    std::unordered_set<const pr_graph *> seen;
    for (int32_t i = 0; i < count; i++) {
        s = check_instance(inst[i], dev, seen);
        if (s == PR_OK && opt.init == PR_INIT_USER && !inst[i].init_vec && !opt.init_vec)
            s = pr_fail(PR_EINVAL, "PR_INIT_USER needs init_vec");
        inst[i].status = s;
        if (s != PR_OK) {
            if (first == PR_OK) { first = s; first_msg = pr_last_error(); }
            continue;
        }
        ok.push_back(i);
    }
    // ---- start vectors on the device (caller order)
    std::vector<std::unique_ptr<PoolBuf>> bufs;
    std::map<std::pair<const void *, const void *>, const double *> init_dev;   // (graph, src) -> device copy
    std::map<std::pair<const pr_graph *, uint64_t>, const double *> learned;
    std::map<const pr_graph *, const void *> learned_feat;
    std::map<std::pair<const pr_graph *, uint64_t>, bool> auto_use;   // PR_INIT_AUTO decisions per (graph, alpha)
    std::map<const pr_graph *, int> alphas_on;                          // distinct alphas per graph
    if (opt.init == PR_INIT_AUTO) {
        std::set<std::pair<const pr_graph *, uint64_t>> seen;
        for (int i : ok) {
            uint64_t ab;
            std::memcpy(&ab, &inst[i].alpha, 8);
            if (seen.insert({inst[i].g, ab}).second) alphas_on[inst[i].g]++;
        }
    }
    auto start_for = [&](const pr_instance &in, const double **out) -> pr_status {
        *out = nullptr;
        if (opt.init == PR_INIT_UNIFORM || opt.init == PR_INIT_CHAIN) return PR_OK;   // chain: set per level below
        size_t bytes = (size_t)in.g->n * sizeof(double);
        if (opt.init == PR_INIT_USER) {
            const double *src = in.init_vec ? in.init_vec : opt.init_vec;
            if (opt.init_on_device) { *out = src; return PR_OK; }
            auto key = std::make_pair((const void *)in.g, (const void *)src);
            auto it = init_dev.find(key);
            if (it != init_dev.end()) { *out = it->second; return PR_OK; }
            bufs.emplace_back(new PoolBuf());
            pr_status a = bufs.back()->alloc(bytes, st);
            if (a != PR_OK) return a;
            PR_CUDA(cudaMemcpyAsync(bufs.back()->p, src, bytes, cudaMemcpyHostToDevice, st));
            *out = (const double *)bufs.back()->p;
            init_dev[key] = *out;
            return PR_OK;
        }
        uint64_t abits;
        std::memcpy(&abits, &in.alpha, 8);
        auto key = std::make_pair(in.g, abits);
        auto it = learned.find(key);
        if (it != learned.end()) { *out = it->second; return PR_OK; }
        if (opt.init == PR_INIT_AUTO) {
            // the learned start where its predicted saving exceeds its measured
            // cost: the network removes `gain` e-folds of the start's error, which
            // at the column's contraction rate (alpha scaled by the graph's
            // measured decay) saves gain / ln(1/rate) updates; an update saved on
            // a column whose launches other columns share is worth the launch
            // time less the latency they share. It costs the network once per
            // alpha and the features once per graph
            auto dit = auto_use.find(key);
            if (dit == auto_use.end()) {
                const double gain = pr_mlp_gain_value(opt.mlp);
                bool use = false;
                if (gain > 0.0 && in.alpha > 0.0) {
                    double t1 = 0.0, lat = 0.0, rho = 0.0, feat_us = 0.0, net_us = 0.0;
                    pr_status ps = pr_graph_pass_model(const_cast<pr_graph *>(in.g), st, &t1, &lat, &rho);
                    if (ps == PR_OK) ps = pr_learned_cost(opt.mlp, in.g, st, &feat_us, &net_us);
                    if (ps != PR_OK) return ps;
                    double rate = rho > 0.0 ? std::min(in.alpha, in.alpha * rho / 0.85) : in.alpha;
                    rate = std::min(std::max(rate, 1e-3), 1.0 - 1e-9);
                    const double per_update = alphas_on[in.g] > 1 ? std::max(t1 - lat, 0.05 * t1) : t1;
                    const double saved = gain / std::log(1.0 / rate) * per_update;
                    use = saved > net_us + feat_us / std::max(1, alphas_on[in.g]);
                }
                dit = auto_use.emplace(key, use).first;
            }
            if (!dit->second) return PR_OK;   // uniform start
        }
        // the features depend on the graph only: one pass per graph serves every alpha
        auto fit = learned_feat.find(in.g);
        if (fit == learned_feat.end()) {
            bufs.emplace_back(new PoolBuf());
            pr_status fs = bufs.back()->alloc(pr_learned_features_bytes(in.g), st);
            if (fs == PR_OK) fs = pr_learned_features(in.g, bufs.back()->p, st);
            if (fs != PR_OK) return fs;
            fit = learned_feat.emplace(in.g, bufs.back()->p).first;
        }
        bufs.emplace_back(new PoolBuf());
        pr_status ls = bufs.back()->alloc(bytes, st);
        if (ls != PR_OK) return ls;
        ls = pr_learned_start(opt.mlp, in.g, in.alpha, (double *)bufs.back()->p, true, st, fit->second);
        if (ls != PR_OK) return ls;
        *out = (const double *)bufs.back()->p;
        learned[key] = *out;
        return PR_OK;
    };
    // ---- columns: one per shared trajectory (graph, alpha, start), or one per instance
    SolveRequest req;
    req.precision = opt.precision;
    req.loop = opt.loop;
    req.switch_tol = opt.switch_tol;
    req.stream = st;
    req.max_passes = opt.max_passes;
    req.kernels = opt.kernels;
    req.persist_wait_us = opt.persist_wait_us;
    std::map<std::tuple<const pr_graph *, uint64_t, const double *>, int> col_of;
    std::vector<std::vector<std::pair<int, int>>> col_taps;   // (instance, tap index)
    for (int i : ok) {
        pr_instance &in = inst[i];
        const double *start = nullptr;
        s = start_for(in, &start);
        if (s != PR_OK) {
            in.status = s;
            if (first == PR_OK) { first = s; first_msg = pr_last_error(); }
            continue;
        }
        uint64_t abits;
        std::memcpy(&abits, &in.alpha, 8);
        auto key = std::make_tuple(in.g, abits, start);
        int c;
        auto it = col_of.find(key);
        if (opt.share_trajectories && it != col_of.end()) {
            c = it->second;
        } else {
            c = (int)req.cols.size();
            req.cols.emplace_back();
            SolveColumn &sc = req.cols.back();
            sc.g = in.g;
            sc.alpha = in.alpha;
            sc.init_dev = start;
            // learned starts come in relabelled order
            sc.learned = (opt.init == PR_INIT_LEARNED || opt.init == PR_INIT_AUTO) && start != nullptr;
            sc.init_relabelled = sc.learned;
            if (opt.share_trajectories) col_of[key] = c;
        }
        SolveColumn &sc = req.cols[c];
        Tap t{};
        t.tau = in.tol;
        t.norm = in.norm;
        t.max_iter = in.max_iter;
        t.alias_of = -1;
        t.out = opt.outputs_on_device ? in.ranks_out : nullptr;
        sc.taps.push_back(t);
        sc.inst.push_back(i);
        sc.host_dst.push_back(opt.outputs_on_device ? nullptr : in.ranks_out);
    }
    if (hist_host && req.cols.size() == 1) {
        req.cols[0].hist_host = hist_host;
        req.cols[0].hist_cap = hist_cap;
    }
    // ---- jobs: the grouping plan, one sub-solve per job precision and width
    std::vector<std::vector<Tap>> taps(req.cols.size());
    auto fail_all = [&](pr_status fs) {
        std::string msg = pr_last_error();
        for (auto &c : req.cols)
            for (int i : c.inst) inst[i].status = fs;
        return pr_fail(fs, msg);
    };
    // solves the columns `cols` of req (the whole request, or one level of an
    // alpha continuation) and adds the launch accounting to `total`
    auto run_columns = [&](const std::vector<int> &cols, SolveStats &total) -> pr_status {
        SolveRequest part;
        part.precision = req.precision;
        part.loop = req.loop;
        part.switch_tol = req.switch_tol;
        part.stream = req.stream;
        part.max_passes = req.max_passes;
        part.kernels = req.kernels;
        part.persist_wait_us = req.persist_wait_us;
        for (int c : cols) part.cols.push_back(req.cols[c]);
        std::vector<SubSolve> plan;
        pr_status ps = pr_plan_request(part, opt.group, plan);
        if (ps != PR_OK) return ps;
        for (const SubSolve &sp : plan) {
            SolveRequest sub;
            sub.precision = sp.precision;
            sub.loop = part.loop;
            sub.switch_tol = part.switch_tol;
            sub.stream = part.stream;
            sub.max_passes = part.max_passes;
            sub.kernels = part.kernels;
            sub.persist_wait_us = part.persist_wait_us;
            std::vector<int> cmap;   // sub-request column -> request column
            for (const auto &jc : sp.jobs) {
                std::vector<int> local;
                for (int c : jc) {
                    local.push_back((int)sub.cols.size());
                    cmap.push_back(cols[c]);
                    sub.cols.push_back(part.cols[c]);
                }
                sub.jobs.push_back(local);
            }
            std::vector<std::vector<Tap>> sub_taps;
            if ((ps = pr_run_solve(sub, sub_taps)) != PR_OK) return ps;
            for (size_t k = 0; k < cmap.size(); k++) taps[cmap[k]] = sub_taps[k];
            total.add(sub.stats);
        }
        return PR_OK;
    };
    if (!req.cols.empty()) {
        SolveStats total;
        if (opt.init != PR_INIT_CHAIN) {
            std::vector<int> all(req.cols.size());
            for (size_t c = 0; c < all.size(); c++) all[c] = (int)c;
            if ((s = run_columns(all, total)) != PR_OK) return fail_all(s);
        } else {
            // alpha continuation: per graph, columns in increasing alpha; level L
            // holds every graph's L-th column and starts it from the final
            // iterate of the graph's column at level L - 1
            std::vector<const pr_graph *> gorder;
            std::map<const pr_graph *, std::vector<int>> per_g;
            for (size_t c = 0; c < req.cols.size(); c++) {
                if (!per_g.count(req.cols[c].g)) gorder.push_back(req.cols[c].g);
                per_g[req.cols[c].g].push_back((int)c);
            }
            size_t levels = 0;
            for (auto &kv : per_g) {
                std::stable_sort(kv.second.begin(), kv.second.end(),
                                 [&](int a, int b) { return req.cols[a].alpha < req.cols[b].alpha; });
                levels = std::max(levels, kv.second.size());
            }
            std::vector<std::unique_ptr<PoolBuf>> finals(req.cols.size());
            for (size_t L = 0; L < levels; L++) {
                std::vector<int> lvl;
                for (const pr_graph *g : gorder) {
                    const auto &v = per_g[g];
                    if (L >= v.size()) continue;
                    const int c = v[L];
                    SolveColumn &sc = req.cols[c];
                    if (L > 0) {
                        sc.init_dev = static_cast<const double *>(finals[v[L - 1]]->p);
                        sc.init_relabelled = false;
                    }
                    if (L + 1 < v.size()) {
                        finals[c].reset(new PoolBuf());
                        if ((s = finals[c]->alloc((size_t)g->n * sizeof(double), st)) != PR_OK) return fail_all(s);
                        sc.final_dev = static_cast<double *>(finals[c]->p);
                    }
                    lvl.push_back(c);
                }
                if ((s = run_columns(lvl, total)) != PR_OK) return fail_all(s);
            }
        }
        pr_record_last_stats(total);
    }
    for (size_t c = 0; c < req.cols.size(); c++)
        for (size_t q = 0; q < req.cols[c].inst.size(); q++) {
            pr_instance &in = inst[req.cols[c].inst[q]];
            const Tap &t = taps[c][q];
            in.iters = t.iters;
            in.err = t.err;
            in.err_l1 = t.err_l1;
            in.converged = t.converged;
            in.status = PR_OK;
        }
    if (first != PR_OK) return pr_fail(first, first_msg);
    return PR_OK;
}

extern "C" pr_status pr_solve_batch(pr_instance *inst, int32_t count, const pr_options *opt) {
    return pr_solve_batch_ex(inst, count, opt, nullptr, 0);
}

extern "C" pr_status pr_solve(const pr_graph *g, double alpha, double tol, int32_t norm, int32_t max_iter,
                              const pr_options *opt, double *ranks_out, int32_t *iters_out, double *err_out,
                              int32_t *converged_out) {
    pr_instance in{};
    in.g = g;
    in.alpha = alpha;
    in.tol = tol;
    in.norm = norm;
    in.max_iter = max_iter;
    in.ranks_out = ranks_out;
    in.init_vec = nullptr;
    double *hist = opt ? opt->err_history : nullptr;
    pr_status s = pr_solve_batch_ex(&in, 1, opt, hist, max_iter);
    if (s != PR_OK) return s;
    if (iters_out) *iters_out = in.iters;
    if (err_out) *err_out = in.err;
    if (converged_out) *converged_out = in.converged;
    return PR_OK;
}
