// pr_noalloc.cu — pr_solve_noalloc: a single-instance solve that allocates no
// memory. Its working set lives in one file-scope device array of fixed size.
//
// Some callers cannot let a library call cudaMalloc: a process whose device
// memory is owned by its own pool or caching allocator (a cudaMalloc outside
// the pool can fail or fragment it), a service running under a fixed memory
// budget, or a latency-critical loop where cudaMalloc/cudaFree would add an
// implicit device synchronisation. This entry point serves them: the caller
// passes the graph (already on the device) and the output buffer, and the
// iterates, contributions, per-CTA partials and loop state use the array
// below instead of fresh allocations.
//
// The array is g_noalloc_scratch. In host code that name is only a host-side
// stand-in for the device variable, so its device address is obtained with
// cudaGetSymbolAddress once per device (with that device current) and passed
// to the kernels. Every GPU that loads this library holds the array until the
// process exits. The address is kept for the life of the process: after a
// cudaDeviceReset of a device the library has used, it is stale (the kernel
// setup records of the other entry points have the same limit).
#include <cstring>
#include <mutex>

#include "pr_kernels.cuh"

namespace {

constexpr size_t kNoAllocBytes = size_t(40) << 20;   // 40 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up on the
// first call per device).
pr_status noalloc_scratch(void **out) {
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return pr_fail(PR_ENOTSUP, "device ordinal out of range for the no-alloc scratch table");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return pr_cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return PR_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" pr_status pr_solve_noalloc(const pr_graph *g, double alpha, double tol, int32_t norm, int32_t max_iter,
                                      double *d_ranks_out, void *stream, int32_t *iters_out, double *err_out,
                                      int32_t *converged_out) {
    pr_clear_error();
    if (!pr_graph_valid(g)) return pr_fail(PR_ESTATE, "not a live graph handle");
    if (!(alpha >= 0.0 && alpha <= 1.0)) return pr_fail(PR_EINVAL, "alpha must be in [0, 1]");
    if (!(tol > 0.0) || !std::isfinite(tol)) return pr_fail(PR_EINVAL, "tol must be positive and finite");
    if (norm < PR_NORM_L1 || norm > PR_NORM_LINF) return pr_fail(PR_EINVAL, "norm must be 1 (L1), 2 (L2) or 3 (Linf)");
    if (max_iter < 1) return pr_fail(PR_EINVAL, "max_iter must be >= 1");
    if (!d_ranks_out) return pr_fail(PR_EINVAL, "d_ranks_out is NULL");
    int dev = 0;
    PR_CUDA(cudaGetDevice(&dev));
    if (dev != g->device)
        return pr_fail(PR_EINVAL, "the graph lives on device " + std::to_string(g->device) + " but device " +
                                      std::to_string(dev) + " is current");
    {
        // the kernels write d_ranks_out: it must be device memory of this GPU
        // (cudaPointerGetAttributes allocates nothing)
        cudaPointerAttributes pa;
        cudaError_t e = cudaPointerGetAttributes(&pa, d_ranks_out);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return pr_fail(PR_EINVAL, "d_ranks_out is not a device pointer");
        }
        if ((pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) || pa.device != dev)
            return pr_fail(PR_EINVAL, "d_ranks_out must be device memory of the current device");
    }
    const TileTable &ut = g->tables[0];
    if (!ut.d_tiles) return pr_fail(PR_ESTATE, "graph has no single-column work table");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    void *kiter = pr_iter_kernel_for(PR_PREC_DF64, 1);
    void *kinit = pr_init_kernel_for(PR_PREC_DF64, 1);
    const size_t smem = pr_tile_smem_bytes(PR_PREC_DF64, 1);
    int sms = 0, occ = 1;
    PR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    pr_status s = pr_kernel_setup(PR_PREC_DF64, 1, &occ);
    if (s != PR_OK) return s;
    // the grid of pr_solve's one-column fused pass
    const int ctas = std::max(1, std::min(sms * occ, tile_ctas(ut.ntiles)));
    // ---- layout inside the scratch array
    const size_t n = (size_t)g->n;
    size_t at = 0;
    const size_t o_job = at; at = align256(at + sizeof(JobDev));
    const size_t o_glob = at; at = align256(at + sizeof(GlobalDev));
    const size_t o_cols = at; at = align256(at + sizeof(ColState));
    const size_t o_tap = at; at = align256(at + sizeof(Tap));
    const size_t o_ctajob = at; at = align256(at + sizeof(int32_t) * ctas);
    const size_t o_part = at; at = align256(at + sizeof(double) * kPartials * ctas);
    const size_t o_cp = at; at = align256(at + sizeof(df64) * std::max(ut.n_chunk_slots, 1));
    const size_t o_cnt = at; at = align256(at + sizeof(uint32_t) * std::max(ut.n_long, 1));
    size_t o_vec[4];
    for (int b = 0; b < 4; b++) { o_vec[b] = at; at = align256(at + sizeof(df64) * (n + kPad)); }
    if (at > kNoAllocBytes)
        return pr_fail(PR_EINVAL, "graph needs " + std::to_string(at) + " bytes of working memory; the no-alloc scratch holds " +
                                      std::to_string(kNoAllocBytes) + " (about 32 bytes per vertex: n <= ~1.2 million)");
    void *base_v = nullptr;
    s = noalloc_scratch(&base_v);
    if (s != PR_OK) return s;
    char *base = static_cast<char *>(base_v);
    // ---- state (host structures copied into the scratch array)
    JobDev job;
    std::memset(&job, 0, sizeof(job));
    job.off = g->d_off;
    job.src = g->d_src;
    job.outdeg = g->d_outdeg;
    job.perm = g->d_perm;
    job.tiles = ut.d_tiles;
    job.slot_base = ut.d_slot_base;
    job.n = g->n;
    job.ntiles = ut.ntiles;
    job.cur = 0;
    job.cta_begin = 0;
    job.cta_count = ctas;
    job.ncols = 1;
    job.alive = 1;
    job.r[0] = base + o_vec[0];
    job.r[1] = base + o_vec[1];
    job.contrib[0] = base + o_vec[2];
    job.contrib[1] = base + o_vec[3];
    job.chunk_part = base + o_cp;
    job.chunk_cnt = reinterpret_cast<uint32_t *>(base + o_cnt);
    job.cta_part = reinterpret_cast<double *>(base + o_part);
    job.cols = reinterpret_cast<ColState *>(base + o_cols);
    job.taps = reinterpret_cast<Tap *>(base + o_tap);
    ColState cs;
    std::memset(&cs, 0, sizeof(cs));
    cs.alpha = alpha;
    cs.c0_base = (1.0 - alpha) / (double)g->n;
    cs.c0_coef = alpha / (double)g->n;
    df64 a = df_from_double(alpha), u = df_from_double(1.0 / (double)g->n);
    std::memcpy(cs.v_alpha, &a, sizeof(a));
    std::memcpy(cs.v_c0, &u, sizeof(u));   // init pass reads the uniform start here
    cs.active = 1;
    cs.tap_begin = 0;
    cs.tap_end = 1;
    cs.init_col_stride = 1;
    Tap tap;
    std::memset(&tap, 0, sizeof(tap));
    tap.tau = tol;
    tap.norm = norm;
    tap.max_iter = max_iter;
    tap.alias_of = -1;
    tap.out = d_ranks_out;
    GlobalDev glob;
    std::memset(&glob, 0, sizeof(glob));
    glob.njobs = 1;
    glob.pass_cap = max_iter + 3;
    PR_CUDA(cudaMemcpyAsync(base + o_job, &job, sizeof(job), cudaMemcpyHostToDevice, st));
    PR_CUDA(cudaMemcpyAsync(base + o_glob, &glob, sizeof(glob), cudaMemcpyHostToDevice, st));
    PR_CUDA(cudaMemcpyAsync(base + o_cols, &cs, sizeof(cs), cudaMemcpyHostToDevice, st));
    PR_CUDA(cudaMemcpyAsync(base + o_tap, &tap, sizeof(tap), cudaMemcpyHostToDevice, st));
    // every CTA belongs to job 0; the scratch keeps the previous call's bytes,
    // so everything that must start at zero is cleared here
    PR_CUDA(cudaMemsetAsync(base + o_ctajob, 0, sizeof(int32_t) * ctas, st));
    PR_CUDA(cudaMemsetAsync(base + o_cnt, 0, sizeof(uint32_t) * std::max(ut.n_long, 1), st));
    JobDev *d_job = reinterpret_cast<JobDev *>(base + o_job);
    GlobalDev *d_glob = reinterpret_cast<GlobalDev *>(base + o_glob);
    const int32_t *d_ctajob = reinterpret_cast<const int32_t *>(base + o_ctajob);
    void *args[] = {(void *)&d_job, (void *)&d_glob, (void *)&d_ctajob};
    PR_CUDA(cudaLaunchKernel(kinit, dim3(ctas), dim3(kBlock), args, 0, st));
    GlobalDev back;
    std::memset(&back, 0, sizeof(back));
    for (int p = 0; p < glob.pass_cap + 1; p++) {
        PR_CUDA(cudaLaunchKernel(kiter, dim3(ctas), dim3(kBlock), args, smem, st));
        PR_CUDA(cudaMemcpyAsync(&back, d_glob, sizeof(back), cudaMemcpyDeviceToHost, st));
        PR_CUDA(cudaStreamSynchronize(st));
        if (!back.alive || back.error) break;
    }
    if (back.error || back.alive) return pr_fail(PR_ETIMEOUT, "device loop did not finish within its pass cap");
    Tap out;
    PR_CUDA(cudaMemcpyAsync(&out, base + o_tap, sizeof(out), cudaMemcpyDeviceToHost, st));
    PR_CUDA(cudaStreamSynchronize(st));
    if (!out.fired) return pr_fail(PR_ETIMEOUT, "the stopping rule never fired");
    if (iters_out) *iters_out = out.iters;
    if (err_out) *err_out = out.err;
    if (converged_out) *converged_out = out.converged;
    return PR_OK;
}
