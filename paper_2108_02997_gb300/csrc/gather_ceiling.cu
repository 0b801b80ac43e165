// gather_ceiling.cu — measurement probes behind bench.py's roofline record
// (libprceiling.so; not part of the PageRank library or its ABI).
//
// The one-column gather of a pass (Section 2's sum over in-edges of r_u/d_u)
// reads E random 8-byte contributions. How fast this GPU can serve such reads
// bounds the gather kernel more tightly than the copy bandwidth does, so the
// bench measures it on the same graph: the in-edge sources in the library's
// relabelled order (in-degree class descending, then out-degree class
// descending, ties by id; rows keep their sources' order), read edge-parallel
// with eight independent gathers per thread in flight and nothing else done
// with the values (they are folded with XOR so that no floating-point
// addition limits the rate):
//   [0] the index stream alone (4E bytes),
//   [1] the index stream and every gather through L1/L2,
//   [2] the same with the first `hub_values` contributions read from shared
//       memory (one 1024-thread CTA per SM), as the gather kernel does,
//   [3] uniform random gathers over a table of the graph's size (the L2's
//       random-sector rate, no reuse).
// Times are microseconds per launch (median of 10 after 3 warm-up launches,
// CUDA events). Buffers are allocated and freed by the call.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

namespace {

constexpr int kPer = 8;

__device__ __forceinline__ unsigned long long bits_of(double x) { return (unsigned long long)__double_as_longlong(x); }

__global__ void idx_only_kernel(const int32_t *__restrict__ idx, long long E, unsigned long long *out) {
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long nth = (long long)gridDim.x * blockDim.x;
    unsigned long long acc = 0;
    for (long long i = tid; i < E; i += nth) acc ^= (unsigned long long)__ldcs(idx + i);
    out[tid] = acc;
}

// hub_n = 0: every gather through L1/L2
__global__ void __launch_bounds__(1024) gather_kernel(const int32_t *__restrict__ idx, const double *__restrict__ c, long long E, int hub_n,
                              unsigned long long *out) {
    extern __shared__ __align__(16) unsigned char smem[];
    double *s_hub = reinterpret_cast<double *>(smem);
    for (int i = threadIdx.x; i < hub_n; i += blockDim.x) s_hub[i] = c[i];
    __syncthreads();
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long nth = (long long)gridDim.x * blockDim.x;
    unsigned long long acc = 0;
    for (long long base = tid; base < E; base += nth * kPer) {
        int u[kPer];
#pragma unroll
        for (int k = 0; k < kPer; k++) {
            const long long i = base + k * nth;
            u[k] = i < E ? __ldcs(idx + i) : -1;
        }
        double x[kPer];
#pragma unroll
        for (int k = 0; k < kPer; k++) x[k] = u[k] < 0 ? 0.0 : (u[k] < hub_n ? s_hub[u[k]] : __ldg(c + u[k]));
#pragma unroll
        for (int k = 0; k < kPer; k++) acc ^= bits_of(x[k]);
    }
    out[tid] = acc;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__global__ void uniform_idx_kernel(int32_t *idx, long long E, uint32_t n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < E; i += (long long)gridDim.x * blockDim.x)
        idx[i] = (int32_t)(((mix64((uint64_t)i * 0x9E3779B97F4A7C15ULL + 12345u) >> 32) * (uint64_t)n) >> 32);
}

int cls(int32_t d) {
    int c = 0;
    while (d) { c++; d >>= 1; }
    return c;
}

template <typename F>
cudaError_t median_us(F launch, double *us) {
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventCreate(&b)) != cudaSuccess) { cudaEventDestroy(a); return e; }
    for (int i = 0; i < 3; i++) launch();
    std::vector<float> t;
    for (int i = 0; i < 10 && e == cudaSuccess; i++) {
        cudaEventRecord(a);
        launch();
        cudaEventRecord(b);
        e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        t.push_back(ms);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    std::sort(t.begin(), t.end());
    *us = t.empty() ? 0.0 : 1e3 * (double)t[t.size() / 2];
    return e;
}

}  // namespace

// Returns 0, or a cudaError_t value, or -1 for bad arguments.
extern "C" int prc_gather_ceiling(int32_t n, int64_t nnz, const int32_t *off, const int32_t *src, const int32_t *outdeg,
                                  int32_t hub_values, double *us_out) {
    if (n < 1 || nnz < 1 || !off || !src || !outdeg || !us_out || hub_values < 0 || hub_values > 24576) return -1;
    for (int32_t v = 0; v < n; v++)
        if (off[v] > off[v + 1] || outdeg[v] < 0) return -1;
    if (off[0] != 0 || off[n] != nnz) return -1;
    // relabelled order: stable counting sort by (in-class desc, out-class desc)
    std::vector<int32_t> key(n), perm(n), inv(n);
    std::vector<int64_t> cnt(33 * 33 + 1, 0);
    for (int32_t v = 0; v < n; v++) {
        key[v] = (32 - cls(off[v + 1] - off[v])) * 33 + (32 - cls(outdeg[v]));
        cnt[key[v] + 1]++;
    }
    for (int k = 0; k < 33 * 33; k++) cnt[k + 1] += cnt[k];
    for (int32_t v = 0; v < n; v++) perm[cnt[key[v]]++] = v;
    for (int32_t i = 0; i < n; i++) inv[perm[i]] = i;
    std::vector<int32_t> idx(nnz);
    int64_t at = 0;
    for (int32_t i = 0; i < n; i++) {
        const int32_t v = perm[i];
        for (int32_t e = off[v]; e < off[v + 1]; e++) {
            const int32_t u = src[e];
            if (u < 0 || u >= n) return -1;
            idx[at++] = inv[u];
        }
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    const int hub_n = std::min<int32_t>(hub_values, n);
    int32_t *d_idx = nullptr, *d_uni = nullptr;
    double *d_c = nullptr;
    unsigned long long *d_out = nullptr;
    const size_t nout = (size_t)sms * 2048;
    e = cudaMalloc(&d_idx, sizeof(int32_t) * (size_t)nnz);
    if (e == cudaSuccess) e = cudaMalloc(&d_uni, sizeof(int32_t) * (size_t)nnz);
    if (e == cudaSuccess) e = cudaMalloc(&d_c, sizeof(double) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&d_out, sizeof(unsigned long long) * nout);
    if (e == cudaSuccess) e = cudaMemcpy(d_idx, idx.data(), sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(d_c, 0, sizeof(double) * (size_t)n);
    const long long E = nnz;
    int occ_i = 0, occ_g = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_i, idx_only_kernel, 256, 0);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(gather_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_g, gather_kernel, 256, 0);
    const size_t hub_bytes = sizeof(double) * (size_t)hub_n;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gather_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(hub_bytes, 1));
    // grids: at most sms * 2048 threads, matching d_out
    if (e == cudaSuccess)
        e = median_us([&] { idx_only_kernel<<<sms * std::max(1, std::min(occ_i, 8)), 256>>>(d_idx, E, d_out); }, &us_out[0]);
    if (e == cudaSuccess)
        e = median_us([&] { gather_kernel<<<sms * std::max(1, std::min(occ_g, 8)), 256>>>(d_idx, d_c, E, 0, d_out); },
                      &us_out[1]);
    if (e == cudaSuccess)
        e = median_us([&] { gather_kernel<<<sms, 1024, hub_bytes>>>(d_idx, d_c, E, hub_n, d_out); }, &us_out[2]);
    if (e == cudaSuccess) {
        uniform_idx_kernel<<<sms * 8, 256>>>(d_uni, E, (uint32_t)n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = median_us([&] { gather_kernel<<<sms * std::max(1, std::min(occ_g, 8)), 256>>>(d_uni, d_c, E, 0, d_out); },
                      &us_out[3]);
    cudaFree(d_idx);
    cudaFree(d_uni);
    cudaFree(d_c);
    cudaFree(d_out);
    return (int)e;
}
