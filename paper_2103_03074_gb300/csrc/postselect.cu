// Post-selection, conditional sampling and the probability histogram of an
// amplitude tensor over the open qubits ("Fidelity" paragraph, Fig. 2, and
// the appendix on conditional and marginal probabilities).
//
// Probabilities are p_i = re_i^2 + im_i^2 in FP64 with each product and the
// sum rounded separately (no fused multiply-add), so that a probability, the
// order of two probabilities and the bin of a scaled probability are the
// same numbers any FP64 evaluation of that formula gives.
//
// Sorting is a bitonic network on (probability bits, index) pairs: the
// stages whose partners lie within 2048 elements run in shared memory, the
// longer ones as one global pass each.  Non-negative doubles order like
// their bit patterns, so the keys are the raw 64-bit patterns.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "tn.h"
#include "tn_internal.h"

namespace tn {
namespace {

constexpr int kLocalBits = 11;  // 2048 elements per shared-memory chunk
constexpr int kLocal = 1 << kLocalBits;
constexpr int kScanBlock = 1024;

__device__ __forceinline__ double prob_of(double2 a) { return __dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y)); }

__global__ void keys_kernel(const double2 *amp, int64_t n, unsigned long long *key, uint32_t *val) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        key[i] = (unsigned long long)__double_as_longlong(prob_of(amp[i]));
        val[i] = (uint32_t)i;
    }
}

// compare-exchange of positions i < j for decreasing order within blocks of
// `size` whose (i & size) bit is 0, increasing where it is 1 (a bitonic merge
// step; the final merge has size = n, so the whole array ends decreasing)
__device__ __forceinline__ void cmpx(unsigned long long &ki, uint32_t &vi, unsigned long long &kj, uint32_t &vj,
                                     bool decreasing) {
    const bool swap = decreasing ? (ki < kj) : (ki > kj);
    if (swap) {
        const unsigned long long tk = ki;
        ki = kj;
        kj = tk;
        const uint32_t tv = vi;
        vi = vj;
        vj = tv;
    }
}

// all stages with stride < chunk: sizes from size_lo to size_hi (powers of
// two; size_lo = 2 sorts the chunk from scratch, size_lo = size_hi merges)
__global__ void __launch_bounds__(kLocal / 2) bitonic_local(unsigned long long *key, uint32_t *val, int64_t n,
                                                            int chunk_bits, int64_t size_lo, int64_t size_hi) {
    __shared__ unsigned long long sk[kLocal];
    __shared__ uint32_t sv[kLocal];
    const int chunk = 1 << chunk_bits;
    const int64_t base = (int64_t)blockIdx.x * chunk;
    for (int t = threadIdx.x; t < chunk; t += blockDim.x) {
        sk[t] = key[base + t];
        sv[t] = val[base + t];
    }
    __syncthreads();
    for (int64_t size = size_lo; size <= size_hi; size <<= 1) {
        int64_t stride = size >> 1;
        if (stride >= chunk) stride = chunk >> 1;
        for (; stride >= 1; stride >>= 1) {
            for (int t = threadIdx.x; t < chunk / 2; t += blockDim.x) {
                // t-th pair: i has a 0 at the stride bit
                const int lo = t & (int)(stride - 1);
                const int i = ((t - lo) << 1) | lo;
                const int j = i | (int)stride;
                const bool dec = ((base + i) & size) == 0;
                cmpx(sk[i], sv[i], sk[j], sv[j], dec);
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < chunk; t += blockDim.x) {
        key[base + t] = sk[t];
        val[base + t] = sv[t];
    }
}

// one stage with stride >= chunk, in global memory
__global__ void bitonic_global(unsigned long long *key, uint32_t *val, int64_t n, int64_t size, int64_t stride) {
    const int64_t pairs = n >> 1;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < pairs; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lo = t & (stride - 1);
        const int64_t i = ((t - lo) << 1) | lo;
        const int64_t j = i | stride;
        unsigned long long ki = key[i], kj = key[j];
        uint32_t vi = val[i], vj = val[j];
        cmpx(ki, vi, kj, vj, (i & size) == 0);
        key[i] = ki;
        key[j] = kj;
        val[i] = vi;
        val[j] = vj;
    }
}

// block sums of the probabilities in the order `key` holds them (sorted) or
// of the amplitude tensor in index order (key == nullptr)
__device__ __forceinline__ double value_at(const unsigned long long *key, const double2 *amp, int64_t i) {
    return key ? __longlong_as_double((long long)key[i]) : prob_of(amp[i]);
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[kScanBlock / 32];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) ws[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) s += ws[q];
    __syncthreads();
    return s;  // valid in thread 0
}

__global__ void __launch_bounds__(kScanBlock) block_sums_kernel(const unsigned long long *key, const double2 *amp,
                                                                int64_t n, double *sums) {
    const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    const double v = i < n ? value_at(key, amp, i) : 0.0;
    const double s = block_sum(v);
    if (threadIdx.x == 0) sums[blockIdx.x] = s;
}

// exclusive prefix of the block sums, in order, by one thread (a few
// thousand values; the order matches a left-to-right sum of the blocks)
__global__ void prefix_serial_kernel(double *sums, int64_t nb) {
    double run = 0.0;
    for (int64_t b = 0; b < nb; b++) {
        const double s = sums[b];
        sums[b] = run;
        run += s;
    }
    sums[nb] = run;
}

// F_j = 2^n / N_j * (sum of the first N_j sorted probabilities) - 1
__global__ void __launch_bounds__(kScanBlock) xeb_points_kernel(const unsigned long long *key, const double *prefix,
                                                                const int64_t *counts, int n_qubits, double *out) {
    const int64_t N = counts[blockIdx.x];
    const int64_t b = (N - 1) / kScanBlock;  // block holding the last selected element
    const int64_t i = b * kScanBlock + threadIdx.x;
    const double v = i < N ? __longlong_as_double((long long)key[i]) : 0.0;
    const double s = block_sum(v);
    if (threadIdx.x == 0) out[blockIdx.x] = ldexp(prefix[b] + s, n_qubits) / (double)N - 1.0;
}

// inclusive prefix within each block plus the block's exclusive prefix:
// cdf[i] = sum of p over indices <= i
__global__ void __launch_bounds__(kScanBlock) cdf_kernel(const double2 *amp, int64_t n, const double *prefix,
                                                         double *cdf) {
    __shared__ double s[kScanBlock];
    const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    s[threadIdx.x] = i < n ? prob_of(amp[i]) : 0.0;
    __syncthreads();
    // Hillis-Steele scan in shared memory
    for (int off = 1; off < kScanBlock; off <<= 1) {
        const double add = threadIdx.x >= (unsigned)off ? s[threadIdx.x - off] : 0.0;
        __syncthreads();
        s[threadIdx.x] += add;
        __syncthreads();
    }
    if (i < n) cdf[i] = prefix[blockIdx.x] + s[threadIdx.x];
}

// smallest i with cdf[i] > u * total
__global__ void sample_kernel(const double *cdf, int64_t n, const double *total, const double *u, int64_t m,
                              int64_t *out) {
    const double tot = *total;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const double t = u[j] * tot;
        int64_t lo = 0, hi = n - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (cdf[mid] > t) hi = mid;
            else lo = mid + 1;
        }
        out[j] = lo;
    }
}

__global__ void copy_order_kernel(const uint32_t *val, int64_t n, int64_t *order) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        order[i] = (int64_t)val[i];
}

// bin of x = p * scale: floor(x / width) for x < x_max, else the overflow bin
__global__ void hist_kernel(const double2 *amp, int64_t n, double scale, double x_max, int n_bins,
                            unsigned long long *counts) {
    extern __shared__ unsigned long long hs[];
    for (int b = threadIdx.x; b <= n_bins; b += blockDim.x) hs[b] = 0;
    __syncthreads();
    const double width = x_max / n_bins;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = __dmul_rn(prob_of(amp[i]), scale);
        int b = n_bins;
        if (x < x_max) {
            b = (int)(x / width);
            if (b >= n_bins) b = n_bins - 1;  // x just below x_max whose quotient rounds up
        }
        atomicAdd(&hs[b], 1ull);
    }
    __syncthreads();
    for (int b = threadIdx.x; b <= n_bins; b += blockDim.x)
        if (hs[b]) atomicAdd(&counts[b], hs[b]);
}

int grid_of(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return (int)g;
}

// device scratch of one call, allocated from the stream-ordered pool
struct Scratch {
    cudaStream_t s;
    std::vector<void *> ptrs;
    explicit Scratch(cudaStream_t st) : s(st) {}
    template <typename T>
    T *get(size_t count) {
        void *p = nullptr;
        if (cudaMallocAsync(&p, count * sizeof(T), s) != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return static_cast<T *>(p);
    }
    ~Scratch() {
        for (void *p : ptrs) cudaFreeAsync(p, s);
    }
};

int sort_desc(const double2 *amp, int64_t n, unsigned long long *key, uint32_t *val, cudaStream_t s) {
    keys_kernel<<<grid_of(n, 256), 256, 0, s>>>(amp, n, key, val);
    const int cb = n >= kLocal ? kLocalBits : __builtin_ctzll((unsigned long long)n);
    const int64_t chunk = (int64_t)1 << cb;
    const int64_t nchunks = n / chunk;
    if (chunk >= 2)
        bitonic_local<<<(unsigned)nchunks, (unsigned)(chunk / 2), 0, s>>>(key, val, n, cb, 2, chunk);
    for (int64_t size = chunk << 1; size <= n; size <<= 1) {
        for (int64_t stride = size >> 1; stride >= chunk; stride >>= 1)
            bitonic_global<<<grid_of(n / 2, 256), 256, 0, s>>>(key, val, n, size, stride);
        bitonic_local<<<(unsigned)nchunks, (unsigned)(chunk / 2), 0, s>>>(key, val, n, cb, size, size);
    }
    return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

}  // namespace
}  // namespace tn

using namespace tn;

extern "C" int tn_postselect_xeb(const double *d_amp, int n_open, int n_qubits, int n_points, const int64_t *counts,
                                 double *out_xeb, int64_t *d_order, tn_stream_t stream) {
    if (!d_amp || n_open < 0 || n_open > 31 || n_qubits < n_open || n_qubits > 1000 || n_points < 0 ||
        (n_points > 0 && (!counts || !out_xeb)))
        return fail(TN_ERR_ARG, "tn_postselect_xeb: bad arguments");
    const int64_t n = (int64_t)1 << n_open;
    for (int j = 0; j < n_points; j++)
        if (counts[j] < 1 || counts[j] > n) return fail(TN_ERR_ARG, "tn_postselect_xeb: counts must lie in [1, 2^n_open]");
    if (n_points > 65535) return fail(TN_ERR_ARG, "tn_postselect_xeb: at most 65535 points");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const double2 *amp = reinterpret_cast<const double2 *>(d_amp);
    int rc = TN_OK;
    {
        Scratch sc(s);
        const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
        unsigned long long *key = sc.get<unsigned long long>(n);
        uint32_t *val = sc.get<uint32_t>(n);
        double *prefix = sc.get<double>(nb + 1);
        int64_t *dcounts = sc.get<int64_t>(n_points > 0 ? n_points : 1);
        double *dout = sc.get<double>(n_points > 0 ? n_points : 1);
        if (!key || !val || !prefix || !dcounts || !dout) return fail(TN_ERR_OOM, "tn_postselect_xeb: scratch");
        if (sort_desc(amp, n, key, val, s) != TN_OK) return fail(TN_ERR_CUDA, "tn_postselect_xeb: sort launch");
        if (d_order) copy_order_kernel<<<grid_of(n, 256), 256, 0, s>>>(val, n, d_order);
        if (n_points > 0) {
            block_sums_kernel<<<(unsigned)nb, kScanBlock, 0, s>>>(key, nullptr, n, prefix);
            prefix_serial_kernel<<<1, 1, 0, s>>>(prefix, nb);
            cudaMemcpyAsync(dcounts, counts, sizeof(int64_t) * n_points, cudaMemcpyHostToDevice, s);
            xeb_points_kernel<<<(unsigned)n_points, kScanBlock, 0, s>>>(key, prefix, dcounts, n_qubits, dout);
            cudaMemcpyAsync(out_xeb, dout, sizeof(double) * n_points, cudaMemcpyDeviceToHost, s);
        }
        if (cudaGetLastError() != cudaSuccess) rc = fail(TN_ERR_CUDA, "tn_postselect_xeb: launch");
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(TN_ERR_CUDA, "tn_postselect_xeb: stream");
    return rc;
}

extern "C" int tn_conditional_sample(const double *d_amp, int n_open, int64_t n_samples, const double *d_u,
                                     int64_t *d_out, tn_stream_t stream) {
    if (!d_amp || n_open < 0 || n_open > 40 || n_samples < 0 || (n_samples > 0 && (!d_u || !d_out)))
        return fail(TN_ERR_ARG, "tn_conditional_sample: bad arguments");
    if (n_samples == 0) return TN_OK;
    const int64_t n = (int64_t)1 << n_open;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const double2 *amp = reinterpret_cast<const double2 *>(d_amp);
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    Scratch sc(s);
    double *prefix = sc.get<double>(nb + 1);
    double *cdf = sc.get<double>(n);
    if (!prefix || !cdf) return fail(TN_ERR_OOM, "tn_conditional_sample: scratch");
    block_sums_kernel<<<(unsigned)nb, kScanBlock, 0, s>>>(nullptr, amp, n, prefix);
    prefix_serial_kernel<<<1, 1, 0, s>>>(prefix, nb);
    cdf_kernel<<<(unsigned)nb, kScanBlock, 0, s>>>(amp, n, prefix, cdf);
    sample_kernel<<<grid_of(n_samples, 256), 256, 0, s>>>(cdf, n, prefix + nb, d_u, n_samples, d_out);
    if (cudaGetLastError() != cudaSuccess) return fail(TN_ERR_CUDA, "tn_conditional_sample: launch");
    return TN_OK;
}

extern "C" int tn_probability_histogram(const double *d_amp, int n_open, double scale, int n_bins, double x_max,
                                        int64_t *d_counts, tn_stream_t stream) {
    if (!d_amp || !d_counts || n_open < 0 || n_open > 40 || n_bins < 1 || n_bins > 4096 || !(x_max > 0.0) ||
        !(scale > 0.0))
        return fail(TN_ERR_ARG, "tn_probability_histogram: bad arguments");
    const int64_t n = (int64_t)1 << n_open;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_counts, 0, sizeof(int64_t) * (n_bins + 1), s) != cudaSuccess)
        return fail(TN_ERR_CUDA, "tn_probability_histogram: memset");
    hist_kernel<<<grid_of(n, 256), 256, sizeof(unsigned long long) * (n_bins + 1), s>>>(
        reinterpret_cast<const double2 *>(d_amp), n, scale, x_max, n_bins,
        reinterpret_cast<unsigned long long *>(d_counts));
    if (cudaGetLastError() != cudaSuccess) return fail(TN_ERR_CUDA, "tn_probability_histogram: launch");
    return TN_OK;
}
