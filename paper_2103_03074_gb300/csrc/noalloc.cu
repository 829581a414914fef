// Allocation-free split-precision complex GEMM.
//
// Some callers cannot allocate device memory at the point where they need a
// product: code running under an allocator owned by another framework with a
// fixed budget, real-time loops that must not call into the driver's
// allocator, or library code that is handed device buffers and nothing else.
// For them this entry point computes C = A B on the tensor cores (the TF32x3
// or BF16x3 split form of the library's GEMM) using only the buffers the
// caller passes plus one fixed scratch array that lives in this file as a
// __device__ variable: every GPU that loads the library holds that array
// (kScratchBytes) until the process exits, and no call here allocates or
// frees anything.
//
// The scratch holds the hi/lo planes of A and B.  Host code cannot use the
// array's name as a device address (it names a host-side shadow), so the
// first call on each device looks the address up with cudaGetSymbolAddress
// while that device is current and caches it.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "kernels.h"
#include "tc_gemm.h"
#include "tn_internal.h"

namespace tn {

namespace {

constexpr size_t kScratchBytes = 32ull << 20;  // 32 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// device address of the scratch array on the current device (looked up once)
int scratch_for_current_device(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(TN_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(TN_ERR_ARG, "device index beyond the supported range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(TN_ERR_CUDA, std::string("cudaGetSymbolAddress(noalloc scratch): ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return TN_OK;
}

bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }
int log2i(int64_t x) {
    int r = 0;
    while ((1ll << r) < x) r++;
    return r;
}

// Bit-permute arguments for one operand with row bits (rb) and k bits (kb):
// source layout is [rows][k] (row-major) or [k][rows] (k_major_src = false),
// destination is K-major planes [rows][k].  Tile = the source's and the
// destination's lowest bits (up to kTileMaxBits).
BitPermArgs split_args(const float2 *src, void *dst, int rb, int kb, bool src_row_major, int mode) {
    BitPermArgs a;
    std::memset(&a, 0, sizeof a);
    const int r = rb + kb;
    a.in = src;
    a.out = dst;
    a.rank = r;
    a.mode = mode;
    a.plane_stride = 1ll << r;
    // dest position p: k bits at 0..kb-1, row bits at kb..r-1
    int src_pos[kMaxRank];
    for (int p = 0; p < r; p++) {
        const bool is_k = p < kb;
        const int j = is_k ? p : p - kb;  // bit j of k or of row
        src_pos[p] = src_row_major ? (is_k ? j : kb + j) : (is_k ? rb + j : j);
    }
    int dst_of_src[kMaxRank];
    for (int p = 0; p < r; p++) dst_of_src[src_pos[p]] = p;
    const int nt = r < kTileMaxBits ? r : kTileMaxBits;
    bool in_tile[kMaxRank] = {false};
    int cnt = 0;
    for (int i = 0; i < r && cnt < nt; i++) {
        if (!in_tile[i]) { in_tile[i] = true; cnt++; }
        if (cnt < nt && !in_tile[dst_of_src[i]]) { in_tile[dst_of_src[i]] = true; cnt++; }
    }
    int tile[kTileMaxBits];
    for (int p = 0; p < r; p++) {
        if (in_tile[p]) tile[a.n_tile++] = p;
        else {
            a.rest_dst[a.n_rest] = p;
            a.rest_src[a.n_rest] = src_pos[p];
            a.n_rest++;
        }
    }
    for (int j = 0; j < a.n_tile; j++) a.tile_dst[j] = tile[j];
    // read order: tile bits by ascending source position
    int order[kTileMaxBits];
    for (int j = 0; j < a.n_tile; j++) order[j] = j;
    for (int i = 1; i < a.n_tile; i++)
        for (int j = i; j > 0 && src_pos[tile[order[j]]] < src_pos[tile[order[j - 1]]]; j--) {
            int t = order[j];
            order[j] = order[j - 1];
            order[j - 1] = t;
        }
    for (int j = 0; j < a.n_tile; j++) {
        a.rd_w[j] = order[j];
        a.rd_src[j] = src_pos[tile[order[j]]];
    }
    return a;
}

}  // namespace

}  // namespace tn

using namespace tn;

extern "C" int tn_gemm_split_noalloc(const float *d_A, const float *d_B, float *d_C, int64_t M, int64_t N,
                                     int64_t K, tn_form form, tn_stream_t stream) {
    if (!d_A || !d_B || !d_C) return fail(TN_ERR_ARG, "tn_gemm_split_noalloc: NULL buffer");
    if (form != TN_BF16X3 && form != TN_TF32X3)
        return fail(TN_ERR_ARG, "tn_gemm_split_noalloc: form must be TN_BF16X3 or TN_TF32X3");
    if (!is_pow2(M) || !is_pow2(N) || !is_pow2(K))
        return fail(TN_ERR_ARG, "tn_gemm_split_noalloc: M, N and K must be powers of two");
    if (M < 64 || N < 32 || K < 32)
        return fail(TN_ERR_ARG, "tn_gemm_split_noalloc: need M >= 64, N >= 32, K >= 32");
    const int es = tc_plane_bytes(form);
    const double need = 4.0 * (double)es * ((double)M + (double)N) * (double)K;
    if (need > (double)kScratchBytes)
        return fail(TN_ERR_ARG, "tn_gemm_split_noalloc: 4 * plane bytes * (M + N) * K = " +
                                    std::to_string((long long)need) + " bytes exceeds the " +
                                    std::to_string((long long)kScratchBytes) + "-byte scratch array");
    if (!tc_form_available(form)) return fail(TN_ERR_ARG, "tn_gemm_split_noalloc: tensor-core form not available");
    void *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned char *planesA = static_cast<unsigned char *>(scratch);
    unsigned char *planesB = planesA + (size_t)4 * es * M * K;  // 256-byte aligned: M K >= 2048
    const int mode = es == 2 ? 1 : 2;
    const int mb = log2i(M), nb = log2i(N), kb = log2i(K);
    // A [M][K] row-major -> planes [q][M][K]; B [K][N] row-major -> planes [q][N][K]
    BitPermArgs sa = split_args(reinterpret_cast<const float2 *>(d_A), planesA, mb, kb, true, mode);
    BitPermArgs sb = split_args(reinterpret_cast<const float2 *>(d_B), planesB, nb, kb, false, mode);
    cudaError_t e = launch_bitperm(sa, s);
    if (e == cudaSuccess) e = launch_bitperm(sb, s);
    if (e != cudaSuccess) return fail(TN_ERR_CUDA, std::string("tn_gemm_split_noalloc split: ") + cudaGetErrorString(e));
    TcGemm g;
    std::memset(&g, 0, sizeof g);
    g.a.H = 1;
    g.a.M = M;
    g.a.N = N;
    g.a.K = K;
    g.a.sCh = M * N;
    g.a.sCm = N;
    g.a.sCn = 1;
    g.a.C = reinterpret_cast<float2 *>(d_C);
    g.form = form;
    g.planesA = planesA;
    g.planesB = planesB;
    g.ksplit = tc_choose_ksplit(g.a, form);
    if (!tc_prepare(g)) return fail(TN_ERR_CUDA, "tn_gemm_split_noalloc: TMA descriptor encoding failed");
    e = launch_gemm_tc(g, s);
    if (e != cudaSuccess) return fail(TN_ERR_CUDA, std::string("tn_gemm_split_noalloc GEMM: ") + cudaGetErrorString(e));
    // The GEMM's pipeline waits are bounded; one that expires leaves C
    // partial and sets the library's device error word.  Read and clear the
    // word here (this synchronises the stream), so the caller learns of it
    // from this call and no later call reports it.
    if (tc_read_error(s) != 0)
        return fail(TN_ERR_TIMEOUT, "tn_gemm_split_noalloc: a bounded tensor-core pipeline wait expired");
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(TN_ERR_CUDA, std::string("tn_gemm_split_noalloc: ") + cudaGetErrorString(e));
    return TN_OK;
}
