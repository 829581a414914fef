// CUDA kernels of the plain FP32 form of the sliced contraction, plus the
// slice extraction, cross-slice FP64 sum and probability/XEB reductions.
//
// Every tensor has bond dimension 2 on every axis, so an element address is a
// bit string: each label owns one bit position.  Index maps are therefore bit
// scatters and gathers, computed in registers.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "kernels.h"

namespace tn {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 152 * 16;  // grid-stride cap: 16 resident CTAs x 152 SMs

__device__ __forceinline__ uint64_t insert_zeros(uint64_t x, const int *pos, int n) {
    // pos ascending, in final coordinates
    for (int i = 0; i < n; i++) {
        int p = pos[i];
        uint64_t lo = x & ((1ull << p) - 1);
        x = ((x >> p) << (p + 1)) | lo;
    }
    return x;
}

__device__ __forceinline__ uint64_t scatter_bits(uint64_t v, const int *pos, int n) {
    uint64_t r = 0;
    for (int j = 0; j < n; j++) r |= ((v >> j) & 1ull) << pos[j];
    return r;
}

__device__ __forceinline__ uint32_t gather_bits(uint64_t v, const int *bit, int n) {
    uint32_t r = 0;
    for (int j = 0; j < n; j++) r |= (uint32_t)((v >> bit[j]) & 1ull) << j;
    return r;
}

__device__ __forceinline__ void cfma(float2 &acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}

// One atomic max per warp of the per-thread maxima mx (non-negative floats
// order like their bit patterns); every lane of the warp calls it.
__device__ __forceinline__ void publish_max(unsigned *slot, float mx) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) atomicMax(slot, __float_as_uint(mx));
}

__device__ __forceinline__ float absmax2(float m, float2 v) { return fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y))); }

int grid_for(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    if (b > kMaxBlocks) b = kMaxBlocks;
    return (int)b;
}

// ---------------------------------------------------------------- small step
// Work item = (row r, chunk of NC outputs n).  Rows vary fastest, so the
// threads of a warp read and write consecutive addresses where T's and C's
// low bits are row bits, and read the same S values (shared-memory
// broadcast).  One chunk covers all outputs up to N = 32, so T is read once.
// rows is a power of two: index arithmetic uses masks and shifts.
template <int NC>
__global__ void __launch_bounds__(kThreads) small_kernel(const SmallArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int KS = 1 << a.nK, NS = 1 << a.nN, HS = 1 << a.nH;
    const int SS = HS * KS * NS;
    float2 *S_sm = reinterpret_cast<float2 *>(smem);
    // offsets of the k and n bits in T and C: 64-bit (a tensor of more than
    // 2^32 elements has K or N bits at positions >= 32)
    uint64_t *offT = reinterpret_cast<uint64_t *>(S_sm + SS);
    uint64_t *offC = offT + KS;
    for (int idx = threadIdx.x; idx < SS; idx += blockDim.x) {
        uint32_t n = idx & (NS - 1), k = (idx >> a.nN) & (KS - 1), h = idx >> (a.nN + a.nK);
        uint64_t addr = scatter_bits(h, a.hposS, a.nH) | scatter_bits(k, a.kposS, a.nK) |
                        scatter_bits(n, a.nposS, a.nN);
        S_sm[idx] = a.S[addr];
    }
    for (int k = threadIdx.x; k < KS; k += blockDim.x) offT[k] = scatter_bits(k, a.kposT, a.nK);
    for (int n = threadIdx.x; n < NS; n += blockDim.x) offC[n] = scatter_bits(n, a.nposC, a.nN);
    __syncthreads();
    const int nc = NS < NC ? NS : NC;  // outputs per item
    constexpr int kNcBits = NC == 32 ? 5 : (NC == 16 ? 4 : 3);
    const int chunk_bits = a.nN > kNcBits ? a.nN - kNcBits : 0;
    const int rbits = a.row_bits;
    const int64_t items = a.rows << chunk_bits;
    float mx = 0.f;  // of the values stored (max_slot)
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < items; w += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = w & (a.rows - 1);
        const int n0 = (int)(w >> rbits) * NC;
        const uint64_t tb = insert_zeros((uint64_t)r, a.tins, a.n_tins);
        const uint64_t cb = insert_zeros((uint64_t)r, a.cins, a.n_cins);
        const uint32_t h = gather_bits((uint64_t)r, a.hbitR, a.nH);
        const float2 *Sh = S_sm + (size_t)h * KS * NS + n0;
        float2 acc[NC];
#pragma unroll
        for (int j = 0; j < NC; j++) acc[j] = make_float2(0.f, 0.f);
        // T in batches of 4 values (independent loads in flight; larger
        // batches cost occupancy with 32 outputs per item), S pairs
        // read as 16-byte broadcasts
        for (int k0 = 0; k0 < KS; k0 += 4) {
            float2 t[4];
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (k0 + k < KS) t[k] = a.T[tb + offT[k0 + k]];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (k0 + k < KS) {
                    const float2 *Sk = Sh + (k0 + k) * NS;
                    if (NC >= 2 && nc == NC) {
#pragma unroll
                        for (int j = 0; j < NC; j += 2) {
                            const float4 s2 = *reinterpret_cast<const float4 *>(Sk + j);
                            cfma(acc[j], t[k], make_float2(s2.x, s2.y));
                            cfma(acc[j + 1], t[k], make_float2(s2.z, s2.w));
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < NC; j++)
                            if (j < nc) cfma(acc[j], t[k], Sk[j]);
                    }
                }
            }
        }
#pragma unroll
        for (int j = 0; j < NC; j++)
            if (j < nc) {
                a.C[cb + offC[n0 + j]] = acc[j];
                mx = absmax2(mx, acc[j]);
            }
    }
    if (a.max_slot) publish_max(a.max_slot, mx);
}

// ------------------------------------ small steps as tasks of one launch
// The small steps near the leaves of a contraction tree touch a few thousand
// elements each: as separate launches each costs several microseconds of
// launch and drain for well under a microsecond of work.  Here they are the
// tasks of one persistent launch.  Blocks claim units (up to kTaskUnitItems
// items of one task) in task order from an atomic counter; a unit first
// waits until the tasks it reads from have finished all their units, then
// stages its task's S in shared memory and computes its items as
// small_kernel does.  Tasks are listed producers first and a block claims
// its next unit only after finishing the current one, so every unit that a
// waiting block depends on is held by a block that is running: the waits
// end.  They are bounded all the same (task_error, then the unit is skipped).
__device__ int task_error = 0;
constexpr uint32_t kTaskSpinLimit = 1u << 21;

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t insert_zeros8(uint64_t x, const int8_t *pos, int n) {
    for (int i = 0; i < n; i++) {
        const int p = pos[i];
        x = ((x >> p) << (p + 1)) | (x & ((1ull << p) - 1));
    }
    return x;
}

__device__ __forceinline__ uint64_t scatter_bits8(uint64_t v, const int8_t *pos, int n) {
    uint64_t r = 0;
    for (int j = 0; j < n; j++) r |= ((v >> j) & 1ull) << pos[j];
    return r;
}

// items [w0, w1) of task t; S staged at S_sm[h][k][n]; inputs are read
// through L2 (ld.global.cg): a producer of this launch wrote them from
// another SM, and this SM's L1 may hold older lines of the same arena bytes
template <int NC>
__device__ __forceinline__ void task_items(const SmallTask &t, const float2 *S_sm, const uint64_t *offT,
                                           const uint64_t *offC, int64_t w0, int64_t w1) {
    const int KS = 1 << t.nK, NS = 1 << t.nN;
    const int nc = NS < NC ? NS : NC;
    for (int64_t w = w0 + threadIdx.x; w < w1; w += blockDim.x) {
        const int64_t r = w & (t.rows - 1);
        const int n0 = (int)(w >> t.row_bits) * NC;
        const uint64_t tb = insert_zeros8((uint64_t)r, t.tins, t.n_tins);
        const uint64_t cb = insert_zeros8((uint64_t)r, t.cins, t.n_cins);
        uint32_t h = 0;
        for (int j = 0; j < t.nH; j++) h |= (uint32_t)((r >> t.hbitR[j]) & 1) << j;
        const float2 *Sh = S_sm + (size_t)h * KS * NS + n0;
        float2 acc[NC];
#pragma unroll
        for (int j = 0; j < NC; j++) acc[j] = make_float2(0.f, 0.f);
        for (int k = 0; k < KS; k++) {
            const float2 tv = __ldcg(t.T + tb + offT[k]);
            const float2 *Sk = Sh + k * NS;
#pragma unroll
            for (int j = 0; j < NC; j++)
                if (j < nc) cfma(acc[j], tv, Sk[j]);
        }
#pragma unroll
        for (int j = 0; j < NC; j++)
            if (j < nc) t.C[cb + offC[n0 + j]] = acc[j];
    }
}

__global__ void __launch_bounds__(kThreads, 2)
    small_task_kernel(const SmallTask *__restrict__ tasks, const int *__restrict__ unit_task, int total_units,
                      int *ctr) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(16) SmallTask st;
    __shared__ int s_unit, s_ok;
    static_assert(sizeof(SmallTask) % 4 == 0, "task copied as words");
    for (;;) {
        if (threadIdx.x == 0) s_unit = atomicAdd(&ctr[0], 1);
        __syncthreads();
        const int u = s_unit;
        if (u >= total_units) break;
        const int ti = unit_task[u];
        {
            const int *src = reinterpret_cast<const int *>(tasks + ti);
            int *dst = reinterpret_cast<int *>(&st);
            for (int q = threadIdx.x; q < (int)(sizeof(SmallTask) / 4); q += blockDim.x) dst[q] = src[q];
        }
        if (threadIdx.x == 0) {
            // wait (bounded) for the producing tasks; acquire pairs with
            // their release below
            int ok = 1;
            const SmallTask &mine = tasks[ti];
            for (int d = 0; d < mine.n_deps && ok; d++) {
                const int dj = mine.dep[d];
                const int need = tasks[dj].n_units;
                for (uint32_t it = 0; ld_acquire_gpu(&ctr[1 + dj]) < need; it++) {
                    if (it >= kTaskSpinLimit ||
                        ((it & 1023u) == 1023u && *reinterpret_cast<volatile int *>(&task_error) != 0)) {
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            if (!ok) atomicExch(&task_error, 1);
            s_ok = ok;
        }
        __syncthreads();
        if (s_ok) {
            const int KS = 1 << st.nK, NS = 1 << st.nN, HS = 1 << st.nH;
            const int SS = HS * KS * NS;
            float2 *S_sm = reinterpret_cast<float2 *>(smem);
            uint64_t *offT = reinterpret_cast<uint64_t *>(S_sm + SS);
            uint64_t *offC = offT + KS;
            for (int idx = threadIdx.x; idx < SS; idx += blockDim.x) {
                const uint32_t n = idx & (NS - 1), k = (idx >> st.nN) & (KS - 1), h = idx >> (st.nN + st.nK);
                const uint64_t addr = scatter_bits8(h, st.hposS, st.nH) | scatter_bits8(k, st.kposS, st.nK) |
                                      scatter_bits8(n, st.nposS, st.nN);
                S_sm[idx] = __ldcg(st.S + addr);
            }
            for (int k = threadIdx.x; k < KS; k += blockDim.x) offT[k] = scatter_bits8(k, st.kposT, st.nK);
            for (int n = threadIdx.x; n < NS; n += blockDim.x) offC[n] = scatter_bits8(n, st.nposC, st.nN);
            __syncthreads();
            const int nc_bits = st.nc == 32 ? 5 : (st.nc == 16 ? 4 : 3);
            const int chunk_bits = st.nN > nc_bits ? st.nN - nc_bits : 0;
            const int64_t items = st.rows << chunk_bits;
            const int64_t w0 = (int64_t)(u - st.first_unit) * kTaskUnitItems;
            const int64_t w1 = w0 + kTaskUnitItems < items ? w0 + kTaskUnitItems : items;
            if (st.nc == 8) task_items<8>(st, S_sm, offT, offC, w0, w1);
            else if (st.nc == 16) task_items<16>(st, S_sm, offT, offC, w0, w1);
            else task_items<32>(st, S_sm, offT, offC, w0, w1);
        }
        // every thread's stores of this unit, then one release per unit
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&ctr[1 + ti], 1);
        }
    }
}

// ------------------------------------------------- small step, K per warp
// For steps with a long K (>= 32) and too few (row, output chunk) items to
// fill the GPU with one thread per item: one warp per item, lanes taking
// k = lane, lane + 32, ...; the partial sums are combined by warp shuffles
// and lane j stores output j.
template <int NC>
__global__ void __launch_bounds__(kThreads) small_ksplit_kernel(const SmallArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int KS = 1 << a.nK, NS = 1 << a.nN, HS = 1 << a.nH;
    const int SS = HS * KS * NS;
    float2 *S_sm = reinterpret_cast<float2 *>(smem);
    // offsets of the k and n bits in T and C: 64-bit (a tensor of more than
    // 2^32 elements has K or N bits at positions >= 32)
    uint64_t *offT = reinterpret_cast<uint64_t *>(S_sm + SS);
    uint64_t *offC = offT + KS;
    for (int idx = threadIdx.x; idx < SS; idx += blockDim.x) {
        uint32_t n = idx & (NS - 1), k = (idx >> a.nN) & (KS - 1), h = idx >> (a.nN + a.nK);
        uint64_t addr = scatter_bits(h, a.hposS, a.nH) | scatter_bits(k, a.kposS, a.nK) |
                        scatter_bits(n, a.nposS, a.nN);
        S_sm[idx] = a.S[addr];
    }
    for (int k = threadIdx.x; k < KS; k += blockDim.x) offT[k] = scatter_bits(k, a.kposT, a.nK);
    for (int n = threadIdx.x; n < NS; n += blockDim.x) offC[n] = scatter_bits(n, a.nposC, a.nN);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int nc = NS < NC ? NS : NC;
    constexpr int kNcBits = NC == 32 ? 5 : (NC == 16 ? 4 : 3);
    const int chunk_bits = a.nN > kNcBits ? a.nN - kNcBits : 0;
    const int rbits = a.row_bits;
    const int64_t items = a.rows << chunk_bits;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float mx = 0.f;  // of the values stored (max_slot)
    for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < items; w += warps) {
        const int64_t r = w & (a.rows - 1);
        const int n0 = (int)(w >> rbits) * NC;
        const uint64_t tb = insert_zeros((uint64_t)r, a.tins, a.n_tins);
        const uint64_t cb = insert_zeros((uint64_t)r, a.cins, a.n_cins);
        const uint32_t h = gather_bits((uint64_t)r, a.hbitR, a.nH);
        const float2 *Sh = S_sm + (size_t)h * KS * NS + n0;
        float2 acc[NC];
#pragma unroll
        for (int j = 0; j < NC; j++) acc[j] = make_float2(0.f, 0.f);
        for (int k = lane; k < KS; k += 32) {
            const float2 t = a.T[tb + offT[k]];
            const float2 *Sk = Sh + k * NS;
#pragma unroll
            for (int j = 0; j < NC; j++)
                if (j < nc) cfma(acc[j], t, Sk[j]);
        }
        float2 mine = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < NC; j++) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                acc[j].x += __shfl_xor_sync(0xffffffffu, acc[j].x, off);
                acc[j].y += __shfl_xor_sync(0xffffffffu, acc[j].y, off);
            }
            if (lane == j) mine = acc[j];
        }
        if (lane < nc) {
            a.C[cb + offC[n0 + lane]] = mine;
            mx = absmax2(mx, mine);
        }
    }
    if (a.max_slot) publish_max(a.max_slot, mx);
}

// ------------------------------------------------------ small step, tiled
// For steps whose K and N are both 4..32 wide and whose T has many rows:
// a CTA walks tiles of 2^tb consecutive rows.  The tile's T values (a few
// contiguous runs) are copied with cp.async into shared memory as [k][row],
// two tiles deep, so the next tile's copies are in flight while this one is
// multiplied and stored; each thread forms an RPT x NPT block of outputs
// (RPT rows, NPT consecutive n), reading RPT T values and NPT S values per k
// (4 FMAs per complex MAC against (RPT + NPT / 2) / (RPT * NPT) shared-memory
// loads); the outputs go through shared memory as [n][row] and out in C's
// own contiguous runs.  S sits in shared memory whole, as in the row
// kernel; the tile's h is constant (its bits lie above the tile).
__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ uint32_t smem_u32_k(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// rows per tile of the tiled small-step kernel: 1024 / N row groups of
// RPT rows, RPT the largest of 4, 2, 1 whose shared memory (two T stages,
// plus the C tile unless outputs are stored from registers) fits in 72 KB
__host__ __device__ constexpr int small_tile_rpt(int KS, int NS, bool direct) {
    return ((2 * KS + (direct ? 0 : NS)) * (4 * (1024 / NS) + 1) * 8 <= 72 * 1024)   ? 4
           : ((2 * KS + (direct ? 0 : NS)) * (2 * (1024 / NS) + 1) * 8 <= 72 * 1024) ? 2
                                                                                     : 1;
}

// STORE 1 (direct): C's five lowest positions are row bits, so a warp's 32
// consecutive rows are 32 consecutive C addresses and outputs are stored
// straight from registers.  STORE 0: outputs go through shared memory and
// out in C's own runs.  STORE 2 (planar): through shared memory and out as
// the next tensor-core step's hi/lo planes, in destination runs, two
// neighbouring elements per thread.
template <int NK, int NN, int STORE>
__global__ void __launch_bounds__(kThreads, 3) small_tiled_kernel(const SmallArgs a) {
    constexpr bool DIRECT = STORE == 1;
    constexpr int KS = 1 << NK, NS = 1 << NN, NPT = 4;
    constexpr int NG = NS / NPT, RG = kThreads / NG;
    constexpr int RPT = small_tile_rpt(KS, NS, DIRECT);
    constexpr int RT = RG * RPT, RP = RT + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    const int HS = 1 << a.nH;
    const int SS = HS * KS * NS;
    float2 *S_s = reinterpret_cast<float2 *>(smem);
    float2 *T_s = S_s + SS;                                  // two stages of KS * RP
    float2 *C_s = T_s + 2 * KS * RP;                         // NS * RP (unless DIRECT)
    uint64_t *offT_s = reinterpret_cast<uint64_t *>(C_s + (DIRECT ? 0 : NS * RP));
    uint64_t *offC_s = offT_s + 32;  // 64 low-bit entries, then 64 high-bit entries
    uint32_t *runDstT_s = reinterpret_cast<uint32_t *>(offC_s + 128);
    uint32_t *dstLoT_s = runDstT_s + 32, *dstHiT_s = dstLoT_s + 64;
    uint32_t *runSrcC_s = dstHiT_s + 64, *srcLoC_s = runSrcC_s + 128, *srcHiC_s = srcLoC_s + 64;
    for (int idx = threadIdx.x; idx < SS; idx += blockDim.x) {
        uint32_t n = idx & (NS - 1), k = (idx >> NN) & (KS - 1), h = idx >> (NN + NK);
        uint64_t addr = scatter_bits(h, a.hposS, a.nH) | scatter_bits(k, a.kposS, NK) | scatter_bits(n, a.nposS, NN);
        S_s[idx] = a.S[addr];
    }
    for (int i = threadIdx.x; i < 64; i += blockDim.x) {
        if (i < 32) {
            offT_s[i] = a.runOffT[i];
            runDstT_s[i] = a.runDstT[i];
        }
        offC_s[i] = a.runOffCLo[i];
        offC_s[64 + i] = a.runOffCHi[i];
        runSrcC_s[i] = a.runSrcCLo[i];
        runSrcC_s[64 + i] = a.runSrcCHi[i];
        dstLoT_s[i] = a.dstLoT[i];
        dstHiT_s[i] = a.dstHiT[i];
        srcLoC_s[i] = a.srcLoC[i];
        srcHiC_s[i] = a.srcHiC[i];
    }
    __syncthreads();
    const int rgi = threadIdx.x % RG, ngi = threadIdx.x / RG;
    const int64_t n_tiles = a.rows >> a.tb;
    constexpr int ET = RT * KS, EC = RT * NS;
    const int lt = a.lt, lc = a.lc;
    const uint32_t ltmask = (1u << lt) - 1, lcmask = (1u << lc) - 1;
    const uint32_t T_s_addr = smem_u32_k(T_s);
    constexpr uint32_t kStageBytes = KS * RP * sizeof(float2);
    // direct stores: this thread's row offsets in C (the tile base adds the
    // bits above the tile) and its outputs' n offsets
    uint64_t rowC[RPT], nC[NPT];
    if (DIRECT) {
#pragma unroll
        for (int i = 0; i < RPT; i++) rowC[i] = insert_zeros((uint64_t)(rgi + i * RG), a.cins, a.n_cins);
#pragma unroll
        for (int j = 0; j < NPT; j++) nC[j] = scatter_bits((uint64_t)(ngi * NPT + j), a.nposC, NN);
    }
    auto issue = [&](int64_t tile, int stage) {
        const float2 *Tt = a.T + insert_zeros((uint64_t)tile << a.tb, a.tins, a.n_tins);
        const uint32_t base = T_s_addr + stage * kStageBytes;
#pragma unroll 4
        for (int f = threadIdx.x; f < ET; f += kThreads) {
            const uint32_t e = f & ltmask;
            const uint32_t d = runDstT_s[f >> lt] + dstLoT_s[e & 63] + dstHiT_s[e >> 6];
            cp_async8(base + d * (uint32_t)sizeof(float2), Tt + offT_s[f >> lt] + e);
        }
    };
    int stage = 0;
    float mx = 0.f;  // of the values computed (max_slot; complex64 stores only)
    if ((int64_t)blockIdx.x < n_tiles) issue(blockIdx.x, 0);
    cp_async_commit();
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t next = tile + gridDim.x;
        if (next < n_tiles) issue(next, stage ^ 1);
        cp_async_commit();
        cp_async_wait1();  // this tile's copies (all but the newest group) have landed
        __syncthreads();
        const uint64_t r0 = (uint64_t)tile << a.tb;
        float2 *Ct = a.C + insert_zeros(r0, a.cins, a.n_cins);
        const uint32_t h = gather_bits(r0, a.hbitR, a.nH);
        float2 acc[RPT][NPT];
#pragma unroll
        for (int i = 0; i < RPT; i++)
#pragma unroll
            for (int j = 0; j < NPT; j++) acc[i][j] = make_float2(0.f, 0.f);
        const float2 *Sh = S_s + (size_t)h * KS * NS + ngi * NPT;
        const float2 *Tr = T_s + stage * KS * RP + rgi;
#pragma unroll
        for (int k = 0; k < KS; k++) {
            float2 tv[RPT], sv[NPT];
#pragma unroll
            for (int i = 0; i < RPT; i++) tv[i] = Tr[k * RP + i * RG];
#pragma unroll
            for (int j = 0; j < NPT; j += 2) {
                const float4 s2 = *reinterpret_cast<const float4 *>(Sh + k * NS + j);
                sv[j] = make_float2(s2.x, s2.y);
                sv[j + 1] = make_float2(s2.z, s2.w);
            }
#pragma unroll
            for (int i = 0; i < RPT; i++)
#pragma unroll
                for (int j = 0; j < NPT; j++) cfma(acc[i][j], tv[i], sv[j]);
        }
        if (STORE != 2 && a.max_slot) {
#pragma unroll
            for (int i = 0; i < RPT; i++)
#pragma unroll
                for (int j = 0; j < NPT; j++) mx = absmax2(mx, acc[i][j]);
        }
        if (DIRECT) {
            __syncthreads();  // every thread's reads of this stage are done
#pragma unroll
            for (int i = 0; i < RPT; i++)
#pragma unroll
                for (int j = 0; j < NPT; j++) Ct[rowC[i] + nC[j]] = acc[i][j];
        } else {
#pragma unroll
            for (int i = 0; i < RPT; i++)
#pragma unroll
                for (int j = 0; j < NPT; j++) C_s[(ngi * NPT + j) * RP + rgi + i * RG] = acc[i][j];
            __syncthreads();
            if (STORE == 0) {
                for (int f = threadIdx.x; f < EC; f += kThreads) {
                    const uint32_t u = f >> lc, e = f & lcmask;
                    Ct[offC_s[u & 63] + offC_s[64 + (u >> 6)] + e] =
                        C_s[runSrcC_s[u & 63] + runSrcC_s[64 + (u >> 6)] + srcLoC_s[e & 63] + srcHiC_s[e >> 6]];
                }
            } else {
                // destination of the tile's first element: the row bits above
                // the tile, each at its destination position
                uint64_t dbase = 0;
                for (int i = a.tb; i < a.row_bits; i++) dbase |= ((r0 >> i) & 1ull) << a.drow[i];
                for (int f = 2 * threadIdx.x; f < EC; f += 2 * kThreads) {
                    const uint32_t u = f >> lc, e = f & lcmask;  // e even, e + 1 in the same run
                    const uint32_t rs = runSrcC_s[u & 63] + runSrcC_s[64 + (u >> 6)];
                    const float2 v0 = C_s[rs + srcLoC_s[e & 63] + srcHiC_s[e >> 6]];
                    const float2 v1 = C_s[rs + srcLoC_s[(e + 1) & 63] + srcHiC_s[(e + 1) >> 6]];
                    const uint64_t d = dbase + offC_s[u & 63] + offC_s[64 + (u >> 6)] + e;
                    const Pieces p0 = split_value(a.planar_mode, v0, 0), p1 = split_value(a.planar_mode, v1, 0);
                    if (a.planar_mode == 2) {
                        uint2 *P = reinterpret_cast<uint2 *>(a.C);
#pragma unroll
                        for (int q = 0; q < 4; q++) P[(d + q * a.plane_stride) >> 1] = make_uint2(p0.q[q], p1.q[q]);
                    } else {
                        uint32_t *P = reinterpret_cast<uint32_t *>(a.C);
#pragma unroll
                        for (int q = 0; q < 4; q++) P[(d + q * a.plane_stride) >> 1] = p0.q[q] | (p1.q[q] << 16);
                    }
                }
            }
        }
        stage ^= 1;
        // the copies into the stage just read are issued in the next
        // iteration, after every thread has passed the barrier above (its
        // reads of that stage done); the next C_s stores follow the next
        // first barrier, after every thread's reads of C_s
    }
    cp_async_wait_all();
    if (STORE != 2 && a.max_slot) publish_max(a.max_slot, mx);
}

// ------------------------------------------------------- tiled bit permute
// one destination element
__device__ __forceinline__ void store_elem(const BitPermArgs &a, uint64_t d, float2 v, int e) {
    if (a.mode == 0) {
        reinterpret_cast<float2 *>(a.out)[d] = v;
        return;
    }
    if (mode_3m(a.mode)) {
        const Pieces6 pc = split_value_3m(a.mode, v, e);
        if (mode_word(a.mode)) {
            uint32_t *P = reinterpret_cast<uint32_t *>(a.out);
            for (int q = 0; q < 6; q++) P[d + q * a.plane_stride] = pc.q[q];
        } else {
            uint16_t *P = reinterpret_cast<uint16_t *>(a.out);
            for (int q = 0; q < 6; q++) P[d + q * a.plane_stride] = (uint16_t)pc.q[q];
        }
        return;
    }
    const Pieces pc = split_value(a.mode, v, e);
    const int np = mode_planes(a.mode);
    if (a.mode == 2) {
        uint32_t *P = reinterpret_cast<uint32_t *>(a.out);
        for (int q = 0; q < np; q++) P[d + q * a.plane_stride] = pc.q[q];
    } else {
        uint16_t *P = reinterpret_cast<uint16_t *>(a.out);
        for (int q = 0; q < np; q++) P[d + q * a.plane_stride] = (uint16_t)pc.q[q];
    }
}

// destination elements d and d + 1 (d even): one vector store per plane
__device__ __forceinline__ void store_pair(const BitPermArgs &a, uint64_t d, float2 v0, float2 v1, int e) {
    if (a.mode == 0) {
        reinterpret_cast<float4 *>(a.out)[d >> 1] = make_float4(v0.x, v0.y, v1.x, v1.y);
        return;
    }
    if (mode_3m(a.mode)) {
        const Pieces6 p0 = split_value_3m(a.mode, v0, e), p1 = split_value_3m(a.mode, v1, e);
        if (mode_word(a.mode)) {
            uint2 *P = reinterpret_cast<uint2 *>(a.out);
            for (int q = 0; q < 6; q++) P[(d + q * a.plane_stride) >> 1] = make_uint2(p0.q[q], p1.q[q]);
        } else {
            uint32_t *P = reinterpret_cast<uint32_t *>(a.out);
            for (int q = 0; q < 6; q++) P[(d + q * a.plane_stride) >> 1] = p0.q[q] | (p1.q[q] << 16);
        }
        return;
    }
    const Pieces p0 = split_value(a.mode, v0, e), p1 = split_value(a.mode, v1, e);
    const int np = mode_planes(a.mode);
    if (a.mode == 2) {
        uint2 *P = reinterpret_cast<uint2 *>(a.out);
        for (int q = 0; q < np; q++) P[(d + q * a.plane_stride) >> 1] = make_uint2(p0.q[q], p1.q[q]);
    } else {
        uint32_t *P = reinterpret_cast<uint32_t *>(a.out);
        for (int q = 0; q < np; q++) P[(d + q * a.plane_stride) >> 1] = p0.q[q] | (p1.q[q] << 16);
    }
}

// Each CTA builds the tile's offset tables once, then walks tiles two at a
// time (two independent read batches in flight per thread).  Source bit 0
// and destination bit 0 are always tile bits (the first read-order and the
// first write-order bit), so with aligned buffers a thread moves two
// neighbouring elements per load and per store.
__global__ void __launch_bounds__(kThreads) bitperm_kernel(const BitPermArgs a) {
    constexpr int T = 1 << kTileMaxBits;
    __shared__ float2 buf[2][T];
    // a tile bit that is low in one layout can sit at position 32 or above in
    // the other (tensors of more than 2^32 elements): 64-bit tile offsets
    __shared__ uint64_t src_off[T], dst_off[T];
    __shared__ uint32_t w_of[T];
    // the rest index scattered 6 bits at a time through lookup tables
    constexpr int kChunk = 6, kChunks = (kMaxRank + kChunk - 1) / kChunk;
    __shared__ uint64_t rest_tab[2][kChunks][1 << kChunk];
    const int n_chunk = (a.n_rest + kChunk - 1) / kChunk;
    for (int i = threadIdx.x; i < n_chunk << kChunk; i += blockDim.x) {
        const int c = i >> kChunk, v = i & ((1 << kChunk) - 1);
        const int nb = min(kChunk, a.n_rest - c * kChunk);
        uint64_t so = 0, d = 0;
        for (int j = 0; j < nb; j++) {
            const uint64_t b = (uint64_t)((v >> j) & 1);
            so |= b << a.rest_src[c * kChunk + j];
            d |= b << a.rest_dst[c * kChunk + j];
        }
        rest_tab[0][c][v] = so;
        rest_tab[1][c][v] = d;
    }
    const int tile = 1 << a.n_tile;
    for (int e = threadIdx.x; e < tile; e += blockDim.x) {
        uint32_t w = 0;
        uint64_t so = 0, d = 0;
        for (int j = 0; j < a.n_tile; j++) {
            const uint32_t b = (e >> j) & 1u;
            w |= b << a.rd_w[j];
            so |= (uint64_t)b << a.rd_src[j];
            d |= (uint64_t)b << a.tile_dst[j];
        }
        src_off[e] = so;
        w_of[e] = w;
        dst_off[e] = d;
    }
    const int es = mode_scaled(a.mode) ? fp16s_exponent(__uint_as_float(*a.scale)) : 0;
    __syncthreads();
    const int64_t n_rest = 1ll << a.n_rest;
    const int half = tile >> 1;
    for (int64_t r0 = 2 * (int64_t)blockIdx.x; r0 < n_rest; r0 += 2 * (int64_t)gridDim.x) {
        const int nr = (r0 + 1 < n_rest) ? 2 : 1;
        uint64_t s_rest[2], d_rest[2];
        for (int q = 0; q < nr; q++) {
            s_rest[q] = d_rest[q] = 0;
            const uint64_t rr = (uint64_t)(r0 + q);
            for (int c = 0; c < n_chunk; c++) {
                const int v = (int)((rr >> (c * kChunk)) & ((1 << kChunk) - 1));
                s_rest[q] |= rest_tab[0][c][v];
                d_rest[q] |= rest_tab[1][c][v];
            }
        }
        if (a.pair_rd) {
            for (int e2 = threadIdx.x; e2 < half; e2 += blockDim.x) {
                const uint64_t so = src_off[2 * e2];
                const uint32_t w0 = w_of[2 * e2], w1 = w_of[2 * e2 + 1];
                const float4 v0 = reinterpret_cast<const float4 *>(a.in)[(s_rest[0] | so) >> 1];
                if (nr == 2) {
                    const float4 v1 = reinterpret_cast<const float4 *>(a.in)[(s_rest[1] | so) >> 1];
                    buf[1][w0] = make_float2(v1.x, v1.y);
                    buf[1][w1] = make_float2(v1.z, v1.w);
                }
                buf[0][w0] = make_float2(v0.x, v0.y);
                buf[0][w1] = make_float2(v0.z, v0.w);
            }
        } else {
            for (int e = threadIdx.x; e < tile; e += blockDim.x) {
                const uint64_t so = src_off[e];
                const uint32_t w = w_of[e];
                const float2 v0 = a.in[s_rest[0] | so];
                if (nr == 2) buf[1][w] = a.in[s_rest[1] | so];
                buf[0][w] = v0;
            }
        }
        __syncthreads();
        if (a.pair_wr) {
            for (int q = 0; q < nr; q++)
                for (int e2 = threadIdx.x; e2 < half; e2 += blockDim.x)
                    store_pair(a, d_rest[q] | dst_off[2 * e2], buf[q][2 * e2], buf[q][2 * e2 + 1], es);
        } else {
            for (int q = 0; q < nr; q++)
                for (int e = threadIdx.x; e < tile; e += blockDim.x) store_elem(a, d_rest[q] | dst_off[e], buf[q][e], es);
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------- max |x|
__global__ void __launch_bounds__(kThreads) maxabs_kernel(const MaxAbsArgs a) {
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = a.in[i];
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    // non-negative floats order like their bit patterns
    if ((threadIdx.x & 31) == 0) atomicMax(a.slot, __float_as_uint(m));
}

// --------------------------------------------------------------- FP32 GEMM
// 64 x 64 output tile per CTA, 256 threads, each 4 x 4 complex outputs,
// K staged through shared memory 16 at a time.  Each K tile is summed into
// a fresh partial that is then added to the running sum (blocked
// summation): the rounding error of a length-K dot product then grows like
// sqrt(16) + sqrt(K / 16) roundings instead of sqrt(K), which keeps the
// plain FP32 form within 1e-5 of the exact amplitudes on deep circuits
// (K up to 2^11 per step).
constexpr int BM = 64, BN = 64, BK = 16;

__global__ void __launch_bounds__(256) gemm_f32_kernel(const GemmArgs a) {
    __shared__ float2 As[BK][BM + 1];
    __shared__ float2 Bs[BK][BN + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
    for (int64_t h = blockIdx.z; h < a.H; h += gridDim.z) {
        const float2 *Ab = a.A + h * a.sAh;
        const float2 *Bb = a.B + h * a.sBh;
        float2 acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) acc[i][j] = make_float2(0.f, 0.f);
        const bool a_kfast = a.sAk == 1, b_nfast = a.sBn == 1;
        for (int64_t k0 = 0; k0 < a.K; k0 += BK) {
#pragma unroll
            for (int i = 0; i < (BM * BK) / 256; i++) {
                int e = tid + i * 256;
                int kk, mm;
                if (a_kfast) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
                int64_t m = m0 + mm, k = k0 + kk;
                As[kk][mm] = (m < a.M && k < a.K) ? Ab[m * a.sAm + k * a.sAk] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < (BN * BK) / 256; i++) {
                int e = tid + i * 256;
                int kk, nn;
                if (b_nfast) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
                int64_t n = n0 + nn, k = k0 + kk;
                Bs[kk][nn] = (n < a.N && k < a.K) ? Bb[k * a.sBk + n * a.sBn] : make_float2(0.f, 0.f);
            }
            __syncthreads();
            float2 part[4][4];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) part[i][j] = make_float2(0.f, 0.f);
#pragma unroll
            for (int kk = 0; kk < BK; kk++) {
                float2 av[4], bv[4];
#pragma unroll
                for (int i = 0; i < 4; i++) av[i] = As[kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; j++) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) cfma(part[i][j], av[i], bv[j]);
            }
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    acc[i][j].x += part[i][j].x;
                    acc[i][j].y += part[i][j].y;
                }
            __syncthreads();
        }
        float2 *Cb = a.C + h * a.sCh;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            int64_t m = m0 + ty + 16 * i;
            if (m >= a.M) continue;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                int64_t n = n0 + tx + 16 * j;
                if (n < a.N) Cb[m * a.sCm + n * a.sCn] = acc[i][j];
            }
        }
    }
}

// ---------------------------------------------------------- slice extraction
__global__ void __launch_bounds__(kThreads) extract_kernel(const ExtractEntry *e, int n_entries,
                                                           uint64_t slice_base) {
    const ExtractEntry &x = e[blockIdx.y];
    uint64_t fixed = 0;
    for (int f = 0; f < x.nf; f++) fixed |= ((slice_base >> x.sbit[f]) & 1ull) << x.fpos[f];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < x.n_out; j += gridDim.x * blockDim.x)
        x.dst[j] = x.src[insert_zeros((uint64_t)j, x.fpos_sorted, x.nf) | fixed];
}

// ------------------------------------------------------ cross-slice FP64 sum
__global__ void __launch_bounds__(kThreads) accum_warp_kernel(const AccumArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t n_out = 1ll << a.n_open;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t o = warp; o < n_out; o += n_warps) {
        const uint64_t ob = scatter_bits((uint64_t)o, a.opos, a.n_open);
        double sr = 0.0, si = 0.0;
        for (int64_t b = a.b_lo + lane; b < a.b_hi; b += 32) {
            const float2 v = a.R[ob | scatter_bits((uint64_t)b, a.bpos, a.n_batch)];
            sr += (double)v.x;
            si += (double)v.y;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            sr += __shfl_xor_sync(0xffffffffu, sr, off);
            si += __shfl_xor_sync(0xffffffffu, si, off);
        }
        if (lane == 0) {
            double2 cur = a.amp[o];
            cur.x += sr;
            cur.y += si;
            a.amp[o] = cur;
        }
    }
}

__global__ void __launch_bounds__(kThreads) accum_thread_kernel(const AccumArgs a) {
    const int64_t n_out = 1ll << a.n_open;
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_out; o += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t ob = scatter_bits((uint64_t)o, a.opos, a.n_open);
        double sr = 0.0, si = 0.0;
        for (int64_t b = a.b_lo; b < a.b_hi; b++) {
            const float2 v = a.R[ob | scatter_bits((uint64_t)b, a.bpos, a.n_batch)];
            sr += (double)v.x;
            si += (double)v.y;
        }
        double2 cur = a.amp[o];
        cur.x += sr;
        cur.y += si;
        a.amp[o] = cur;
    }
}

// -------------------------------------------------- probabilities and XEB sums
__global__ void __launch_bounds__(kThreads) prob_kernel(const double2 *amp, int64_t n, double *prob, double *out) {
    double s = 0.0, mx = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = amp[i];
        const double p = v.x * v.x + v.y * v.y;
        if (prob) prob[i] = p;
        s += p;
        mx = fmax(mx, p);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, off);
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    }
    __shared__ double ws[kThreads / 32], wm[kThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { ws[w] = s; wm[w] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bs = 0.0, bm = 0.0;
        for (int i = 0; i < kThreads / 32; i++) { bs += ws[i]; bm = fmax(bm, wm[i]); }
        atomicAdd(out, bs);
        // non-negative doubles order like their bit patterns
        atomicMax(reinterpret_cast<unsigned long long *>(out + 2), (unsigned long long)__double_as_longlong(bm));
    }
}

__global__ void xeb_finalize_kernel(double *out, int scale_exp) { out[1] = ldexp(out[0], scale_exp) - 1.0; }

}  // namespace

cudaError_t set_max_dynamic_smem(const void *kernel, int bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> done;  // (kernel, device) -> bytes set
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    auto it = done.find({kernel, dev});
    if (it != done.end() && it->second >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done[{kernel, dev}] = bytes;
    return e;
}

template <int NC>
cudaError_t launch_small_nc(const SmallArgs &a, int grid, size_t smem, cudaStream_t s) {
    cudaError_t e = set_max_dynamic_smem((const void *)small_kernel<NC>, 100 * 1024);
    if (e != cudaSuccess) return e;
    small_kernel<NC><<<grid, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

namespace {
constexpr size_t kTiledTableBytes = (32 + 128) * 8 + (32 + 64 + 64 + 128 + 64 + 64) * 4;
size_t small_tiled_smem(const SmallArgs &a) {
    const size_t KS = (size_t)1 << a.nK, NS = (size_t)1 << a.nN, HS = (size_t)1 << a.nH;
    const size_t RP = ((size_t)1 << a.tb) + 1;
    return (HS * KS * NS + (2 * KS + (a.tiled == 2 ? 0 : NS)) * RP) * sizeof(float2) + kTiledTableBytes;
}

// contiguous-run structure of a tile over `tb` row bits plus the nX bits at
// xpos (bit j of x at position xpos[j]) of a tensor of rank `rank`, whose
// row bits fill the other positions in increasing order.  Shared-memory
// index of (x, row) = x * RP + row.
bool tile_runs(int rank, int tb, int nX, const int *xpos, int RP, int &l, int &n_run, uint64_t *run_off,
               uint32_t *run_sm, uint32_t *lo, uint32_t *hi) {
    std::vector<int> xbit(rank, -1);
    for (int j = 0; j < nX; j++) {
        if (xpos[j] < 0 || xpos[j] >= rank) return false;
        xbit[xpos[j]] = j;
    }
    // weight (shared-memory index step) of each position inside the run
    std::vector<uint32_t> w;
    int rows_seen = 0, p = 0;
    for (; p < rank; p++) {
        if (xbit[p] >= 0) {
            w.push_back((uint32_t)(1u << xbit[p]) * (uint32_t)RP);
        } else {
            if (rows_seen == tb) break;
            w.push_back(1u << rows_seen);
            rows_seen++;
        }
    }
    if (rows_seen != tb) return false;
    l = p;
    if (l > 12) return false;
    std::vector<int> high;  // x bits above the run
    for (int q = p; q < rank; q++)
        if (xbit[q] >= 0) high.push_back(q);
    if (high.size() > 5) return false;
    n_run = 1 << (int)high.size();
    for (int u = 0; u < 32; u++) {
        uint64_t off = 0;
        uint32_t sm = 0;
        if (u < n_run)
            for (size_t i = 0; i < high.size(); i++)
                if ((u >> i) & 1) {
                    off |= 1ull << high[i];
                    sm += (uint32_t)(1u << xbit[high[i]]) * (uint32_t)RP;
                }
        run_off[u] = off;
        run_sm[u] = sm;
    }
    for (int v = 0; v < 64; v++) {
        uint32_t a = 0, b = 0;
        for (int j = 0; j < 6; j++) {
            if (((v >> j) & 1) == 0) continue;
            if (j < l) a += w[j];
            if (j + 6 < l) b += w[j + 6];
        }
        lo[v] = a;
        hi[v] = b;
    }
    return true;
}

// contiguous-run structure of a tile given each tile bit's position in the
// tensor written and its weight (shared-memory index step); run tables in
// two levels (low and high six bits of the run index)
bool tile_runs_pos(std::vector<std::pair<int, uint32_t>> bits, int &l, int &n_run, uint64_t *off_lo,
                   uint64_t *off_hi, uint32_t *sm_lo, uint32_t *sm_hi, uint32_t *lo, uint32_t *hi) {
    std::sort(bits.begin(), bits.end());
    int p = 0;
    while (p < (int)bits.size() && bits[p].first == p) p++;
    l = p;
    const int nh = (int)bits.size() - l;
    if (l > 12 || nh > 12) return false;
    n_run = 1 << nh;
    for (int v = 0; v < 64; v++) {
        uint64_t ol = 0, oh = 0;
        uint32_t sl = 0, sh = 0;
        for (int i = 0; i < 6; i++) {
            if (((v >> i) & 1) == 0) continue;
            if (i < nh) {
                ol |= 1ull << bits[l + i].first;
                sl += bits[l + i].second;
            }
            if (i + 6 < nh) {
                oh |= 1ull << bits[l + 6 + i].first;
                sh += bits[l + 6 + i].second;
            }
        }
        off_lo[v] = ol;
        off_hi[v] = oh;
        sm_lo[v] = sl;
        sm_hi[v] = sh;
    }
    for (int v = 0; v < 64; v++) {
        uint32_t a = 0, b = 0;
        for (int j = 0; j < 6; j++) {
            if (((v >> j) & 1) == 0) continue;
            if (j < l) a += bits[j].second;
            if (j + 6 < l) b += bits[j + 6].second;
        }
        lo[v] = a;
        hi[v] = b;
    }
    return true;
}

// the C tile's bits: the first tb row positions (weights 1 << i) and the N
// positions (weights (1 << j) * RP), each at position dest(q) of C position q
std::vector<std::pair<int, uint32_t>> c_tile_bits(const SmallArgs &a, int row_bits, int tb, int RP,
                                                  const int *cdest) {
    const int rc = row_bits + a.nN;
    std::vector<char> isn(rc, 0);
    for (int j = 0; j < a.nN; j++) isn[a.nposC[j]] = 1;
    std::vector<int> rowpos;
    for (int q = 0; q < rc; q++)
        if (!isn[q]) rowpos.push_back(q);
    std::vector<std::pair<int, uint32_t>> bits;
    for (int i = 0; i < tb; i++) bits.push_back({cdest ? cdest[rowpos[i]] : rowpos[i], 1u << i});
    for (int j = 0; j < a.nN; j++)
        bits.push_back({cdest ? cdest[a.nposC[j]] : a.nposC[j], (1u << j) * (uint32_t)RP});
    return bits;
}

// Resident CTAs per SM times the SM count of the current device, for a
// kernel at a given dynamic shared-memory size (cached per device; the
// kernel's shared-memory limit must already be raised).
int64_t resident_ctas(const void *kernel, size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<std::pair<const void *, size_t>, int>, int64_t> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_pair(std::make_pair(kernel, smem), dev);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int occ = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kThreads, smem) != cudaSuccess || occ < 1) occ = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
    return cache[key] = (int64_t)occ * sms;
}

template <int NK, int NN, int STORE>
cudaError_t launch_small_tiled_t(const SmallArgs &a, cudaStream_t s) {
    const size_t smem = small_tiled_smem(a);
    const void *kernel = (const void *)small_tiled_kernel<NK, NN, STORE>;
    cudaError_t e = set_max_dynamic_smem(kernel, 160 * 1024);
    if (e != cudaSuccess) return e;
    const int64_t tiles = a.rows >> a.tb;
    const int grid = (int)std::min<int64_t>(tiles, resident_ctas(kernel, smem));
    small_tiled_kernel<NK, NN, STORE><<<grid, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int NK, int NN>
cudaError_t launch_small_tiled_kn(const SmallArgs &a, cudaStream_t s) {
    if (a.tiled == 2) return launch_small_tiled_t<NK, NN, 1>(a, s);
    if (a.tiled == 3) return launch_small_tiled_t<NK, NN, 2>(a, s);
    return launch_small_tiled_t<NK, NN, 0>(a, s);
}

template <int NK>
cudaError_t launch_small_tiled_k(const SmallArgs &a, cudaStream_t s) {
    switch (a.nN) {
    case 2: return launch_small_tiled_kn<NK, 2>(a, s);
    case 3: return launch_small_tiled_kn<NK, 3>(a, s);
    case 4: return launch_small_tiled_kn<NK, 4>(a, s);
    case 5: return launch_small_tiled_kn<NK, 5>(a, s);
    }
    return cudaErrorInvalidValue;
}
}  // namespace

void prepare_small_tiled(SmallArgs &a) {
    a.tiled = 0;
    const int nK = a.nK, nN = a.nN;
    if (nK < 2 || nK > 5 || nN < 2 || nN > 5 || a.rows < 4096 || (a.rows & (a.rows - 1)) != 0) return;
    const int KS = 1 << nK, NS = 1 << nN;
    // N <= 8: the row kernel reads T once with direct loads and is bound by
    // memory; staging T through shared memory only pays for K = 32 with K
    // bits among T's five lowest positions (measured on GB300: 8 x 8 steps
    // of 2^22 rows 0.113-0.117 ms on the row kernel against 0.12-0.14 ms
    // tiled; 32 x 8 with low K bits 0.164 ms against 0.110 ms)
    bool t_rows_low = true;
    for (int j = 0; j < nK; j++)
        if (a.kposT[j] < 5) t_rows_low = false;
    if (NS <= 8 && (KS < 32 || t_rows_low)) return;
    // outputs stored from registers when C's five lowest positions are row bits
    bool direct = true;
    for (int j = 0; j < nN; j++)
        if (a.nposC[j] < 5) direct = false;
    const int rpt = small_tile_rpt(KS, NS, direct);
    const int RT = (1024 / NS) * rpt;
    if (RT > a.rows) return;
    int tb = 0;
    while ((1 << tb) < RT) tb++;
    for (int j = 0; j < a.nH; j++)
        if (a.hbitR[j] < tb) return;
    int row_bits = 0;
    while (((int64_t)1 << row_bits) < a.rows) row_bits++;
    SmallArgs t = a;
    t.tb = tb;
    t.rpt = rpt;
    t.npt = 4;
    t.row_bits = row_bits;
    if (!tile_runs(row_bits + nK, tb, nK, a.kposT, RT + 1, t.lt, t.n_runT, t.runOffT, t.runDstT, t.dstLoT,
                   t.dstHiT))
        return;
    if (!tile_runs_pos(c_tile_bits(a, row_bits, tb, RT + 1, nullptr), t.lc, t.n_runC, t.runOffCLo, t.runOffCHi,
                       t.runSrcCLo, t.runSrcCHi, t.srcLoC, t.srcHiC))
        return;
    t.tiled = direct ? 2 : 1;
    if (small_tiled_smem(t) > 150 * 1024) return;
    a = t;
}

template <int NC>
cudaError_t launch_small_ksplit_nc(const SmallArgs &a, int grid, size_t smem, cudaStream_t s) {
    cudaError_t e = set_max_dynamic_smem((const void *)small_ksplit_kernel<NC>, 100 * 1024);
    if (e != cudaSuccess) return e;
    small_ksplit_kernel<NC><<<grid, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_small_ksplit(const SmallArgs &a, int nc, int grid, size_t smem, cudaStream_t s) {
    if (nc == 8) return launch_small_ksplit_nc<8>(a, grid, smem, s);
    if (nc == 16) return launch_small_ksplit_nc<16>(a, grid, smem, s);
    return launch_small_ksplit_nc<32>(a, grid, smem, s);
}

int prepare_small_planar(SmallArgs &a, const int *cdest, int mode, int64_t plane_stride, int *run_bits) {
    if (run_bits) *run_bits = -1;
    if (!a.tiled || (mode != 1 && mode != 2)) return 1;
    SmallArgs t = a;
    const int KS = 1 << a.nK, NS = 1 << a.nN;
    const int rpt = small_tile_rpt(KS, NS, false);
    const int RT = (1024 / NS) * rpt;
    if (RT > a.rows) return 2;
    int tb = 0;
    while ((1 << tb) < RT) tb++;
    for (int j = 0; j < a.nH; j++)
        if (a.hbitR[j] < tb) return 2;
    int row_bits = 0;
    while (((int64_t)1 << row_bits) < a.rows) row_bits++;
    const int rc = row_bits + a.nN;
    if (rc > kMaxRank) return 2;
    t.tb = tb;
    t.rpt = rpt;
    t.npt = 4;
    t.row_bits = row_bits;
    if (!tile_runs(row_bits + a.nK, tb, a.nK, a.kposT, RT + 1, t.lt, t.n_runT, t.runOffT, t.runDstT, t.dstLoT,
                   t.dstHiT))
        return 3;
    const std::vector<std::pair<int, uint32_t>> bits = c_tile_bits(a, row_bits, tb, RT + 1, cdest);
    for (const auto &b : bits)
        if (b.first < 0 || b.first >= rc) return 4;
    const bool runs_ok = tile_runs_pos(bits, t.lc, t.n_runC, t.runOffCLo, t.runOffCHi, t.runSrcCLo, t.runSrcCHi,
                                       t.srcLoC, t.srcHiC);
    if (run_bits) *run_bits = t.lc;
    if (!runs_ok || t.lc < 5) return 4;  // destination runs of at least 32 elements
    // destination of each row bit above the tile
    std::vector<char> isn(rc, 0);
    for (int j = 0; j < a.nN; j++) isn[a.nposC[j]] = 1;
    std::vector<int> rowpos;
    for (int q = 0; q < rc; q++)
        if (!isn[q]) rowpos.push_back(q);
    std::memset(t.drow, 0, sizeof t.drow);
    for (int i = tb; i < row_bits; i++) t.drow[i] = (int8_t)cdest[rowpos[i]];
    t.planar_mode = mode;
    t.plane_stride = plane_stride;
    t.tiled = 3;
    if (small_tiled_smem(t) > 150 * 1024) return 5;
    a = t;
    return 0;
}

cudaError_t launch_small(const SmallArgs &args, cudaStream_t s) {
    if (args.max_slot) {
        if (args.tiled == 3) return cudaErrorInvalidValue;  // planes out: no complex64 max
        cudaError_t e = cudaMemsetAsync(args.max_slot, 0, sizeof(unsigned), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(args.max_slot + 2, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
    }
    if (args.tiled) {
        switch (args.nK) {
        case 2: return launch_small_tiled_k<2>(args, s);
        case 3: return launch_small_tiled_k<3>(args, s);
        case 4: return launch_small_tiled_k<4>(args, s);
        case 5: return launch_small_tiled_k<5>(args, s);
        }
        return cudaErrorInvalidValue;
    }
    SmallArgs a = args;
    const int KS = 1 << a.nK, NS = 1 << a.nN, HS = 1 << a.nH;
    const size_t smem = (size_t)HS * KS * NS * sizeof(float2) + (size_t)(KS + NS) * sizeof(uint64_t);
    if (a.rows < 1 || (a.rows & (a.rows - 1)) != 0) return cudaErrorInvalidValue;
    a.row_bits = __builtin_ctzll((unsigned long long)a.rows);
    const int nc = NS <= 8 ? 8 : (NS <= 16 ? 16 : 32);  // outputs per work item
    const int64_t items = a.rows * (NS > nc ? NS / nc : 1);
    if (a.nK >= 5 && items < 152 * 128) {
        // long K, few items: one warp per item (K split over the lanes)
        const int grid = (int)std::min<int64_t>((items * 32 + kThreads - 1) / kThreads, kMaxBlocks);
        return launch_small_ksplit(a, nc, grid, smem, s);
    }
    const int grid = grid_for(items);
    if (nc == 8) return launch_small_nc<8>(a, grid, smem, s);
    if (nc == 16) return launch_small_nc<16>(a, grid, smem, s);
    return launch_small_nc<32>(a, grid, smem, s);
}

SmallTask make_small_task(const SmallArgs &a) {
    SmallTask t;
    std::memset(&t, 0, sizeof t);
    t.T = a.T;
    t.S = a.S;
    t.C = a.C;
    t.rows = a.rows;
    t.row_bits = a.rows > 0 ? __builtin_ctzll((unsigned long long)a.rows) : 0;
    t.nK = a.nK;
    t.nN = a.nN;
    t.nH = a.nH;
    const int NS = 1 << a.nN;
    t.nc = NS <= 8 ? 8 : (NS <= 16 ? 16 : 32);
    t.n_tins = a.n_tins;
    t.n_cins = a.n_cins;
    for (int j = 0; j < kSmallMaxBits; j++) {
        t.tins[j] = (int8_t)a.tins[j];
        t.cins[j] = (int8_t)a.cins[j];
        t.kposT[j] = (int8_t)a.kposT[j];
        t.nposC[j] = (int8_t)a.nposC[j];
        t.kposS[j] = (int8_t)a.kposS[j];
        t.nposS[j] = (int8_t)a.nposS[j];
    }
    for (int j = 0; j < kMaxHBits; j++) {
        t.hbitR[j] = (int8_t)a.hbitR[j];
        t.hposS[j] = (int8_t)a.hposS[j];
    }
    return t;
}

cudaError_t launch_small_tasks(const SmallTask *d_tasks, const int *d_unit_task, int total_units, int *d_ctr,
                               int n_tasks, cudaStream_t s) {
    if (total_units <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(d_ctr, 0, sizeof(int) * (size_t)(n_tasks + 1), s);
    if (e != cudaSuccess) return e;
    // S of at most 2^12 values, 2^kTaskMaxK K offsets and 2^12 N offsets
    constexpr int kSmem = 4096 * 8 + (1 << kTaskMaxK) * 8 + 4096 * 8;
    e = set_max_dynamic_smem((const void *)small_task_kernel, kSmem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::min(total_units, 2 * sms);
    small_task_kernel<<<grid, kThreads, kSmem, s>>>(d_tasks, d_unit_task, total_units, d_ctr);
    return cudaGetLastError();
}

int small_task_read_error(cudaStream_t s) {
    int v = 0, zero = 0;
    cudaMemcpyFromSymbolAsync(&v, task_error, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
    cudaMemcpyToSymbolAsync(task_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
    return v;
}

cudaError_t launch_bitperm(const BitPermArgs &args, cudaStream_t s) {
    BitPermArgs a = args;
    // pairs of neighbouring elements: source / destination bit 0 lies in the
    // tile (always, for rank >= 1); vector accesses need 16-byte aligned input
    // (leaf tensors can start at odd element offsets) and an aligned output
    const uintptr_t in = reinterpret_cast<uintptr_t>(a.in), out = reinterpret_cast<uintptr_t>(a.out);
    const bool tile_ok = a.n_tile >= 1 && a.rd_src[0] == 0 && a.tile_dst[0] == 0;
    a.pair_rd = tile_ok && (in % 16) == 0;
    a.pair_wr = tile_ok && (out % 16) == 0 && (a.mode == 0 || (a.plane_stride % 2) == 0);
    const int64_t pairs = ((1ll << a.n_rest) + 1) / 2;
    const int grid = (int)(pairs < kMaxBlocks ? pairs : kMaxBlocks);
    bitperm_kernel<<<grid, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gemm_f32(const GemmArgs &a, cudaStream_t s) {
    dim3 grid((unsigned)((a.M + BM - 1) / BM), (unsigned)((a.N + BN - 1) / BN),
              (unsigned)(a.H < 65535 ? a.H : 65535));
    if (grid.y > 65535 || (a.M + BM - 1) / BM > 0x7fffffff) return cudaErrorInvalidConfiguration;
    gemm_f32_kernel<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_extract(const ExtractEntry *d_entries, int n_entries, int max_out, uint64_t slice_base,
                           cudaStream_t s) {
    if (n_entries == 0) return cudaSuccess;
    dim3 grid((unsigned)((max_out + kThreads - 1) / kThreads), (unsigned)n_entries);
    extract_kernel<<<grid, kThreads, 0, s>>>(d_entries, n_entries, slice_base);
    return cudaGetLastError();
}

namespace {
__global__ void c128_to_c64_kernel(const double2 *src, float2 *dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = src[i];
        dst[i] = make_float2((float)v.x, (float)v.y);
    }
}
}  // namespace

cudaError_t launch_c128_to_c64(const double2 *src, float2 *dst, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    c128_to_c64_kernel<<<grid_for(n), kThreads, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_maxabs(const MaxAbsArgs &a, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(a.slot, 0, sizeof(unsigned), s);
    if (e == cudaSuccess && a.companion) e = cudaMemsetAsync(a.companion, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    maxabs_kernel<<<grid_for(a.n), kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_accum(const AccumArgs &a, cudaStream_t s) {
    const int64_t n_out = 1ll << a.n_open;
    const int64_t nb = a.b_hi - a.b_lo;
    if (nb >= 16) {
        accum_warp_kernel<<<grid_for(n_out * 32), kThreads, 0, s>>>(a);
    } else {
        accum_thread_kernel<<<grid_for(n_out), kThreads, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_prob_xeb(const double2 *amp, int64_t n, double *prob, double *d_out3, int scale_exp,
                            cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(d_out3, 0, 3 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    prob_kernel<<<grid_for(n), kThreads, 0, s>>>(amp, n, prob, d_out3);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    xeb_finalize_kernel<<<1, 1, 0, s>>>(d_out3, scale_exp);
    return cudaGetLastError();
}

cudaError_t launch_zero_f64(double *p, int64_t n, cudaStream_t s) {
    return cudaMemsetAsync(p, 0, (size_t)n * sizeof(double), s);
}

}  // namespace tn
