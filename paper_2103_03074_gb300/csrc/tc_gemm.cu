// Split-precision complex GEMM on the 5th-generation tensor cores (tcgen05).
//
// C[h, m, n] = sum_k A[h, m, k] B[h, k, n] for complex64 operands with the
// strided layout of GemmArgs, in four forms:
//   BF16x3:  x = hi + lo with hi = bf16(x), lo = bf16(x - hi) (Henry, Tang &
//            Heinecke 2019), kind::f16 MMAs, 16 K values per MMA;
//   TF32x3:  hi = tf32(x), lo = tf32(x - hi) (Ootomo & Yokota 2022), kind::tf32
//            MMAs, 8 K values per MMA;
//   FP16X3:  each operand scaled by a power of two 2^-e so that its largest
//            |re|, |im| lies in [2^13, 2^14), then hi = fp16(x), lo = fp16(x -
//            hi): 22 significant bits like TF32x3 at the kind::f16 rate, the
//            scale keeping hi and (above 2^-3 of it) lo in fp16's normal range;
//   FP16S:   the scaled value as one fp16 piece.
// A real product x*y is hi_x hi_y + hi_x lo_y + lo_x hi_y; the scaled forms'
// results are multiplied back by 2^(eA + eB) in the epilogue (exact).
//
// The split of each operand into four K-major planes (re_hi, im_hi, re_lo,
// im_lo) is done beforehand by the tiled bit-permute kernel, fused with
// whatever label permutation the operand needs (kernels.cu).  Because B's
// re and im planes of one precision sit next to each other, a 64-column B
// tile of both is one 128-row operand S = [B_re | B_im], and a complex
// product needs two real MMAs of N = 128 per piece pair:
//   P += A_re S = [A_re B_re | A_re B_im],  Q += A_im S = [A_im B_re | A_im B_im],
// re = P_left - Q_right, im = P_right + Q_left, combined in FP32 registers.
// That is 6 MMAs of 128 x 128 per K step for the hi/lo forms (2 for FP16S),
// reading 1.5x fewer shared-memory bytes per MAC than 128 x 64 MMAs.
// tc_gemm_kernel is warp-specialised.  Warp 0 issues TMA loads of the planes
// into a shared-memory ring (128-byte K chunks: 128-byte swizzle, 2 stages;
// 64-byte chunks: 64-byte swizzle, 4 stages); warp 1 issues the MMAs of each
// group of chunks into one of two tensor-memory accumulator sets {P, Q};
// warps 2-17 (four per tensor-memory lane group, a quarter of the tile's
// columns each) read each finished group's accumulators (tcgen05.ld) and add
// them into FP32 registers with round-to-nearest.  Sixteen epilogue warps (four
// per scheduler) keep short-K GEMMs, whose time is the epilogue's, issuing.  Reading out every few
// hundred bytes of K keeps the tensor core's truncating accumulation to a few
// dozen MMAs (small correction addends aligned to a large running sum lose
// their low bits, so the count of MMAs into one accumulator sets the error).
//
// CTA tile: 128 (M) x 64 (N); a K chunk is 64 or 128 bytes of a plane row.
// The kernel is persistent: one CTA per SM walks the tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ... with N tiles varying fastest, so the CTAs that
// run at the same time share A tiles (read from DRAM about once, re-served
// from L2).  The TMA ring, the accumulator sets and the read-out groups run
// on across tile boundaries, so a tile's epilogue (staged through shared
// memory in two halves and written as whole rows) overlaps the next tile's
// loads and MMAs.  GEMMs with fewer tiles than SMs split K over CTAs and add
// their partial tiles with atomics into a zeroed output.  Every mbarrier wait
// is bounded; on expiry the kernel records an error in tc_error and returns
// after freeing its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>

#include "tc_gemm.h"

namespace tn {

__device__ int tc_error = 0;

namespace {

constexpr int TM = 128, TN = 64;
// defaults from sweeps on a 4 x 8192 x 512 x 2048 GEMM and the 30-qubit
// workload: 128-byte chunks beat 64-byte ones at every read-out interval.
// Reading the accumulators out every 256 bytes of K keeps TF32x3 at 3.5e-6
// relative amplitude error there (512 bytes: 2% faster, 5.3e-6); the BF16x3
// and FP16S errors are set by their operand pieces, not by the interval, so
// they read out every 512 bytes.
constexpr int kDefaultChunkBytes = 128;
__host__ __device__ constexpr int default_flush_bytes(tn_form f) {
    return (f == TN_TF32X3 || f == TN_FP16X3) ? 256 : 512;
}
// warp 0: TMA producer; warp 1: MMA issuer; warps 2 .. 2 + EW - 1: the EW
// (8 or 16) accumulator read-out and epilogue warps, EW / 4 per TMEM lane
// group (a warp reads the lanes 32 (w mod 4) .. + 31), each 64 / (EW / 4)
// of the tile's complex columns.  Sixteen epilogue warps (18 in all, at most
// 96 registers: five warps share one scheduler's 16,384 registers) serve
// GEMMs whose tiles have one accumulator read-out (short K, the epilogue is
// their time); eight (168 registers) the others.
constexpr int kFlushWarp0 = 2;
__host__ __device__ constexpr int ep_threads(int ew) { return 32 * (kFlushWarp0 + ew); }
constexpr int kTmemCols = 512;  // 2 sets x {P, Q} x 128 columns

// operand forms of the kernel template
constexpr int kBF16 = 0, kTF32 = 1, kFP16 = 2, kFP16X3 = 3;
// one piece per value (planes re, im) or hi/lo pieces (re_hi, im_hi, re_lo, im_lo)
__host__ __device__ constexpr bool kind_split(int kind) { return kind != kFP16; }
// operands carry a per-operand power-of-two scale that the epilogue undoes
__host__ __device__ constexpr bool kind_scaled(int kind) { return kind == kFP16 || kind == kFP16X3; }

// Shared-memory ring for a K chunk of CB bytes per plane row: NP planes of A
// (128 rows) and of B (64 rows, so that planes 2j and 2j + 1 form one
// 128-row operand) per stage (4 for the hi/lo split forms, 2 for
// FP16S); as many stages as fit in 192 KB, at most 6.  64-byte chunks use the
// 64-byte swizzle, 128-byte chunks the 128-byte swizzle.  Behind the ring: the
// epilogue's staging area for half a tile (64 rows of 64 complex values).
template <int CB, int NP = 4>
struct Ring {
    static constexpr int kAPlane = TM * CB;
    static constexpr int kBPlane = TN * CB;
    static constexpr int kStageBytes = NP * kAPlane + NP * kBPlane;
    static constexpr int kStages = (196608 / kStageBytes) < 6 ? (196608 / kStageBytes) : 6;
    static constexpr int kOutRS = 66;  // staging row stride in float2 (16-byte aligned rows)
    static constexpr int kOutBytes = (TM / 2) * kOutRS * 8;
    static constexpr int kJtabBytes = 64 * 8;  // planar epilogue: (stage offset, destination offset) per group
    static constexpr int kSmem = kStages * kStageBytes + kOutBytes + 1024 + 256 + kJtabBytes;
    static_assert(kSmem <= 232448, "shared memory per CTA");
};
constexpr uint32_t kSpinLimit = 1u << 24;
// planar output by TMA: one plane's half tile (64 x 64 16-bit pieces) per
// 8 KB of the epilogue's staging area
constexpr int kTmaPlaneBytes = 8192;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// K-major swizzled operand layout of a CB-byte chunk row
template <int CB>
struct Swz {
    static constexpr uint32_t kSBO = 8 * CB;                // 8 rows of one swizzle atom
    static constexpr uint64_t kLayout = CB == 64 ? 4 : (CB == 32 ? 6 : 2);  // descriptor swizzle code
};

template <int CB>
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(16 >> 4) << 16;               // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(Swz<CB>::kSBO >> 4) << 32;   // stride byte offset: 8 rows
    d |= (uint64_t)1 << 46;                       // descriptor version
    d |= Swz<CB>::kLayout << 61;                  // swizzle mode
    return d;
}

// instruction descriptor (kind::f16 / kind::tf32): D f32, K-major A and B
__host__ __device__ constexpr uint32_t make_idesc(uint32_t ab_format, int M, int N, bool neg_a) {
    return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((neg_a ? 1u : 0u) << 13) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (KIND == kTF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    }
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, P;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait for the phase of `parity`.  On expiry it records the error in
// tc_error; once any wait has given up, the others stop early, so a stalled
// pipeline unwinds in one expiry instead of one per remaining wait.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (uint32_t i = 0; i < kSpinLimit; i++) {
        if (mbar_try(mbar, parity)) return true;
        if ((i & 1023u) == 1023u && *reinterpret_cast<volatile int *>(&tc_error) != 0) return false;
    }
    atomicExch(&tc_error, 1);
    return false;
}

// Bounded wait that is not cut short by tc_error: used on the way out to let
// this CTA's own copies and MMAs land before its memory is released.
__device__ __forceinline__ void mbar_drain(uint32_t mbar, uint32_t parity) {
    for (uint32_t i = 0; i < kSpinLimit; i++)
        if (mbar_try(mbar, parity)) return;
    atomicExch(&tc_error, 1);
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            int c4, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5, %6}], [%7];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, const uint32_t *w) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3])
                 : "memory");
}

// bulk tensor store of a shared-memory box (bulk-group completion)
__device__ __forceinline__ void tma_store_5d(const CUtensorMap *map, uint32_t src, int c0, int c1, int c2, int c3,
                                             int c4) {
    asm volatile("cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the committed stores have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// the committed stores have completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// generic-proxy shared-memory writes made visible to the bulk copies
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t *r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------- GEMM
struct GemmTcParams {
    float2 *C;
    int64_t H, M, N, K;  // K in complex elements
    int64_t sCh, sCm, sCn;
    int k_chunk;       // K values per chunk
    int klo_bits;      // plane layout: K value kc at (kc & (2^klo_bits - 1), kc >> klo_bits); 31 = unchunked
    int ksplit;        // K partitions (> 1: atomic adds into a zeroed C)
    int flush_chunks;  // chunks per accumulator read-out
    int gm, gn;        // M and N tiles
    int64_t tiles;     // gn * gm * H * ksplit (< 2^32: the tile decode is 32-bit)
    int all_chunks;    // K chunks of the whole K range
    int part_len;      // K chunks per K part (the last part may be shorter or empty)
    const unsigned *scales;  // scaled forms: max-abs slots of A and B (float bits)
    unsigned *max_slot;      // optional: atomic max of |re|, |im| over C (float bits)
    TcPlanarOut out;         // planar epilogue (out.mode > 0)
    // planar output whose lowest destination bits are the tile's column bits
    // c0, c1, ...: log2 of the runs of consecutive destination elements a
    // lane stores straight from its registers (0: staged through shared
    // memory)
    int direct_run;
    TcTmaOut tma;  // tma.on: planar output written to shared memory in box order and stored by TMA
};

// tile t -> (n tile, m tile, batch h, K part); N tiles vary fastest
struct TileCoord {
    int64_t n0, m0;
    int h, part;
};
__device__ __forceinline__ TileCoord tile_coord(const GemmTcParams &p, int64_t tile) {
    // 32-bit unsigned division (the launcher keeps the tile count below 2^32)
    uint32_t t = (uint32_t)tile;
    const uint32_t gn = (uint32_t)p.gn, gm = (uint32_t)p.gm, ks = (uint32_t)p.ksplit;
    TileCoord c;
    uint32_t q = t / gn;
    c.n0 = (int64_t)(t - q * gn) * TN;
    t = q;
    q = t / gm;
    c.m0 = (int64_t)(t - q * gm) * TM;
    t = q;
    q = t / ks;
    c.h = (int)q;
    c.part = (int)(t - q * ks);
    return c;
}

// [c_begin, c_begin + count) = the K chunks of one K part
__device__ __forceinline__ int part_chunks(const GemmTcParams &p, int part, int &c_begin) {
    c_begin = part * p.part_len;
    const int c_end = min(p.all_chunks, c_begin + p.part_len);
    return c_end > c_begin ? c_end - c_begin : 0;
}

__device__ __forceinline__ uint64_t scatter8(uint64_t v, const int8_t *pos, int n) {
    uint64_t r = 0;
    for (int j = 0; j < n; j++) r |= ((v >> j) & 1ull) << pos[j];
    return r;
}

// The split mode of the planes a GEMM of kernel form KIND writes for the
// next step of the same form: 1 bf16 hi/lo, 2 tf32 hi/lo, 3 scaled fp16, 4
// scaled fp16 hi/lo; 5-7 the 3M modes of 1, 2 and 4 (a third value re + im).
__host__ __device__ constexpr int planar_mode_of(int kind, bool m3) {
    return kind == kBF16 ? (m3 ? 5 : 1) : kind == kTF32 ? (m3 ? 6 : 2) : kind == kFP16 ? 3 : (m3 ? 7 : 4);
}

// Pieces of two values x0, x1 that the epilogue has already scaled (the
// scaled modes' 2^-e is folded into the accumulator scale): round to
// nearest hi = piece(x), lo = piece(x - hi), as the split pass rounds them.
// 16-bit modes pack the two values' pieces into one word each (x0 low).
template <int MODE>
__device__ __forceinline__ void pieces_pair16(float x0, float x1, uint32_t &hi, uint32_t &lo) {
    if constexpr (mode_base(MODE) == 1) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    } else {
        const __half2 h = __floats2half2_rn(x0, x1);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        if constexpr (mode_base(MODE) == 4) {
            const float2 hf = __half22float2(h);
            const __half2 l = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
            lo = *reinterpret_cast<const uint32_t *>(&l);
        } else {
            lo = 0u;
        }
    }
}

// the values an element contributes to the planes: re, im (and re + im for
// the 3M modes)
template <int MODE>
__device__ __forceinline__ float value_of(float2 v, int c) {
    return c == 0 ? v.x : (c == 1 ? v.y : v.x + v.y);
}

template <int MODE>
struct PlaneShape {
    static constexpr int kValues = mode_3m(MODE) ? 3 : 2;     // values per element
    static constexpr int kPieces = MODE == 3 ? 1 : 2;         // hi (and lo) per value; plane q =
                                                              // piece * kValues + value
    static constexpr bool kWord = mode_word(MODE);            // 32-bit (tf32) pieces
};

// Store the pieces of n (1, 2 or 4) neighbouring elements v[0 .. n) at plane
// offset d (a multiple of n) of every plane.
template <int MODE, int NE>
__device__ __forceinline__ void plane_store(const TcPlanarOut &o, uint64_t d, const float2 *v) {
    using PS = PlaneShape<MODE>;
    if constexpr (PS::kWord) {
        uint32_t *P = reinterpret_cast<uint32_t *>(o.planes) + d;
#pragma unroll
        for (int c = 0; c < PS::kValues; c++) {
            uint32_t hi[NE], lo[NE];
#pragma unroll
            for (int e = 0; e < NE; e++) {
                const float x = value_of<MODE>(v[e], c);
                hi[e] = tf32_rna(x);
                lo[e] = tf32_rna(x - __uint_as_float(hi[e]));
            }
            uint32_t *Ph = P + (int64_t)c * o.plane_stride, *Pl = P + (int64_t)(PS::kValues + c) * o.plane_stride;
            if constexpr (NE == 4) {
                *reinterpret_cast<uint4 *>(Ph) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                *reinterpret_cast<uint4 *>(Pl) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
            } else if constexpr (NE == 2) {
                *reinterpret_cast<uint2 *>(Ph) = make_uint2(hi[0], hi[1]);
                *reinterpret_cast<uint2 *>(Pl) = make_uint2(lo[0], lo[1]);
            } else {
                *Ph = hi[0];
                *Pl = lo[0];
            }
        }
    } else {
        uint16_t *P = reinterpret_cast<uint16_t *>(o.planes) + d;
#pragma unroll
        for (int c = 0; c < PS::kValues; c++) {
            uint16_t *Ph = P + (int64_t)c * o.plane_stride;
            uint16_t *Pl = P + (int64_t)(PS::kValues + c) * o.plane_stride;
            if constexpr (NE == 1) {
                uint32_t hi, lo;
                pieces_pair16<MODE>(value_of<MODE>(v[0], c), 0.f, hi, lo);
                *Ph = (uint16_t)hi;
                if constexpr (PS::kPieces == 2) *Pl = (uint16_t)lo;
            } else {
                uint32_t hi[NE / 2], lo[NE / 2];
#pragma unroll
                for (int e = 0; e < NE / 2; e++)
                    pieces_pair16<MODE>(value_of<MODE>(v[2 * e], c), value_of<MODE>(v[2 * e + 1], c), hi[e], lo[e]);
                if constexpr (NE == 4) {
                    *reinterpret_cast<uint2 *>(Ph) = make_uint2(hi[0], hi[1]);
                    if constexpr (PS::kPieces == 2) *reinterpret_cast<uint2 *>(Pl) = make_uint2(lo[0], lo[1]);
                } else {
                    *reinterpret_cast<uint32_t *>(Ph) = hi[0];
                    if constexpr (PS::kPieces == 2) *reinterpret_cast<uint32_t *>(Pl) = lo[0];
                }
            }
        }
    }
}

// NW consecutive 32-bit words to p (16-byte aligned for NW >= 4, 8-byte for 2)
template <int NW>
__device__ __forceinline__ void store_words(void *p, const uint32_t *w) {
    if constexpr (NW == 1) {
        *reinterpret_cast<uint32_t *>(p) = w[0];
    } else if constexpr (NW == 2) {
        *reinterpret_cast<uint2 *>(p) = make_uint2(w[0], w[1]);
    } else {
#pragma unroll
        for (int i = 0; i < NW / 4; i++)
            reinterpret_cast<uint4 *>(p)[i] = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
    }
}

// Direct planar store of one lane's KCW columns of its row (re[], im[], the
// values already scaled for the planes): the columns form KCW / R runs of R
// consecutive destination elements (the destination's lowest log2 R bits
// are the tile's lowest column bits); run_off4[v] is the destination offset
// of the lane's columns 4v .. 4v + 3 relative to rbase.
template <int MODE, int KCW, int R>
__device__ __forceinline__ void direct_store(const TcPlanarOut &o, uint64_t rbase, const uint32_t *run_off4,
                                             const float *re, const float *im) {
    using PS = PlaneShape<MODE>;
#pragma unroll
    for (int u = 0; u < KCW / R; u++) {
        const uint64_t d = rbase + run_off4[u * (R / 4)];
#pragma unroll
        for (int c = 0; c < PS::kValues; c++) {
            if constexpr (PS::kWord) {
                uint32_t hi[R], lo[R];
#pragma unroll
                for (int e = 0; e < R; e++) {
                    const int i = u * R + e;
                    const float x = c == 0 ? re[i] : (c == 1 ? im[i] : re[i] + im[i]);
                    hi[e] = tf32_rna(x);
                    lo[e] = tf32_rna(x - __uint_as_float(hi[e]));
                }
                uint32_t *P = reinterpret_cast<uint32_t *>(o.planes) + d;
                store_words<R>(P + (int64_t)c * o.plane_stride, hi);
                store_words<R>(P + (int64_t)(PS::kValues + c) * o.plane_stride, lo);
            } else {
                uint32_t hi[R / 2], lo[R / 2];
#pragma unroll
                for (int e = 0; e < R / 2; e++) {
                    const int i = u * R + 2 * e;
                    const float x0 = c == 0 ? re[i] : (c == 1 ? im[i] : re[i] + im[i]);
                    const float x1 = c == 0 ? re[i + 1] : (c == 1 ? im[i + 1] : re[i + 1] + im[i + 1]);
                    pieces_pair16<MODE>(x0, x1, hi[e], lo[e]);
                }
                uint16_t *P = reinterpret_cast<uint16_t *>(o.planes) + d;
                store_words<R / 2>(P + (int64_t)c * o.plane_stride, hi);
                if constexpr (PS::kPieces == 2) store_words<R / 2>(P + (int64_t)(PS::kValues + c) * o.plane_stride, lo);
            }
        }
    }
}

// Planar epilogue tables.  The half tile's elements are enumerated in
// destination order j = (j_hi, j_lo): j_lo (6 bits; 7 for quads) is lane
// k l + q (k = 2 elements per lane, or 4 when the destination's two lowest
// bits both come from the tile), j_hi a group.  Per lane: stage and
// destination offsets of its j_lo; per group (shared memory, computed once
// per launch): those of j_hi.
struct PlanarLane {
    int s[4];       // staging offset (row * RS + column)
    uint32_t d[4];  // destination offset
    bool pair;      // d[1] = d[0] + 1 with d[0] even: one vector store per plane
    bool quad;      // d[q] = d[0] + q with d[0] a multiple of 4
};

__device__ __forceinline__ bool planar_quad(const TcPlanarOut &o) {
    return o.ntb >= 7 && o.tpos[0] == 0 && o.tpos[1] == 1;
}
__device__ __forceinline__ int planar_nlo(const TcPlanarOut &o) {
    return planar_quad(o) ? 7 : (o.ntb < 6 ? o.ntb : 6);
}

__device__ __forceinline__ void planar_bits(const TcPlanarOut &o, int j, int k0, int k1, int RS, int &so,
                                            uint32_t &d) {
    int r = 0, c = 0;
    d = 0;
    for (int k = k0; k < k1; k++)
        if ((j >> (k - k0)) & 1) {
            const int b = o.tb[k];
            if (b < 6) c |= 1 << b;
            else r |= 1 << (b - 6);
            d |= 1u << o.tpos[k];
        }
    so = r * RS + c;
}

__device__ __forceinline__ PlanarLane planar_lane(const TcPlanarOut &o, int lane, int RS) {
    PlanarLane L;
    const int nlo = planar_nlo(o);
    L.quad = planar_quad(o);
    const int per = L.quad ? 4 : 2;
    for (int q = 0; q < 4; q++) {
        L.s[q] = 0;
        L.d[q] = 0;
        if (q < per) planar_bits(o, per * lane + q, 0, nlo, RS, L.s[q], L.d[q]);
    }
    L.pair = o.ntb >= 6 && o.tpos[0] == 0;
    return L;
}

// Split the staged half tile (rows mh .. mh + 63) into the next step's
// planes: epilogue warp fw takes the groups j_hi = fw, fw + EW, ...; each
// lane two (or four) neighbouring elements of a group.  The staged values
// are already scaled for the planes.  base = the destination offset of the
// half tile's element (0, 0).
template <int MODE, int EW>
__device__ __forceinline__ void planar_write(const TcPlanarOut &o, uint64_t base, const float2 *st,
                                             const uint2 *jtab, const PlanarLane &L, int fw, int lane) {
    const int nlo = planar_nlo(o);
    const int n_hi = 1 << (o.ntb - nlo);
    if (L.quad) {
        for (int jh = fw; jh < n_hi; jh += EW) {
            const uint2 g = jtab[jh];
            float2 v[4];
            // (8-byte reads: two 16-byte reads of row neighbours measured
            // slower on the 53-qubit step's staged GEMM)
#pragma unroll
            for (int q = 0; q < 4; q++) v[q] = st[(int)g.x + L.s[q]];
            plane_store<MODE, 4>(o, base + g.y + L.d[0], v);  // offset a multiple of 4
        }
        return;
    }
    const bool v1 = 2 * lane + 1 < (1 << nlo), v0 = 2 * lane < (1 << nlo);
    for (int jh = fw; jh < n_hi; jh += EW) {
        const uint2 g = jtab[jh];
        float2 v[2];
        v[0] = st[(int)g.x + L.s[0]];
        v[1] = st[(int)g.x + L.s[1]];
        if (L.pair) {
            plane_store<MODE, 2>(o, base + g.y + L.d[0], v);
        } else {
            if (v0) plane_store<MODE, 1>(o, base + g.y + L.d[0], v);
            if (v1) plane_store<MODE, 1>(o, base + g.y + L.d[1], v + 1);
        }
    }
}

template <int KIND, int CB, bool M3, int EW>
__global__ void __launch_bounds__(ep_threads(EW), 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   const __grid_constant__ CUtensorMap mapC, const GemmTcParams p) {
    constexpr int kFlushWarps = EW;
    constexpr int kCW = TN / (EW / 4);  // complex columns per epilogue warp
    constexpr int NP = M3 ? 6 : (kind_split(KIND) ? 4 : 2);
    using R = Ring<CB, NP>;
    constexpr int kAPlane = R::kAPlane, kBPlane = R::kBPlane;
    constexpr int kStageBytes = R::kStageBytes, kStages = R::kStages;
    const int F = p.flush_chunks;
    // the TMA-stored planar output reuses the staging area: four planes of
    // 8 KB, 1024-byte aligned (128-byte swizzle)
    static_assert(4 * kTmaPlaneBytes <= R::kOutBytes && (kStages * kStageBytes) % 1024 == 0, "TMA staging");
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float2 *stage_out = reinterpret_cast<float2 *>(smem + kStages * kStageBytes);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + kStages * kStageBytes + R::kOutBytes);
    uint64_t *full = bar, *empty = bar + kStages, *tfull = bar + 2 * kStages, *tempty = bar + 2 * kStages + 2;
    uint64_t *drain = bar + 2 * kStages + 4;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 2 * kStages + 5);
    uint2 *jtab = reinterpret_cast<uint2 *>(smem + kStages * kStageBytes + R::kOutBytes + 256);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; s++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])));
        }
        for (int t = 0; t < 2; t++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tfull[t])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&tempty[t])), "r"(kFlushWarps));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(drain)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer: every chunk of every tile of this CTA
        if (lane == 0) {
            int cc = 0;  // chunks loaded so far (ring position)
            bool ok = true;
            for (int64_t tile = blockIdx.x; ok && tile < p.tiles; tile += gridDim.x) {
                const TileCoord tc = tile_coord(p, tile);
                int c_begin;
                const int n_chunks = part_chunks(p, tc.part, c_begin);
                for (int c = 0; c < n_chunks; c++, cc++) {
                    const int s = cc % kStages, use = cc / kStages;
                    if (use > 0 && !mbar_wait(smem_u32(&empty[s]), (use - 1) & 1)) { ok = false; break; }
                    unsigned char *st = smem + s * kStageBytes;
                    const uint32_t fb = smem_u32(&full[s]);
                    mbar_expect_tx(fb, kStageBytes);
                    const int kc = (c_begin + c) * p.k_chunk;
                    const int klo = kc & ((1 << p.klo_bits) - 1), khi = kc >> p.klo_bits;
                    tma_load_5d(smem_u32(st), &mapA, klo, (int)tc.m0, khi, tc.h, 0, fb);
                    tma_load_5d(smem_u32(st + NP * kAPlane), &mapB, klo, (int)tc.n0, khi, tc.h, 0, fb);
                }
            }
            // let every issued load land before the CTA can exit (a no-op
            // when the consumer has seen them all)
            for (int s = 0; s < kStages && s < cc; s++) {
                const int uses = (cc - s + kStages - 1) / kStages;
                mbar_drain(smem_u32(&full[s]), (uses - 1) & 1);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t fmt = KIND == kTF32 ? 2u : (KIND == kBF16 ? 1u : 0u);  // tf32 / bf16 / f16
            constexpr uint32_t ID = make_idesc(fmt, TM, 2 * TN, false);
            int cc = 0, gc = 0;  // chunks consumed, read-out groups started
            bool ok = true;
            for (int64_t tile = blockIdx.x; ok && tile < p.tiles; tile += gridDim.x) {
                int c_begin;
                const int n_chunks = part_chunks(p, tile_coord(p, tile).part, c_begin);
                for (int c = 0; c < n_chunks; c++, cc++) {
                    const int s = cc % kStages, use = cc / kStages;
                    const int g = gc + c / F;  // read-out group (never spans two tiles)
                    const int t = g & 1, tuse = g >> 1;
                    const bool first = (c % F) == 0;
                    const bool last = (c % F) == F - 1 || c == n_chunks - 1;
                    if (!mbar_wait(smem_u32(&full[s]), use & 1)) { ok = false; break; }
                    if (first && tuse > 0 && !mbar_wait(smem_u32(&tempty[t]), (tuse - 1) & 1)) { ok = false; break; }
                    fence_after();
                    const uint32_t a0 = smem_u32(smem + s * kStageBytes), b0 = a0 + NP * kAPlane;
                    if constexpr (M3) {
                        // 3M: T1 = A_re B_re, T2 = A_im B_im, T3 = A_s B_s (s = re + im),
                        // each from the hi*hi, hi*lo and lo*hi piece products, N = 64
                        constexpr uint32_t ID3 = make_idesc(fmt, TM, TN, false);
                        const uint32_t d1 = tmem + t * 256;
#pragma unroll
                        for (int ks = 0; ks < CB / 32; ks++) {
                            const uint32_t ko = ks * 32;
                            const uint32_t acc = (first && ks == 0) ? 0u : 1u;
#pragma unroll
                            for (int pr = 0; pr < 3; pr++) {
                                const uint32_t dd = d1 + pr * TN;
                                const uint64_t ah = make_desc<CB>(a0 + pr * kAPlane + ko);
                                const uint64_t al = make_desc<CB>(a0 + (pr + 3) * kAPlane + ko);
                                const uint64_t bh = make_desc<CB>(b0 + pr * kBPlane + ko);
                                const uint64_t bl = make_desc<CB>(b0 + (pr + 3) * kBPlane + ko);
                                mma<KIND>(dd, ah, bh, ID3, acc);
                                mma<KIND>(dd, ah, bl, ID3, 1u);
                                mma<KIND>(dd, al, bh, ID3, 1u);
                            }
                        }
                        mma_commit(smem_u32(&empty[s]));
                        if (last) mma_commit(smem_u32(&tfull[t]));
                        continue;
                    }
                    const uint32_t dP = tmem + t * 256, dQ = dP + 128;
#pragma unroll
                    for (int ks = 0; ks < CB / 32; ks++) {  // MMA K steps of 32 bytes
                        const uint32_t ko = ks * 32;
                        const uint32_t acc = (first && ks == 0) ? 0u : 1u;  // each group starts fresh sums
                        const uint64_t ar = make_desc<CB>(a0 + ko), ai = make_desc<CB>(a0 + kAPlane + ko);
                        const uint64_t S = make_desc<CB>(b0 + ko);  // [re | im] of the (hi) piece
                        mma<KIND>(dP, ar, S, ID, acc);
                        mma<KIND>(dQ, ai, S, ID, acc);
                        if (kind_split(KIND)) {
                            // corrections hi*lo + lo*hi into the same sums
                            const uint64_t arl = make_desc<CB>(a0 + 2 * kAPlane + ko);
                            const uint64_t ail = make_desc<CB>(a0 + 3 * kAPlane + ko);
                            const uint64_t Sl = make_desc<CB>(b0 + 2 * kBPlane + ko);
                            mma<KIND>(dP, ar, Sl, ID, 1u);
                            mma<KIND>(dP, arl, S, ID, 1u);
                            mma<KIND>(dQ, ai, Sl, ID, 1u);
                            mma<KIND>(dQ, ail, S, ID, 1u);
                        }
                    }
                    mma_commit(smem_u32(&empty[s]));
                    if (last) mma_commit(smem_u32(&tfull[t]));
                }
                gc += (n_chunks + F - 1) / F;
            }
            // every MMA issued has completed before the tensor memory is freed
            if (cc > 0) {
                mma_commit(smem_u32(drain));
                mbar_drain(smem_u32(drain), 0);
            }
        }
    } else if (warp >= kFlushWarp0) {
        // ---------------- accumulator read-out + epilogue (16 warps)
        const int fw = warp - kFlushWarp0;
        const int lg = warp & 3, cq = fw >> 2;  // TMEM lane group, column quarter
        const uint32_t lane_off = (uint32_t)(lg * 32) << 16;
        int e_scale = 0;
        if (kind_scaled(KIND))
            e_scale = fp16s_exponent(__uint_as_float(p.scales[0])) + fp16s_exponent(__uint_as_float(p.scales[1]));
        // Scaled planar output (modes 3, 4): the planes' exponent comes from a
        // bound, since the output's max is known only after the last tile.
        // With the operands' true maxima below 2^(tA + 14) and 2^(tB + 14)
        // (tA, tB their scale exponents), a component of C is below
        // 2K 2^(tA + 14) 2^(tB + 14), so e_out = tA + tB + 15 + ceil(log2 K)
        // keeps every scaled value below 2^14.  The next step reads e_out
        // from the max slot (2^(e_out + 13)) and the output's true max from
        // the slot two places on, so the bound never builds on another bound.
        int e_out = 0;
        if (kind_scaled(KIND) && mode_scaled(p.out.mode)) {
            int lk = 0;
            while (((int64_t)1 << lk) < p.K) lk++;
            float mA = __uint_as_float(p.scales[2]), mB = __uint_as_float(p.scales[3]);
            if (!(mA > 0.f)) mA = __uint_as_float(p.scales[0]);
            if (!(mB > 0.f)) mB = __uint_as_float(p.scales[1]);
            e_out = fp16s_exponent(mA) + fp16s_exponent(mB) + 15 + lk;
        }
        // accumulator scale 2^(e_scale - e_out) as one or two normal powers of two
        const int e_acc = e_scale - e_out;
        const int e_1 = (e_acc >= -126 && e_acc <= 127) ? e_acc : e_acc / 2;
        const float sc1 = __int_as_float((127 + e_1) << 23), sc2 = __int_as_float((127 + e_acc - e_1) << 23);
        float run_max = 0.f;
        // every flush warp walks every tile of this CTA and reaches the same
        // named barriers even after a failed wait (it then skips waits,
        // tensor-memory reads and stores), so the warps never part ways
        // direct planar store: the destination offset of this lane's row
        // (TMEM lane = tile row) and of its columns' 4-element runs
        constexpr int kRuns4 = kCW / 4;
        uint32_t run_off4[kRuns4];
        uint64_t row_off = 0;
        if (p.direct_run > 0) {
            const int row = lg * 32 + lane;
#pragma unroll
            for (int v = 0; v < kRuns4; v++) run_off4[v] = 0;
            for (int k = 0; k < p.out.ntb; k++) {
                const int b = p.out.tb[k];
                if (b >= 6) {
                    if ((row >> (b - 6)) & 1) row_off |= 1ull << p.out.tpos[k];
                } else {
#pragma unroll
                    for (int v = 0; v < kRuns4; v++)
                        if (((cq * kCW + 4 * v) >> b) & 1) run_off4[v] |= 1u << p.out.tpos[k];
                }
            }
            if (row >> 6) row_off |= 1ull << p.out.mpos[6];
        }
        PlanarLane pl;
        if (p.out.mode != 0) {
            pl = planar_lane(p.out, lane, R::kOutRS);
            const int nlo = planar_nlo(p.out);
            for (int jh = fw * 32 + lane; jh < (1 << (p.out.ntb - nlo)); jh += kFlushWarps * 32) {
                int so;
                uint32_t d;
                planar_bits(p.out, jh, nlo, p.out.ntb, R::kOutRS, so, d);
                jtab[jh] = make_uint2((uint32_t)so, d);
            }
            // published to the other epilogue warps by the first staging barrier
        }
        int gc = 0;
        bool ok = true;
        for (int64_t tile = blockIdx.x; tile < p.tiles; tile += gridDim.x) {
            const TileCoord tc = tile_coord(p, tile);
            int c_begin;
            const int n_chunks = part_chunks(p, tc.part, c_begin);
            float acc_re[kCW], acc_im[kCW];
#pragma unroll
            for (int j = 0; j < kCW; j++) acc_re[j] = acc_im[j] = 0.f;
            const int n_groups = (n_chunks + F - 1) / F;
            for (int gi = 0; gi < n_groups; gi++, gc++) {
                const int t = gc & 1, tuse = gc >> 1;
                if (ok && !mbar_wait(smem_u32(&tfull[t]), tuse & 1)) ok = false;
                // one outcome per warp: the tensor-memory loads below are
                // warp-collective (.sync.aligned)
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) continue;
                fence_after();
                const uint32_t base = tmem + t * 256 + lane_off + cq * kCW;
                if constexpr (M3) {
#pragma unroll
                    for (int q = 0; q < kCW / 16; q++) {
                        uint32_t r0[16], r1[16], r2[16];
                        tmem_ld16(base + q * 16, r0);             // T1 = A_re B_re
                        tmem_ld16(base + TN + q * 16, r1);        // T2 = A_im B_im
                        tmem_ld16(base + 2 * TN + q * 16, r2);    // T3 = (A_re + A_im)(B_re + B_im)
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 16; j++) {
                            const float t1 = __uint_as_float(r0[j]), t2 = __uint_as_float(r1[j]);
                            acc_re[q * 16 + j] += t1 - t2;
                            acc_im[q * 16 + j] += __uint_as_float(r2[j]) - (t1 + t2);
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < (M3 ? 0 : kCW / 16); q++) {
                    // real parts, then imaginary parts: two loads in flight at
                    // a time keep the epilogue within its register budget
                    uint32_t r0[16], r1[16];
                    tmem_ld16(base + q * 16, r0);        // P left:  A_re B_re
                    tmem_ld16(base + 192 + q * 16, r1);  // Q right: A_im B_im
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 16; j++) acc_re[q * 16 + j] += __uint_as_float(r0[j]) - __uint_as_float(r1[j]);
                    tmem_ld16(base + 64 + q * 16, r0);   // P right: A_re B_im
                    tmem_ld16(base + 128 + q * 16, r1);  // Q left:  A_im B_re
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 16; j++) acc_im[q * 16 + j] += __uint_as_float(r0[j]) + __uint_as_float(r1[j]);
                }
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&tempty[t]));
            }
            if (kind_scaled(KIND)) {
                // undo the operands' power-of-two scales and, for scaled
                // planes, apply the planes' 2^-e_out in the same product
                // (exact: a product with a normal power of two; outside the
                // normal range two such products, exact while the
                // intermediate stays normal)
#pragma unroll
                for (int j = 0; j < kCW; j++) {
                    acc_re[j] *= sc1;
                    acc_im[j] *= sc1;
                }
                if (sc2 != 1.f) {
#pragma unroll
                    for (int j = 0; j < kCW; j++) {
                        acc_re[j] *= sc2;
                        acc_im[j] *= sc2;
                    }
                }
            }
            if (p.max_slot && ok) {
                // running max |re|, |im| of the values written (rows and
                // columns past the edge hold zeros: their operand rows were
                // zero-filled); published once per warp after the last tile
#pragma unroll
                for (int j = 0; j < kCW; j++) run_max = fmaxf(run_max, fmaxf(fabsf(acc_re[j]), fabsf(acc_im[j])));
            }
            float2 *Ch = p.C + (int64_t)tc.h * p.sCh;
            if (p.ksplit > 1) {
                // partial K range: add into the zeroed output
                const int64_t m = tc.m0 + lg * 32 + lane;
                if (ok && m < p.M && n_chunks > 0) {
#pragma unroll
                    for (int j = 0; j < kCW; j++) {
                        const int64_t n = tc.n0 + cq * kCW + j;
                        if (n < p.N) atomicAdd(Ch + m * p.sCm + n * p.sCn, make_float2(acc_re[j], acc_im[j]));
                    }
                }
                continue;
            }
            // stage half a tile (64 rows) at a time, then write whole rows: a
            // warp stores one 512-byte row per instruction
            constexpr int RS = R::kOutRS;
            // planar output: destination offset of the tile's element (0, 0)
            const uint64_t pbase = p.out.mode != 0 ? (scatter8((uint64_t)tc.h, p.out.hpos, p.out.nH) |
                                                      scatter8((uint64_t)tc.m0, p.out.mpos, p.out.nM) |
                                                      scatter8((uint64_t)tc.n0, p.out.npos, p.out.nN))
                                                   : 0;
            constexpr int kMode = planar_mode_of(KIND, M3);
            if constexpr (!mode_word(kMode) && !mode_3m(kMode) && EW == 8) {
                if (p.tma.on) {
                    // planar output by TMA (full tiles, 16-bit planes): per
                    // half tile, the writing lanes put their rows' pieces in
                    // shared memory in the order of the destination box
                    // (128-byte rows, 128-byte swizzle: the 16-byte chunk
                    // index is XORed with the row index mod 8), then one
                    // thread stores each plane's box with one bulk tensor
                    // copy.  Every epilogue warp reaches both barriers of
                    // each half.
                    using PS = PlaneShape<kMode>;
                    const bool issuer = fw == 0 && lane == 0;
                    const int r = (lg & 1) * 32 + lane;  // row within the half tile
                    uint32_t erow = 0;
#pragma unroll
                    for (int i = 0; i < 6; i++) erow |= (uint32_t)((r >> i) & 1) << p.tma.boxbit[6 + i];
                    const uint32_t sbase = smem_u32(stage_out);
#pragma unroll
                    for (int hp = 0; hp < 2; hp++) {
                        if (issuer) bulk_wait_read();  // the previous boxes have left shared memory
                        asm volatile("bar.sync 1, %0;" ::"n"(32 * kFlushWarps) : "memory");
                        if ((lg >> 1) == hp && ok) {
#pragma unroll
                            for (int u = 0; u < kCW / 8; u++) {
                                // eight columns c0..c2 = 0..7: 16 consecutive bytes of the box
                                const int col0 = cq * kCW + 8 * u;
                                uint32_t e = erow;
#pragma unroll
                                for (int i = 3; i < 6; i++) e |= (uint32_t)((col0 >> i) & 1) << p.tma.boxbit[i];
                                const uint32_t o = 2u * e;
                                const uint32_t sw = o ^ (((o >> 7) & 7u) << 4);
#pragma unroll
                                for (int c = 0; c < PS::kValues; c++) {
                                    uint32_t hi[4], lo[4];
#pragma unroll
                                    for (int w = 0; w < 4; w++) {
                                        const int j = 8 * u + 2 * w;
                                        pieces_pair16<kMode>(c == 0 ? acc_re[j] : acc_im[j],
                                                             c == 0 ? acc_re[j + 1] : acc_im[j + 1], hi[w], lo[w]);
                                    }
                                    st_shared_v4(sbase + c * kTmaPlaneBytes + sw, hi);
                                    if constexpr (PS::kPieces == 2)
                                        st_shared_v4(sbase + (PS::kValues + c) * kTmaPlaneBytes + sw, lo);
                                }
                            }
                            fence_proxy_async();
                        }
                        asm volatile("bar.sync 1, %0;" ::"n"(32 * kFlushWarps) : "memory");
                        if (issuer && ok) {
                            // box coordinates: the half tile's destination
                            // base cut into the dimensions' bit fields (its
                            // tile bits are zero: every coordinate is a
                            // whole box, the innermost one 0)
                            const uint64_t db = hp ? (pbase | (1ull << p.out.mpos[6])) : pbase;
                            int crd[5];
#pragma unroll
                            for (int i = 0; i < 5; i++) {
                                const uint64_t f = i < p.tma.nd ? (db >> p.tma.start[i]) : 0;
                                crd[i] = (int)(i < p.tma.nd - 1 ? (f & ((1ull << p.tma.bits[i]) - 1)) : f);
                            }
                            for (int q = 0; q < p.tma.np; q++) {
                                int cq5[5] = {crd[0], crd[1], crd[2], crd[3], crd[4]};
                                cq5[p.tma.nd - 1] += (int)(q * p.tma.plane_step);
                                tma_store_5d(&mapC, sbase + q * kTmaPlaneBytes, cq5[0], cq5[1], cq5[2], cq5[3],
                                             cq5[4]);
                            }
                            bulk_commit();
                        }
                    }
                    continue;
                }
            }
            if (p.direct_run > 0) {
                // full tiles only (the launcher checks M and N): every lane
                // stores its own row's columns, no staging
                if (ok) {
                    constexpr int MODE = planar_mode_of(KIND, M3);
                    const uint64_t rb = pbase + row_off;
                    direct_store<MODE, kCW, mode_word(MODE) ? 4 : 8>(p.out, rb, run_off4, acc_re, acc_im);
                }
                continue;
            }
#pragma unroll
            for (int hp = 0; hp < 2; hp++) {
                if ((lg >> 1) == hp) {
                    // two complex values per 16-byte store (rows are 528 bytes
                    // apart: eight lanes cover the 32 banks, no conflicts)
                    const int r = (lg & 1) * 32 + lane;
                    float4 *row4 = reinterpret_cast<float4 *>(stage_out + r * RS + cq * kCW);
#pragma unroll
                    for (int j = 0; j < kCW; j += 2)
                        row4[j >> 1] = make_float4(acc_re[j], acc_im[j], acc_re[j + 1], acc_im[j + 1]);
                }
                asm volatile("bar.sync 1, %0;" ::"n"(32 * kFlushWarps) : "memory");
                if (p.out.mode != 0) {
                    // m bit 6 is the half (m0 is a multiple of 128); with
                    // M <= 64 the second half lies past M and is skipped
                    if (ok && tc.m0 + hp * (TM / 2) < p.M)
                        planar_write<planar_mode_of(KIND, M3), EW>(
                            p.out, hp ? (pbase | (1ull << p.out.mpos[6])) : pbase, stage_out, jtab, pl, fw, lane);
                }
                for (int rr = fw; ok && p.out.mode == 0 && rr < TM / 2; rr += kFlushWarps) {
                    const int64_t mm = tc.m0 + hp * (TM / 2) + rr;
                    if (mm >= p.M) break;
                    const int64_t n = tc.n0 + 2 * lane;
                    float2 *dst = Ch + mm * p.sCm;
                    if (p.sCn == 1 && n + 1 < p.N) {
                        const float4 v = *reinterpret_cast<const float4 *>(stage_out + rr * RS + 2 * lane);
                        *reinterpret_cast<float4 *>(dst + n) = v;
                    } else {
                        if (n < p.N) dst[n * p.sCn] = stage_out[rr * RS + 2 * lane];
                        if (n + 1 < p.N) dst[(n + 1) * p.sCn] = stage_out[rr * RS + 2 * lane + 1];
                    }
                }
                asm volatile("bar.sync 1, %0;" ::"n"(32 * kFlushWarps) : "memory");
            }
        }
        // the planes' last boxes are written before the CTA exits
        if (p.tma.on && fw == 0 && lane == 0) bulk_wait_all();
        if (p.max_slot && ok) {
            // one atomic per warp and launch; non-negative floats order like
            // their bit patterns
            float mx = run_max;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
            if (lane == 0) {
                if (mode_scaled(p.out.mode)) {
                    // the written values carry 2^-e_out: the output's true max
                    // (exact), and the planes' exponent for the next step
                    atomicMax(p.max_slot + 2, __float_as_uint(ldexpf(mx, e_out)));
                    atomicMax(p.max_slot, __float_as_uint(ldexpf(1.f, e_out + 13)));
                } else {
                    atomicMax(p.max_slot, __float_as_uint(mx));
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

// ------------------------------------------- small step on the tensor cores
// A small step C[r, n] = sum_k T[r, k] S[k, n] (S of K x N values, K and N of
// 16 or 32; T and C with their rows' 7 lowest bits at their 7 lowest
// positions, so every (k, 128-row tile) of T and (n, tile) of C is 1 KB of
// consecutive memory) with the split of T into pieces done in shared memory:
// no split pass over T, and the complex multiply-adds on the tensor cores
// instead of the CUDA cores' FP32 pipe.  One CTA of 256 threads walks
// 128-row tiles: cp.async brings the next tile's T while the current one is
// split (per tile: FP16X3 scales the tile by 2^-e_t, e_t from its own
// largest |re|, |im|, which is exact because every row of C depends on its
// own row of T only), multiplied (P = A_re [S_re | S_im], Q = A_im [S_re |
// S_im], three piece products each, one elected thread) and read back from
// tensor memory into C.  S is split once per CTA (FP16X3: scaled by its own
// max).  Pieces, products and the FP32 read-out are those of the GEMM, so
// the step has the GEMM's accuracy.
struct SmallTcParams {
    const float2 *T;
    const float2 *S;
    float2 *C;
    int64_t tiles;  // rows / 128
    int nK, nN;
    int n_tins, n_cins;
    int tins[kSmallMaxBits], cins[kSmallMaxBits];
    uint64_t offT[32];  // T offset of k
    uint64_t offC[32];  // C offset of n
    uint32_t offS[32 * 32];  // S offset of (k, n): k * N + n
    unsigned *max_slot;  // optional: max |re|, |im| of C (float bits)
};

constexpr int kSmallTcThreads = 256;

__device__ __forceinline__ uint64_t small_tc_insert(uint64_t x, const int *pos, int n) {
    for (int i = 0; i < n; i++) {
        const int q = pos[i];
        x = ((x >> q) << (q + 1)) | (x & ((1ull << q) - 1));
    }
    return x;
}

// byte offset of (row, 16-byte chunk c) in a K-major operand of CB-byte rows
// with the CB-byte swizzle (the layout TMA writes and the MMA descriptors of
// make_desc<CB> read): address bits 4.. XOR address bits 7..
template <int CB>
__device__ __forceinline__ uint32_t swz_off(int row, int c) {
    const uint32_t lin = (uint32_t)row * CB + (uint32_t)c * 16;
    constexpr uint32_t kMask = CB == 128 ? 7u : (CB == 64 ? 3u : 1u);
    return lin ^ (((lin >> 7) & kMask) << 4);
}

// pieces of 8 consecutive K values x[0..7] of one row into the hi and lo
// words of one 16-byte chunk (16-bit pieces: 8 values; tf32: 4 values use
// words 0..3 of hi/lo, the caller passes them in two halves)
template <int KIND>
__device__ __forceinline__ void small_tc_pieces(const float *x, uint32_t *hi, uint32_t *lo) {
    if constexpr (KIND == kTF32) {
#pragma unroll
        for (int e = 0; e < 4; e++) {
            hi[e] = tf32_rna(x[e]);
            lo[e] = tf32_rna(x[e] - __uint_as_float(hi[e]));
        }
    } else {
#pragma unroll
        for (int e = 0; e < 4; e++) {
            if constexpr (KIND == kBF16) {
                const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * e], x[2 * e + 1]);
                const float2 hf = __bfloat1622float2(h);
                const __nv_bfloat162 l = __floats2bfloat162_rn(x[2 * e] - hf.x, x[2 * e + 1] - hf.y);
                hi[e] = *reinterpret_cast<const uint32_t *>(&h);
                lo[e] = *reinterpret_cast<const uint32_t *>(&l);
            } else {
                const __half2 h = __floats2half2_rn(x[2 * e], x[2 * e + 1]);
                const float2 hf = __half22float2(h);
                const __half2 l = __floats2half2_rn(x[2 * e] - hf.x, x[2 * e + 1] - hf.y);
                hi[e] = *reinterpret_cast<const uint32_t *>(&h);
                lo[e] = *reinterpret_cast<const uint32_t *>(&l);
            }
        }
    }
}

// Shared memory of the small-step kernel (CB = K bytes of a plane row,
// NK K values): T staging, two tiles of [k][128 rows] complex64; A planes
// (re_hi, im_hi, re_lo, im_lo) of 128 rows; B planes (hi, lo) of 2N rows
// ([S_re | S_im] transposed); tile scalars; barrier and tensor-memory slot.
template <int CB, int NK>
struct SmallTcSmem {
    static constexpr int kStage = NK * 128 * 8;
    static constexpr int kAPlane = 128 * CB;
    static constexpr int kBPlane = 64 * CB;  // up to 2N = 64 rows
    static constexpr int kA = 2 * kStage;                  // offsets (1024-aligned)
    static constexpr int kB = kA + 4 * kAPlane;
    static constexpr int kMisc = kB + 2 * kBPlane;
    static constexpr int kBytes = kMisc + 256 + 1024;      // + alignment slack
};

template <int KIND, int CB>
__global__ void __launch_bounds__(kSmallTcThreads, 2) small_tc_kernel(const SmallTcParams p) {
    constexpr int ES = KIND == kTF32 ? 4 : 2;  // piece bytes
    constexpr int NK = CB / ES;                 // K values (16 or 32)
    using L = SmallTcSmem<CB, NK>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float2 *stg = reinterpret_cast<float2 *>(smem);
    unsigned char *Ap = smem + L::kA, *Bp = smem + L::kB;
    float *red = reinterpret_cast<float *>(smem + L::kMisc);        // 8 warp maxima
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L::kMisc + 64);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + L::kMisc + 128);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NS = 1 << p.nN;
    constexpr uint32_t kCols = 128;  // P: 2N columns, Q: 2N columns (N <= 32)

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // S: largest |re|, |im| (FP16X3 scale), then its planes: B row n' < N is
    // S_re[., n'], row N + n' is S_im[., n'], K-major
    float smax = 0.f;
    for (int i = tid; i < NK * NS; i += kSmallTcThreads) {
        const float2 v = p.S[p.offS[i]];
        smax = fmaxf(smax, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, off));
    if (lane == 0) red[warp] = smax;
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    smax = 0.f;
#pragma unroll
    for (int w = 0; w < kSmallTcThreads / 32; w++) smax = fmaxf(smax, red[w]);
    const int eS = KIND == kFP16X3 ? fp16s_exponent(smax) : 0;
    for (int task = tid; task < 2 * NS * (NK / 8); task += kSmallTcThreads) {
        // one 16-byte chunk of 8 K values (4 for tf32: two chunks per 8) of B row
        const int row = task / (NK / 8), c8 = task % (NK / 8);
        const int n = row % NS;
        const bool im = row >= NS;
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; e++) {
            const float2 v = p.S[p.offS[(c8 * 8 + e) * NS + n]];
            const float y = im ? v.y : v.x;
            x[e] = KIND == kFP16X3 ? y * __int_as_float((127 - eS) << 23) : y;
        }
        uint32_t hi[8], lo[8];
        small_tc_pieces<KIND>(x, hi, lo);
        if constexpr (KIND == kTF32) {
            small_tc_pieces<KIND>(x + 4, hi + 4, lo + 4);
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const uint32_t o = swz_off<CB>(row, 2 * c8 + h);
                *reinterpret_cast<uint4 *>(Bp + o) = make_uint4(hi[4 * h], hi[4 * h + 1], hi[4 * h + 2], hi[4 * h + 3]);
                *reinterpret_cast<uint4 *>(Bp + L::kBPlane + o) =
                    make_uint4(lo[4 * h], lo[4 * h + 1], lo[4 * h + 2], lo[4 * h + 3]);
            }
        } else {
            const uint32_t o = swz_off<CB>(row, c8);
            *reinterpret_cast<uint4 *>(Bp + o) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4 *>(Bp + L::kBPlane + o) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
    }
    // T tile `tile` into stage `st`: element (k, i) at stg[st][k * 128 + i]
    auto issue = [&](int64_t tile, int st) {
        const uint64_t base = small_tc_insert((uint64_t)tile << 7, p.tins, p.n_tins);
        const uint32_t dst0 = smem_u32(stg + st * (NK * 128));
        for (int c = tid; c < NK * 64; c += kSmallTcThreads) {  // 16-byte pieces: 2 rows
            const int k = c >> 6, i2 = (c & 63) * 2;
            const float2 *src = p.T + base + p.offT[k] + i2;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst0 + (uint32_t)(k * 128 + i2) * 8),
                         "l"(src)
                         : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    const uint32_t idesc = make_idesc(KIND == kTF32 ? 2u : (KIND == kBF16 ? 1u : 0u), 128, 2 * NS, false);
    const int row = tid & 127, half = tid >> 7;  // conversion: one row, half of its K values
    const int lg = warp & 3, ch = warp >> 2;     // read-out: TMEM lane group, half of the N columns
    float cmax = 0.f;
    bool ok = true;
    int st = 0;
    uint32_t phase = 0;
    if ((int64_t)blockIdx.x < p.tiles) issue(blockIdx.x, 0);
    for (int64_t tile = blockIdx.x; tile < p.tiles; tile += gridDim.x) {
        const int64_t next = tile + gridDim.x;
        if (next < p.tiles) {
            issue(next, st ^ 1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        const float2 *T_s = stg + st * (NK * 128);
        // per-tile scale (FP16X3): largest |re|, |im| of the tile
        float x_re[NK / 2], x_im[NK / 2];
        float tmax = 0.f;
#pragma unroll
        for (int e = 0; e < NK / 2; e++) {
            const float2 v = T_s[(half * (NK / 2) + e) * 128 + row];
            x_re[e] = v.x;
            x_im[e] = v.y;
            tmax = fmaxf(tmax, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
        int eT = 0;
        if constexpr (KIND == kFP16X3) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, off));
            if (lane == 0) red[warp] = tmax;
            __syncthreads();
            tmax = 0.f;
#pragma unroll
            for (int w = 0; w < kSmallTcThreads / 32; w++) tmax = fmaxf(tmax, red[w]);
            eT = fp16s_exponent(tmax);
            const float sc = __int_as_float((127 - eT) << 23);
#pragma unroll
            for (int e = 0; e < NK / 2; e++) {
                x_re[e] *= sc;
                x_im[e] *= sc;
            }
        }
        // A planes: this thread's row, K values [half * NK / 2, + NK / 2)
#pragma unroll
        for (int c8 = 0; c8 < NK / 16; c8++) {
#pragma unroll
            for (int comp = 0; comp < 2; comp++) {
                const float *x = (comp ? x_im : x_re) + c8 * 8;
                uint32_t hi[8], lo[8];
                small_tc_pieces<KIND>(x, hi, lo);
                unsigned char *Ph = Ap + comp * L::kAPlane, *Pl = Ap + (2 + comp) * L::kAPlane;
                if constexpr (KIND == kTF32) {
                    small_tc_pieces<KIND>(x + 4, hi + 4, lo + 4);
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        const uint32_t o = swz_off<CB>(row, half * (NK / 8) + 2 * c8 + h);
                        *reinterpret_cast<uint4 *>(Ph + o) =
                            make_uint4(hi[4 * h], hi[4 * h + 1], hi[4 * h + 2], hi[4 * h + 3]);
                        *reinterpret_cast<uint4 *>(Pl + o) =
                            make_uint4(lo[4 * h], lo[4 * h + 1], lo[4 * h + 2], lo[4 * h + 3]);
                    }
                } else {
                    const uint32_t o = swz_off<CB>(row, half * (NK / 16) + c8);
                    *reinterpret_cast<uint4 *>(Ph + o) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                    *reinterpret_cast<uint4 *>(Pl + o) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                }
            }
        }
        // generic-proxy shared-memory writes, then the tensor core reads them
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        fence_before();
        __syncthreads();
        if (tid == 0) {
            fence_after();
            const uint32_t a0 = smem_u32(Ap), b0 = smem_u32(Bp);
            const uint32_t dP = tmem, dQ = tmem + 2 * NS;
#pragma unroll
            for (int ks = 0; ks < CB / 32; ks++) {
                const uint32_t ko = ks * 32;
                const uint64_t ar = make_desc<CB>(a0 + ko), ai = make_desc<CB>(a0 + L::kAPlane + ko);
                const uint64_t arl = make_desc<CB>(a0 + 2 * L::kAPlane + ko);
                const uint64_t ail = make_desc<CB>(a0 + 3 * L::kAPlane + ko);
                const uint64_t S = make_desc<CB>(b0 + ko), Sl = make_desc<CB>(b0 + L::kBPlane + ko);
                const uint32_t acc = ks == 0 ? 0u : 1u;
                mma<KIND>(dP, ar, S, idesc, acc);
                mma<KIND>(dQ, ai, S, idesc, acc);
                mma<KIND>(dP, ar, Sl, idesc, 1u);
                mma<KIND>(dP, arl, S, idesc, 1u);
                mma<KIND>(dQ, ai, Sl, idesc, 1u);
                mma<KIND>(dQ, ail, S, idesc, 1u);
            }
            mma_commit(smem_u32(bar));
        }
        // every thread waits for the products (bounded); one outcome for the
        // block: on expiry it stops after this tile (the products still in
        // flight are drained before the tensor memory is freed)
        if (!mbar_wait(smem_u32(bar), phase)) ok = false;
        ok = __syncthreads_and(ok) != 0;
        fence_after();
        if (ok) {
            phase ^= 1;
            // this warp: rows 32 lg .., columns n in [ch * N / 2, + N / 2)
            // (N = 8: all eight columns in the warps of ch 0)
            const uint32_t base = tmem + ((uint32_t)(lg * 32) << 16);
            const uint64_t cbase = small_tc_insert((uint64_t)tile << 7, p.cins, p.n_cins) + lg * 32 + lane;
            const float sc = KIND == kFP16X3 ? __int_as_float((127 + eT + eS) << 23) : 1.f;
            const int n_lo = NS >= 16 ? ch * (NS / 2) : (ch ? NS : 0);
            const int n_hi = NS >= 16 ? (ch + 1) * (NS / 2) : NS;
            for (int n0 = n_lo; n0 < n_hi; n0 += 8) {
                uint32_t pr[8], pi[8], qr[8], qi[8];
                tmem_ld8(base + n0, pr);           // P left:  A_re S_re
                tmem_ld8(base + NS + n0, pi);      // P right: A_re S_im
                tmem_ld8(base + 2 * NS + n0, qr);  // Q left:  A_im S_re
                tmem_ld8(base + 3 * NS + n0, qi);  // Q right: A_im S_im
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    const float re = (__uint_as_float(pr[j]) - __uint_as_float(qi[j])) * sc;
                    const float im = (__uint_as_float(pi[j]) + __uint_as_float(qr[j])) * sc;
                    p.C[cbase + p.offC[n0 + j]] = make_float2(re, im);
                    cmax = fmaxf(cmax, fmaxf(fabsf(re), fabsf(im)));
                }
            }
        }
        fence_before();
        __syncthreads();  // tensor memory read and A planes free for the next tile
        if (!ok) break;
        st ^= 1;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (!ok && tid == 0) mbar_drain(smem_u32(bar), phase);
    if (p.max_slot && ok) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) cmax = fmaxf(cmax, __shfl_xor_sync(0xffffffffu, cmax, off));
        if (lane == 0) atomicMax(p.max_slot, __float_as_uint(cmax));
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
    }
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// planes of element size es, plane-major as the split pass writes them:
// [np][H][K / Klo][rows][Klo] with Klo = 2^klo_bits values of K (klo_bits =
// 31 or Klo >= K: [np][H][rows][K]); a 5D map over (Klo, rows, K / Klo, H,
// np) whose box = cb bytes of K x box_rows x 1 x 1 x np planes lands in
// shared memory as [plane][row][cb bytes], cb-byte swizzled
bool encode_planes(CUtensorMap *map, void *planes, int64_t H, int64_t rows, int64_t K, int es, int box_rows,
                   int cb, int np, CUtensorMapDataType dtype, int klo_bits) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const int64_t klo = (klo_bits < 31 && ((int64_t)1 << klo_bits) < K) ? ((int64_t)1 << klo_bits) : K;
    const int64_t khi = K / klo;
    cuuint64_t dims[5] = {(cuuint64_t)klo, (cuuint64_t)rows, (cuuint64_t)khi, (cuuint64_t)H, (cuuint64_t)np};
    cuuint64_t strides[4] = {(cuuint64_t)(klo * es), (cuuint64_t)(rows * klo * es), (cuuint64_t)(rows * K * es),
                             (cuuint64_t)(H * rows * K * es)};
    cuuint32_t box[5] = {(cuuint32_t)(cb / es), (cuuint32_t)box_rows, 1, 1, (cuuint32_t)np};
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r = fn(map, dtype, 5, planes, dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    cb == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                             : (cb == 32 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_128B),
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// The box view of a planar output for TMA stores (TcTmaOut), or false when
// the layout does not fit one: 16-bit planes of a 4-product form (hi/lo or
// one scaled piece), full tiles, the half tile's columns c0..c2 at
// destination bits 0..2 (a lane's eight columns are 16 consecutive bytes)
// and bits 0..5 all tile bits (128-byte box rows), at most five dimensions.
bool plan_tma_out(const TcPlanarOut &o, TcTmaOut &t) {
    std::memset(&t, 0, sizeof t);
    if (o.mode != 1 && o.mode != 3 && o.mode != 4) return false;
    if (o.nN < 6 || o.nM < 7 || o.ntb != 12) return false;
    if (o.plane_stride <= 0 || (o.plane_stride & (o.plane_stride - 1)) != 0) return false;
    const int r = __builtin_ctzll((uint64_t)o.plane_stride);
    for (int k = 0; k < 6; k++)
        if (o.tpos[k] != k) return false;
    for (int k = 0; k < 3; k++)
        if (o.tb[k] != k) return false;
    t.np = o.mode == 3 ? 2 : 4;
    t.start[0] = 0;
    t.bits[0] = 6;
    t.box[0] = 6;
    for (int k = 0; k < 6; k++) t.boxbit[o.tb[k]] = (int8_t)k;
    int nd = 1, bb = 6, pos = 6;
    for (int k = 6; k < 12;) {
        const int p0 = o.tpos[k];
        int len = 1;
        while (k + len < 12 && o.tpos[k + len] == p0 + len) len++;
        if (p0 > pos) {  // a gap of non-tile bits: box 1
            if (nd == 5) return false;
            t.start[nd] = (int8_t)pos;
            t.bits[nd] = (int8_t)(p0 - pos);
            t.box[nd] = 0;
            nd++;
        }
        if (nd == 5) return false;
        t.start[nd] = (int8_t)p0;
        t.bits[nd] = (int8_t)len;
        t.box[nd] = (int8_t)len;
        for (int j = 0; j < len; j++) t.boxbit[o.tb[k + j]] = (int8_t)(bb + j);
        bb += len;
        nd++;
        pos = p0 + len;
        k += len;
    }
    if (pos > r) return false;
    // the last dimension runs to the top of a plane; the planes follow it
    t.bits[nd - 1] = (int8_t)(r - t.start[nd - 1]);
    t.plane_step = (int64_t)1 << t.bits[nd - 1];
    t.nd = nd;
    t.on = 1;
    return true;
}

bool encode_tma_out(CUtensorMap *map, const TcPlanarOut &o, const TcTmaOut &t) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[5], strides[4];
    cuuint32_t box[5], estr[5] = {1, 1, 1, 1, 1};
    const int r = __builtin_ctzll((uint64_t)o.plane_stride);
    for (int i = 0; i < 5; i++) {
        if (i < t.nd) {
            dims[i] = (cuuint64_t)1 << t.bits[i];
            if (i == t.nd - 1) dims[i] *= (cuuint64_t)t.np;
            box[i] = 1u << t.box[i];
        } else {
            dims[i] = 1;  // unused dimensions: extent 1 past the planes
            box[i] = 1;
        }
        // byte strides (dimension 0 is contiguous)
        if (i > 0) strides[i - 1] = i < t.nd ? ((cuuint64_t)2 << t.start[i]) : ((cuuint64_t)t.np * 2 << r);
    }
    CUresult res = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 5, o.planes, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return res == CUDA_SUCCESS;
}

}  // namespace

bool tc_planar_tma_fits(const TcPlanarOut &o, TcTmaOut *out) {
    TcTmaOut t;
    const bool fits = tc_planar_direct_run(o) == 0 && plan_tma_out(o, t);
    if (out) *out = t;
    return fits;
}

int tc_planar_direct_run(const TcPlanarOut &o) {
    // Full 128 x 64 tiles whose destination starts with 16 bytes of one row
    // (the tile's column bits c0 .. c(J-1) at positions 0 .. J-1: 8 elements
    // of a 16-bit plane, 4 of a 32-bit one) followed by the row bit r0 at
    // position J: the lanes (rows) of a warp then store 16 bytes each, two
    // neighbouring lanes one whole 32-byte sector, from registers.  Other
    // layouts go through the shared-memory staging (whole 512-byte rows).
    if (o.mode == 0 || o.nN < 6 || o.nM < 7) return 0;
    const int J = mode_word(o.mode) ? 2 : 3;
    if (o.ntb <= J) return 0;
    for (int k = 0; k < J; k++)
        if (o.tb[k] != k || o.tpos[k] != k) return 0;
    return (o.tb[J] == 6 && o.tpos[J] == J) ? J : 0;
}

bool tc_form_available(tn_form form) {
    return (form == TN_BF16X3 || form == TN_TF32X3 || form == TN_FP16S || form == TN_FP16X3) && encode_fn() != nullptr;
}

int tc_plane_bytes(tn_form form) { return form == TN_TF32X3 ? 4 : 2; }

int tc_default_flush_bytes(tn_form form) { return default_flush_bytes(form); }

int tc_plane_count(tn_form form, int products) {
    return form == TN_FP16S ? 2 : (products == 3 ? 6 : 4);
}

bool tc_form_has_3m(tn_form form) { return form == TN_BF16X3 || form == TN_TF32X3 || form == TN_FP16X3; }

bool tc_gemm_suitable(const GemmArgs &a) {
    // narrow N and short K are zero-filled by TMA to the tile (the MMAs on
    // the padding are wasted but the step stays on the tensor cores); a plane
    // row must hold a multiple of 16 bytes (K >= 8 elements)
    return a.M >= 64 && a.N >= 8 && a.K >= 8 && a.H <= 65535 && a.M < (1ll << 31) && a.N < (1ll << 31) &&
           a.K < (1ll << 31);
}

int tc_choose_ksplit(const GemmArgs &a, tn_form form) {
    // the persistent kernel runs one CTA per SM over tiles x K parts; a grid
    // with fewer tiles than SMs splits K so that the work units fill whole
    // waves of the 152 SMs (the makespan is ceil(units / 152) units), with at
    // least 4 K chunks of 64 bytes per part and at most 4 waves of units
    constexpr int64_t kSms = 152;
    const int64_t tiles = ((a.M + TM - 1) / TM) * ((a.N + TN - 1) / TN) * a.H;
    if (tiles >= kSms) return 1;
    const int64_t chunks = (a.K * tc_plane_bytes(form) + 63) / 64;
    int64_t best = 1;
    double best_eff = 0.0;
    for (int64_t s = 1; s <= 64 && tiles * s <= 4 * kSms && chunks / s >= 4; s++) {
        const int64_t units = tiles * s;
        const double eff = (double)units / (double)(((units + kSms - 1) / kSms) * kSms);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = s;
        }
    }
    return (int)best;
}

bool tc_prepare(TcGemm &g) {
    const int es = tc_plane_bytes(g.form);
    if (g.products == 0) g.products = 4;
    if (g.products != 4 && (g.products != 3 || !tc_form_has_3m(g.form))) return false;
    if (g.products == 3) {
        // six planes per operand: 32-byte K chunks (one MMA K step, 32-byte
        // swizzle) keep five ring stages in shared memory; 64-byte chunks on
        // request (two stages)
        g.chunk_bytes = (g.chunk_bytes == 64 && g.a.K * es >= 64) ? 64 : 32;
        if (g.flush_bytes < g.chunk_bytes || g.flush_bytes % g.chunk_bytes) g.flush_bytes = default_flush_bytes(g.form);
    } else {
        if (g.chunk_bytes != 64 && g.chunk_bytes != 128) g.chunk_bytes = kDefaultChunkBytes;
        if (g.flush_bytes < g.chunk_bytes)
            g.flush_bytes = default_flush_bytes(g.form) < g.chunk_bytes ? g.chunk_bytes : default_flush_bytes(g.form);
        if (g.a.K * es < g.chunk_bytes) g.chunk_bytes = 64;
    }
    const int cb = g.chunk_bytes, np = tc_plane_count(g.form, g.products);
    const CUtensorMapDataType dt = g.form == TN_TF32X3 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : g.form == TN_BF16X3 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                         : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    // a chunked layout holds whole runs of 2^k_low_bits K values of 128
    // bytes; a TMA chunk (64 or 128 bytes) stays inside one run
    if (g.k_low_bits > 0 && (((int64_t)es << g.k_low_bits) != 128 || (g.a.K & ((1ll << g.k_low_bits) - 1)) != 0))
        return false;
    const int klo = g.k_low_bits > 0 ? g.k_low_bits : 31;
    if (!encode_planes(reinterpret_cast<CUtensorMap *>(g.mapA), g.planesA, g.a.H, g.a.M, g.a.K, es, TM, cb, np, dt,
                       klo))
        return false;
    if (!encode_planes(reinterpret_cast<CUtensorMap *>(g.mapB), g.planesB, g.a.H, g.a.N, g.a.K, es, TN, cb, np, dt,
                       klo))
        return false;
    // planar output stored by TMA where the layout fits a box view and the
    // epilogue would otherwise stage it (the direct register stores stay)
    std::memset(g.mapC, 0, sizeof g.mapC);
    TcTmaOut t;
    if (g.tma_out_ok && g.products == 4 && g.ksplit <= 1 && g.out.planes && tc_planar_direct_run(g.out) == 0 &&
        plan_tma_out(g.out, t)) {
        if (!encode_tma_out(reinterpret_cast<CUtensorMap *>(g.mapC), g.out, t)) return false;
        g.out_tma = t;
    } else {
        std::memset(&g.out_tma, 0, sizeof g.out_tma);
    }
    return true;
}

template <int KIND, int CB, bool M3, int EW>
cudaError_t launch_ew(const TcGemm &g, const GemmTcParams &p, dim3 grid, cudaStream_t s) {
    constexpr int NP = M3 ? 6 : (kind_split(KIND) ? 4 : 2);
    cudaError_t e = set_max_dynamic_smem((const void *)tc_gemm_kernel<KIND, CB, M3, EW>, Ring<CB, NP>::kSmem);
    if (e != cudaSuccess) return e;
    const CUtensorMap &mA = *reinterpret_cast<const CUtensorMap *>(g.mapA);
    const CUtensorMap &mB = *reinterpret_cast<const CUtensorMap *>(g.mapB);
    const CUtensorMap &mC = *reinterpret_cast<const CUtensorMap *>(g.mapC);
    tc_gemm_kernel<KIND, CB, M3, EW><<<grid, ep_threads(EW), Ring<CB, NP>::kSmem, s>>>(mA, mB, mC, p);
    return cudaGetLastError();
}

// sixteen epilogue warps when a tile has one accumulator read-out (short K:
// the epilogue sets the GEMM's time), else eight
template <int KIND, int CB, bool M3 = false>
cudaError_t launch_variant(const TcGemm &g, GemmTcParams p, dim3 grid, cudaStream_t s) {
    const bool one_readout = p.part_len <= p.flush_chunks;
    // the TMA-stored planar output is compiled into the eight-warp kernel
    // only (the sixteen-warp one has 96 registers a thread): staged there
    if (one_readout) p.tma.on = 0;
    return one_readout ? launch_ew<KIND, CB, M3, 16>(g, p, grid, s) : launch_ew<KIND, CB, M3, 8>(g, p, grid, s);
}

cudaError_t launch_gemm_tc(const TcGemm &g, cudaStream_t s) {
    GemmTcParams p;
    p.C = g.a.C;
    p.H = g.a.H;
    p.M = g.a.M;
    p.N = g.a.N;
    p.K = g.a.K;
    p.sCh = g.a.sCh;
    p.sCm = g.a.sCm;
    p.sCn = g.a.sCn;
    p.k_chunk = g.chunk_bytes / tc_plane_bytes(g.form);
    p.klo_bits = g.k_low_bits > 0 ? g.k_low_bits : 31;
    p.ksplit = g.ksplit > 0 ? g.ksplit : 1;
    p.flush_chunks = g.flush_bytes / g.chunk_bytes;
    if (p.flush_chunks < 1) p.flush_chunks = 1;
    p.scales = g.scales;
    p.max_slot = g.max_slot;
    p.out = g.out;
    // planar output: bf16 / tf32 hi/lo (modes 1, 2) or scaled fp16 (3, 4)
    // with the bound-derived exponent.  Plane offsets are 64-bit (a tile's
    // own offsets 32-bit, checked when the plan builds the tables)
    const bool m3 = g.products == 3;
    if (g.products != 0 && g.products != 4 && !(m3 && tc_form_has_3m(g.form))) return cudaErrorInvalidValue;
    if (m3 && g.chunk_bytes != 32 && g.chunk_bytes != 64) return cudaErrorInvalidValue;  // tc_prepare sets it
    // a GEMM writes the planes of its own form's split (4M or 3M); the
    // kernel's planar epilogue is compiled for that mode only
    const int own_mode = planar_mode_of(g.form == TN_TF32X3   ? kTF32
                                        : g.form == TN_BF16X3 ? kBF16
                                        : g.form == TN_FP16S  ? kFP16
                                                              : kFP16X3,
                                        m3);
    if (p.out.mode != 0 && (p.ksplit > 1 || !p.out.planes || p.out.mode != own_mode ||
                            mode_3m(p.out.mode) != m3 || p.out.plane_stride > (int64_t(1) << 44) ||
                            p.out.ntb > 12))
        return cudaErrorInvalidValue;
    // a scaled planar output needs a scaled form (its operands' exponents)
    // and the slot through which the next step reads the planes' exponent
    if (mode_scaled(p.out.mode) &&
        (!((g.form == TN_FP16S && p.out.mode == 3) || (g.form == TN_FP16X3 && mode_base(p.out.mode) == 4)) ||
         !g.max_slot))
        return cudaErrorInvalidValue;
    if (g.max_slot) {
        if (p.ksplit > 1) return cudaErrorInvalidValue;  // partial tiles: their max is not C's
        // the slot and its companion two places on (the true max, written
        // only by a scaled planar output; 0 tells the consumer to use the slot)
        cudaError_t e = cudaMemsetAsync(g.max_slot, 0, sizeof(unsigned), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(g.max_slot + 2, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
    }
    if ((g.form == TN_FP16S || g.form == TN_FP16X3) && !g.scales) return cudaErrorInvalidValue;
    p.direct_run = tc_planar_direct_run(p.out);
    p.tma = g.out_tma;
    if (p.tma.on && (p.out.mode == 0 || p.ksplit > 1 || g.out.planes == nullptr)) return cudaErrorInvalidValue;
    const int64_t gm = (g.a.M + TM - 1) / TM, gn = (g.a.N + TN - 1) / TN;
    if (gm > INT32_MAX || gn > INT32_MAX) return cudaErrorInvalidConfiguration;
    p.gm = (int)gm;
    p.gn = (int)gn;
    p.tiles = gm * gn * g.a.H * p.ksplit;
    if (p.tiles >= (int64_t(1) << 32)) return cudaErrorInvalidConfiguration;  // 32-bit tile decode
    {
        const int64_t all = (p.K + p.k_chunk - 1) / p.k_chunk;
        if (all > INT32_MAX) return cudaErrorInvalidConfiguration;
        p.all_chunks = (int)all;
        p.part_len = (int)((all + p.ksplit - 1) / p.ksplit);
    }
    if (p.ksplit > 1) {
        // C = [H][M][N] contiguous (the plan's GEMM output layout)
        cudaError_t e = cudaMemsetAsync(g.a.C, 0, (size_t)(g.a.H * g.a.M * g.a.N) * sizeof(float2), s);
        if (e != cudaSuccess) return e;
    }
    // persistent: one CTA per SM (the ring and staging fill the SM's shared
    // memory), at most one per tile
    static std::atomic<int> sm_count[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    int sms = sm_count[dev].load(std::memory_order_relaxed);
    if (sms == 0) {
        cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        sm_count[dev].store(sms, std::memory_order_relaxed);
    }
    dim3 grid((unsigned)(p.tiles < sms ? p.tiles : sms));
    if (m3) {
        const bool c64 = g.chunk_bytes == 64;
        if (g.form == TN_TF32X3)
            return c64 ? launch_variant<kTF32, 64, true>(g, p, grid, s) : launch_variant<kTF32, 32, true>(g, p, grid, s);
        if (g.form == TN_BF16X3)
            return c64 ? launch_variant<kBF16, 64, true>(g, p, grid, s) : launch_variant<kBF16, 32, true>(g, p, grid, s);
        return c64 ? launch_variant<kFP16X3, 64, true>(g, p, grid, s)
                   : launch_variant<kFP16X3, 32, true>(g, p, grid, s);
    }
    if (g.form == TN_TF32X3)
        return g.chunk_bytes == 64 ? launch_variant<kTF32, 64>(g, p, grid, s) : launch_variant<kTF32, 128>(g, p, grid, s);
    if (g.form == TN_BF16X3)
        return g.chunk_bytes == 64 ? launch_variant<kBF16, 64>(g, p, grid, s) : launch_variant<kBF16, 128>(g, p, grid, s);
    if (g.form == TN_FP16X3)
        return g.chunk_bytes == 64 ? launch_variant<kFP16X3, 64>(g, p, grid, s)
                                   : launch_variant<kFP16X3, 128>(g, p, grid, s);
    return g.chunk_bytes == 64 ? launch_variant<kFP16, 64>(g, p, grid, s) : launch_variant<kFP16, 128>(g, p, grid, s);
}

bool small_tc_suitable(const SmallArgs &a, tn_form form) {
    // split forms with 22+ significant bits and bf16x3; K of 16 or 32, N of
    // 8, 16 or 32; no batch bits; whole 128-row tiles whose T and C runs are
    // 128 rows
    if (form != TN_FP16X3 && form != TN_TF32X3 && form != TN_BF16X3) return false;
    if (a.nH != 0 || a.nK < 4 || a.nK > 5 || a.nN < 3 || a.nN > 5 || a.tiled == 3) return false;
    if (a.rows < (1 << 16) || (a.rows & (a.rows - 1)) != 0) return false;
    for (int j = 0; j < a.nK; j++)
        if (a.kposT[j] < 7) return false;
    for (int j = 0; j < a.nN; j++)
        if (a.nposC[j] < 7) return false;
    return true;
}

template <int KIND, int CB>
cudaError_t launch_small_tc_t(const SmallTcParams &p, cudaStream_t s) {
    constexpr int ES = KIND == kTF32 ? 4 : 2;
    using L = SmallTcSmem<CB, CB / ES>;
    static_assert(L::kBytes <= 232448, "shared memory per CTA");
    cudaError_t e = set_max_dynamic_smem((const void *)small_tc_kernel<KIND, CB>, L::kBytes);
    if (e != cudaSuccess) return e;
    static std::atomic<int> sm_count[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    int sms = sm_count[dev].load(std::memory_order_relaxed);
    if (sms == 0) {
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        sm_count[dev].store(sms, std::memory_order_relaxed);
    }
    // two CTAs per SM where shared memory allows (one tile's split and
    // products overlap the other's loads and stores): 228 KB per SM, 1 KB
    // of it reserved per CTA
    e = cudaFuncSetAttribute((const void *)small_tc_kernel<KIND, CB>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    const int per_sm = (2 * (L::kBytes + 1024) <= 228 * 1024) ? 2 : 1;
    const int grid = (int)std::min<int64_t>(p.tiles, (int64_t)sms * per_sm);
    small_tc_kernel<KIND, CB><<<grid, kSmallTcThreads, L::kBytes, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_small_tc(const SmallArgs &a, tn_form form, cudaStream_t s) {
    if (!small_tc_suitable(a, form)) return cudaErrorInvalidValue;
    // 16-byte copies of T rows need a 16-byte aligned T
    if ((reinterpret_cast<uintptr_t>(a.T) & 15) != 0) return cudaErrorMisalignedAddress;
    SmallTcParams p;
    std::memset(&p, 0, sizeof p);
    p.T = a.T;
    p.S = a.S;
    p.C = a.C;
    p.tiles = a.rows >> 7;
    p.nK = a.nK;
    p.nN = a.nN;
    p.n_tins = a.n_tins;
    p.n_cins = a.n_cins;
    for (int j = 0; j < kSmallMaxBits; j++) {
        p.tins[j] = a.tins[j];
        p.cins[j] = a.cins[j];
    }
    const int KS = 1 << a.nK, NS = 1 << a.nN;
    for (int k = 0; k < KS; k++) {
        uint64_t o = 0, os = 0;
        for (int j = 0; j < a.nK; j++)
            if ((k >> j) & 1) {
                o |= 1ull << a.kposT[j];
                os |= 1ull << a.kposS[j];
            }
        p.offT[k] = o;
        for (int n = 0; n < NS; n++) {
            uint64_t on = os;
            for (int j = 0; j < a.nN; j++)
                if ((n >> j) & 1) on |= 1ull << a.nposS[j];
            p.offS[k * NS + n] = (uint32_t)on;
        }
    }
    for (int n = 0; n < NS; n++) {
        uint64_t o = 0;
        for (int j = 0; j < a.nN; j++)
            if ((n >> j) & 1) o |= 1ull << a.nposC[j];
        p.offC[n] = o;
    }
    p.max_slot = a.max_slot;
    if (a.max_slot) {
        cudaError_t e = cudaMemsetAsync(a.max_slot, 0, sizeof(unsigned), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(a.max_slot + 2, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
    }
    if (form == TN_TF32X3) return a.nK == 4 ? launch_small_tc_t<kTF32, 64>(p, s) : launch_small_tc_t<kTF32, 128>(p, s);
    if (form == TN_BF16X3) return a.nK == 4 ? launch_small_tc_t<kBF16, 32>(p, s) : launch_small_tc_t<kBF16, 64>(p, s);
    return a.nK == 4 ? launch_small_tc_t<kFP16X3, 32>(p, s) : launch_small_tc_t<kFP16X3, 64>(p, s);
}

int tc_read_error(cudaStream_t s) {
    int v = 0, zero = 0;
    cudaMemcpyFromSymbolAsync(&v, tc_error, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
    cudaMemcpyToSymbolAsync(tc_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
    return v;
}

}  // namespace tn
