// Kernel argument blocks shared by the host plan compiler and the CUDA
// kernels.  Plain structs passed by value as kernel parameters.
#pragma once
#include <cmath>
#include <cstdint>

#include <cuda_runtime.h>
#ifdef __CUDACC__
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#endif

namespace tn {

constexpr int kMaxRank = 48;     // largest tensor rank a kernel handles
constexpr int kSmallMaxBits = 12;  // small operand: H + K + N bits <= this
constexpr int kMaxHBits = 12;

// One pairwise step where one operand S is small (<= 2^12 values, staged in
// shared memory) and the other, T, is read once: for every index r over T's
// non-K bits,  C[cpos(r) | offC[n]] = sum_k T[tpos(r) | offT[k]] * S[h(r), k, n].
// C's layout is T's with the K labels replaced by the N labels.
struct SmallArgs {
    const float2 *T;
    const float2 *S;
    float2 *C;
    int64_t rows;        // 2^(rank T - nK)
    int row_bits;        // log2 rows (set by the launcher)
    int nK, nN, nH;
    int n_tins;          // K positions of T, ascending (zero insertion turns r into T's base)
    int n_cins;          // N positions of C, ascending
    int tins[kSmallMaxBits];
    int cins[kSmallMaxBits];
    int kposT[kSmallMaxBits];  // position in T of bit j of k
    int nposC[kSmallMaxBits];  // position in C of bit j of n
    int hbitR[kMaxHBits];      // bit of r holding bit j of h
    int hposS[kMaxHBits], kposS[kSmallMaxBits], nposS[kSmallMaxBits];  // positions in S
    int s_rank;
    // Tiled form (filled by prepare_small_tiled; tiled == 0 selects the
    // one-thread-per-row kernel).  A tile is 2^tb consecutive rows r; its T
    // elements are 2^(tb + nK) values made of n_runT contiguous runs of 2^lt
    // elements (T offset tbase(r0) + runOffT[u] + e), staged in shared memory
    // at [k][row] (row stride 2^tb + 1) at runDstT[u] + dstLoT[e & 63] +
    // dstHiT[e >> 6]; the C tile likewise (two-level run tables), read back
    // from [n][row].
    int tiled;
    int tb;              // log2 rows per tile
    int rpt, npt;        // rows and outputs per thread
    int lt, lc;          // contiguous run bits of the T and C tiles
    int n_runT, n_runC;  // runs per tile
    uint64_t runOffT[32];
    uint32_t runDstT[32], dstLoT[64], dstHiT[64];
    // C runs u (up to 4096): offset runOffCLo[u & 63] + runOffCHi[u >> 6],
    // shared-memory index runSrcCLo[u & 63] + runSrcCHi[u >> 6]
    uint64_t runOffCLo[64], runOffCHi[64];
    uint32_t runSrcCLo[64], runSrcCHi[64], srcLoC[64], srcHiC[64];
    // planar store (tiled == 3): instead of complex64 C, the tile writes the
    // next tensor-core step's hi/lo planes (planar_mode 1 bf16, 2 tf32) at C
    // (the planes' base), plane q at offset q * plane_stride; the C tables
    // above then describe runs in the destination layout, and row bit i of r
    // (i >= tb) lands at destination position drow[i]
    int planar_mode;
    int64_t plane_stride;
    int8_t drow[kMaxRank];
    // optional (complex64 C only): receives max |re|, |im| of C (float bits,
    // atomic max; the launcher zeroes it and the slot two places on, which a
    // consumer reads as "no separate true max"), so that the scaled split of
    // C needs no max-abs pass of its own
    unsigned *max_slot;
    // tensor-core form (tn_form of a split form) when the step runs on the
    // tensor cores with T split in shared memory (launch_small_tc); 0: CUDA
    // cores
    int tc_form;
};

// Decide whether a small step takes the tiled kernel and fill its tables
// (host; plan compile time).  Needs rows set and the bit maps complete.
void prepare_small_tiled(SmallArgs &a);

// Make a tiled small step write split planes (mode 1 bf16, 2 tf32; planes of
// plane_stride elements) in a destination layout given by cdest[q], the
// destination position of C position q.  Returns 0 on success; otherwise a
// unchanged and a reason: 1 not tiled, 2 tile does not fit the rows or the
// batch bits, 3 T tables, 4 destination runs shorter than 32 elements or
// more than 32 runs per tile (*run_bits = the run length's bits), 5 shared
// memory.
int prepare_small_planar(SmallArgs &a, const int *cdest, int mode, int64_t plane_stride, int *run_bits);

// Bit permutation through a shared-memory tile, optionally fused with the
// hi/lo split of split-precision GEMM operands.
//   out index d (r bits) <- in[sum_p bit_p(d) << src_pos[p]]
// mode 0: complex64 out[d];
// mode 1/2: four planes (re_hi, im_hi, re_lo, im_lo) of bf16 (1) or tf32 held
//           in 32 bits (2) at d + q * plane_stride, q = 0..3;
// mode 3:   two fp16 planes (re, im) of x * 2^-e, e = ilogb(max|x|) - 13 from
//           the max-abs slot `scale` (a float stored as its bits), so the
//           largest scaled value lies in [2^13, 2^14);
// mode 4:   four fp16 planes (re_hi, im_hi, re_lo, im_lo) of the same scaled
//           value: hi = fp16(x 2^-e), lo = fp16(x 2^-e - hi);
// modes 5, 6, 7: modes 1, 2 and 4 for the 3M complex product: a third value
//           s = re + im (rounded to FP32; after the scale for mode 7) is split
//           like re and im, six planes (re_hi, im_hi, s_hi, re_lo, im_lo, s_lo).
// The tile holds the bits at the source's and the destination's lowest
// positions, so reads and writes are both coalesced.
constexpr int kTileMaxBits = 10;
struct BitPermArgs {
    const float2 *in;
    void *out;
    int rank;
    int mode;
    int64_t plane_stride;
    int n_tile;                      // tile bits
    int tile_dst[kTileMaxBits];      // dest positions of tile bits, ascending (write order)
    int rd_w[kTileMaxBits];          // read order bit j -> index into tile_dst
    int rd_src[kTileMaxBits];        // read order bit j -> source position (ascending)
    int n_rest;                      // remaining bits (grid-strided)
    int rest_dst[kMaxRank];
    int rest_src[kMaxRank];
    const unsigned *scale;           // modes 3, 4: max-abs slot of the operand
    int pair_rd, pair_wr;            // set by the launcher: two neighbouring elements per access
};

// max over |re|, |im| of n complex values into *slot (float bits; the
// launcher zeroes the slot first)
struct MaxAbsArgs {
    const float2 *in;
    int64_t n;
    unsigned *slot;
    unsigned *companion;  // optional: zeroed with the slot (a consumer's true-max slot)
};

// power-of-two exponent e of the FP16S scale for a max-abs value: the largest
// scaled magnitude max * 2^-e lies in [2^13, 2^14)
__host__ __device__ inline int fp16s_exponent(float maxabs) {
    if (!(maxabs > 0.f)) return 0;
    int ex;
    frexpf(maxabs, &ex);  // maxabs in [2^(ex-1), 2^ex)
    return ex - 14;
}

// Split-mode properties (modes of BitPermArgs, TcPlanarOut and SmallArgs)
__host__ __device__ constexpr bool mode_3m(int m) { return m >= 5 && m <= 7; }
// the 4M mode with the same pieces: 5 -> 1, 6 -> 2, 7 -> 4
__host__ __device__ constexpr int mode_base(int m) { return m == 5 ? 1 : m == 6 ? 2 : m == 7 ? 4 : m; }
// pieces held in 32 bits (tf32) rather than 16
__host__ __device__ constexpr bool mode_word(int m) { return mode_base(m) == 2; }
// values scaled by 2^-e before the split (fp16 forms)
__host__ __device__ constexpr bool mode_scaled(int m) { return mode_base(m) == 3 || mode_base(m) == 4; }
// planes written by a split mode
__host__ __device__ constexpr int mode_planes(int m) { return m == 3 ? 2 : (mode_3m(m) ? 6 : 4); }
// the 3M mode with the same pieces (1 -> 5, 2 -> 6, 4 -> 7; others unchanged)
__host__ __device__ constexpr int mode_to_3m(int m) { return m == 1 ? 5 : m == 2 ? 6 : m == 4 ? 7 : m; }

#ifdef __CUDACC__
// round to nearest (ties away) on tf32's 10-bit mantissa, in a 32-bit container
__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// x 2^-e as ldexpf(x, -e) gives it: a multiplication by the power of two
// when 2^-e is a normal float (both round the same), else two such
// multiplications (the same while the intermediate stays normal; e stays in
// [-126, 126] for tensors whose largest value lies between 2^-112 and 2^140)
__device__ __forceinline__ float scale_pow2(float x, int e) {
    const int e1 = (e >= -126 && e <= 126) ? e : e / 2;
    const int e2 = e - e1;
    const float y = x * __int_as_float((127 - e1) << 23);
    return e2 ? y * __int_as_float((127 - e2) << 23) : y;
}

// The pieces of one complex value for the split modes of BitPermArgs
// (1 bf16 hi/lo, 2 tf32 hi/lo, 3 scaled fp16, 4 scaled fp16 hi/lo), plane
// order (re_hi, im_hi, re_lo, im_lo); 16-bit pieces in the low half.
struct Pieces {
    uint32_t q[4];
};
// ... and of the 3M modes 5, 6, 7: (re_hi, im_hi, s_hi, re_lo, im_lo, s_lo)
struct Pieces6 {
    uint32_t q[6];
};

// hi and lo pieces of one (already scaled) real value, for mode_base b
__device__ __forceinline__ void split_real(int b, float x, uint32_t &hi, uint32_t &lo) {
    if (b == 1) {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        hi = __bfloat16_as_ushort(h);
        lo = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
    } else if (b == 2) {
        hi = tf32_rna(x);
        lo = tf32_rna(x - __uint_as_float(hi));
    } else {
        const __half h = __float2half_rn(x);
        hi = __half_as_ushort(h);
        lo = __half_as_ushort(__float2half_rn(x - __half2float(h)));
    }
}

__device__ __forceinline__ Pieces6 split_value_3m(int mode, float2 v, int e) {
    Pieces6 r;
    const int b = mode_base(mode);
    const float xr = b == 4 ? scale_pow2(v.x, e) : v.x, xi = b == 4 ? scale_pow2(v.y, e) : v.y;
    split_real(b, xr, r.q[0], r.q[3]);
    split_real(b, xi, r.q[1], r.q[4]);
    split_real(b, xr + xi, r.q[2], r.q[5]);
    return r;
}

// The re and im pieces are converted as pairs (one packed conversion for two
// values, round to nearest each, as the scalar conversions would).
__device__ __forceinline__ Pieces split_value(int mode, float2 v, int e) {
    Pieces r;
    if (mode == 1) {
        const __nv_bfloat162 h = __float22bfloat162_rn(v);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __float22bfloat162_rn(make_float2(v.x - hf.x, v.y - hf.y));
        r.q[0] = __bfloat16_as_ushort(h.x);
        r.q[1] = __bfloat16_as_ushort(h.y);
        r.q[2] = __bfloat16_as_ushort(l.x);
        r.q[3] = __bfloat16_as_ushort(l.y);
    } else if (mode == 2) {
        const uint32_t rh = tf32_rna(v.x), ih = tf32_rna(v.y);
        r.q[0] = rh;
        r.q[1] = ih;
        r.q[2] = tf32_rna(v.x - __uint_as_float(rh));
        r.q[3] = tf32_rna(v.y - __uint_as_float(ih));
    } else {  // 3, 4: scaled by 2^-e (exact), then one fp16 piece or hi/lo
        const float2 x = make_float2(scale_pow2(v.x, e), scale_pow2(v.y, e));
        const __half2 h = __float22half2_rn(x);
        const float2 hf = __half22float2(h);
        const __half2 l = __float22half2_rn(make_float2(x.x - hf.x, x.y - hf.y));
        r.q[0] = __half_as_ushort(h.x);
        r.q[1] = __half_as_ushort(h.y);
        r.q[2] = __half_as_ushort(l.x);
        r.q[3] = __half_as_ushort(l.y);
    }
    return r;
}

#endif

// Strided batched complex GEMM, all strides in complex elements:
// C[h sCh + m sCm + n sCn] = sum_k A[h sAh + m sAm + k sAk] B[h sBh + k sBk + n sBn]
struct GemmArgs {
    const float2 *A;
    const float2 *B;
    float2 *C;
    int64_t H, M, N, K;
    int64_t sAh, sAm, sAk, sBh, sBk, sBn, sCh, sCm, sCn;
};

// Slice extraction of leaves holding fixed sliced labels: for each entry,
// dst[j] = src[insert_zeros(j, fpos) | sum_f bit(slice_base, sbit[f]) << fpos[f]].
struct ExtractEntry {
    const float2 *src;
    float2 *dst;
    int n_out;
    int nf;
    int fpos_sorted[kMaxRank];
    int fpos[kMaxRank];
    int sbit[kMaxRank];
};

// Cross-slice FP64 sum: amp[o] += sum_{b in [b_lo, b_hi)} R[pos(o, b)].
struct AccumArgs {
    const float2 *R;
    double2 *amp;
    int n_open, n_batch;
    int opos[kMaxRank];  // position in R of bit j of o (j = 0 is the LSB of o)
    int bpos[kMaxRank];  // position in R of bit j of b
    int64_t b_lo, b_hi;
};

// One small step run as a task of the persistent task launch
// (launch_small_tasks): the one-thread-per-item form of SmallArgs (item =
// row r and a chunk of nc outputs), its items cut into units of at most
// kTaskUnitItems, and the tasks of the same launch whose outputs it reads.
// Bit positions fit int8_t (tensor ranks stay below 64).
constexpr int kTaskUnitItems = 1024;  // 4 items per thread of a 256-thread block
constexpr int kTaskMaxK = 7;          // tasks loop over at most 2^7 K values per item
struct SmallTask {
    const float2 *T;
    const float2 *S;
    float2 *C;
    int64_t rows;  // a power of two
    int row_bits, nK, nN, nH;
    int nc;        // outputs per item: 8, 16 or 32
    int n_tins, n_cins;
    int first_unit, n_units;
    int n_deps;
    int dep[2];    // producing tasks of this launch (indices below this task's)
    int8_t tins[kSmallMaxBits], cins[kSmallMaxBits], kposT[kSmallMaxBits], nposC[kSmallMaxBits];
    int8_t hbitR[kMaxHBits], hposS[kMaxHBits], kposS[kSmallMaxBits], nposS[kSmallMaxBits];
};

// launchers (kernels.cu); return cudaSuccess or the launch error
// Raise a kernel's dynamic shared-memory limit to `bytes` on the current
// device.  The attribute belongs to the device, so it is set once per
// (kernel, device) pair; thread-safe.
cudaError_t set_max_dynamic_smem(const void *kernel, int bytes);

cudaError_t launch_small(const SmallArgs &a, cudaStream_t s);
// Many small steps in one persistent launch.  d_tasks[0 .. n_tasks) in
// dependency order; d_unit_task[u] = the task of unit u (units of a task are
// consecutive, tasks in order); d_ctr holds n_tasks + 1 ints that this call
// zeroes first (a unit counter, then the finished units of each task).
cudaError_t launch_small_tasks(const SmallTask *d_tasks, const int *d_unit_task, int total_units, int *d_ctr,
                               int n_tasks, cudaStream_t s);
// SmallTask of a one-thread-per-row small step (host; a's bit maps complete,
// rows set; nK <= kTaskMaxK); pointers are copied as they are
SmallTask make_small_task(const SmallArgs &a);
// reads and clears the task launches' error word (a dependency wait that
// gave up); synchronises the stream
int small_task_read_error(cudaStream_t s);
cudaError_t launch_bitperm(const BitPermArgs &a, cudaStream_t s);
cudaError_t launch_maxabs(const MaxAbsArgs &a, cudaStream_t s);
cudaError_t launch_gemm_f32(const GemmArgs &a, cudaStream_t s);
cudaError_t launch_extract(const ExtractEntry *d_entries, int n_entries, int max_out, uint64_t slice_base,
                           cudaStream_t s);
cudaError_t launch_accum(const AccumArgs &a, cudaStream_t s);
// d_out3: {sum p, 2^scale_exp * sum p - 1, max p}
cudaError_t launch_prob_xeb(const double2 *amp, int64_t n, double *prob, double *d_out3, int scale_exp,
                            cudaStream_t s);
cudaError_t launch_zero_f64(double *p, int64_t n, cudaStream_t s);
// dst[i] = complex64(src[i]) (round to nearest)
cudaError_t launch_c128_to_c64(const double2 *src, float2 *dst, int64_t n, cudaStream_t s);

}  // namespace tn
