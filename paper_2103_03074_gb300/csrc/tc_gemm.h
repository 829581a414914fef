// Tensor-core (tcgen05) split-precision complex GEMM forms.
#pragma once
#include <cuda_runtime.h>

#include "kernels.h"
#include "tn.h"

namespace tn {

// Optional epilogue that writes C straight into the next step's split planes
// (that step's operand layout and split mode) instead of complex64 C, so no
// separate split pass reads C back.  Output element (h, m, n) goes to plane
// offset scatter(h, hpos) | scatter(m, mpos) | scatter(n, npos).  Within the
// epilogue's half tile (64 rows x 64 columns) the tile bits are enumerated in
// destination order (tb / tpos), so a warp's 64 consecutive elements land in
// as few 128-byte segments per plane as the layout allows.
struct TcPlanarOut {
    int mode;               // 0: complex64 C (no split); else a split mode of BitPermArgs (1-4; 5-7 for 3M GEMMs)
    void *planes;
    int64_t plane_stride;   // elements per plane
    int nH, nM, nN;         // bits of h, m, n
    int8_t hpos[kMaxRank], mpos[kMaxRank], npos[kMaxRank];  // destination bit of each bit
    int ntb;                // tile bits, ordered by destination position:
    int8_t tb[12];          //   0..5 column bit c, 6..11 row bit r (of the half tile)
    int8_t tpos[12];        //   their destination positions
};

// Planar output stored by TMA from shared memory (16-bit planes: bf16 or
// fp16 hi/lo, or scaled fp16): the epilogue writes the half tile's 4,096
// elements of each plane to shared memory in the order of one box of a
// five-dimensional view of the destination, then one bulk tensor store per
// plane writes them.  Dimension 0 = destination bits 0..5 (the half tile's
// 64 lowest destination elements, 128 bytes); each further run of
// consecutive tile-bit positions is a dimension whose box spans the run, each
// gap between runs a dimension with a box of 1; the last dimension runs to
// the top of the planes (plane q at coordinate q * plane_step).
struct TcTmaOut {
    int on;              // 1: planes stored by TMA (tc_prepare decides and encodes mapC)
    int np;              // planes
    int nd;              // dimensions in use (at most 5; the rest have extent 1)
    int8_t start[5];     // destination bit where dimension i starts
    int8_t bits[5];      // log2 of its extent (the last: to the top of a plane)
    int8_t box[5];       // log2 of its box
    int8_t boxbit[12];   // box-order bit of tile bit b (0..5: column c_b, 6..11: row r_(b-6))
    int64_t plane_step;  // last-dimension coordinate distance between planes
};

// One tensor-core GEMM: the GemmArgs contract (C = [H][M][N] contiguous) plus
// the split planes of A (rows = M) and B (rows = N), planes[q][h][row][k], and
// their TMA descriptors.
struct TcGemm {
    GemmArgs a;
    tn_form form;
    void *planesA, *planesB;
    int ksplit;       // K partitions over CTAs (1: none)
    int chunk_bytes;  // K chunk per TMA stage and plane row: 64 or 128 (0: default)
    int flush_bytes;  // bytes of K between accumulator read-outs (multiple of chunk_bytes; 0: default)
    const unsigned *scales;  // FP16S / FP16X3: device max-abs slots of A and B (float bits)
    unsigned *max_slot;      // optional: receives max |re|, |im| of C (float bits; zeroed by the launch)
    TcPlanarOut out;         // out.mode 0: plain complex64 C
    // real products per complex product: 4 (0 = 4: P = A_re [B_re|B_im],
    // Q = A_im [B_re|B_im]) or 3 (Gauss 3M: A_re B_re, A_im B_im and
    // (A_re + A_im)(B_re + B_im); six planes per operand, split modes 5-7;
    // hi/lo forms only)
    int products;
    // plane layout: 0 = [q][h][row][K]; b > 0 = [q][h][K >> b][row][2^b]
    // (K cut into runs of 2^b values, 128 bytes of a plane row, each run
    // stored for all rows before the next: a TMA box of 128 rows reads one
    // contiguous block, whatever K is)
    int k_low_bits;
    int tma_out_ok;    // 1: a planar output may be stored by TMA (tc_prepare decides from its layout)
    TcTmaOut out_tma;  // set by tc_prepare from `out` (out_tma.on 0: stores from the epilogue warps)
    alignas(64) unsigned char mapA[128];
    alignas(64) unsigned char mapB[128];
    alignas(64) unsigned char mapC[128];
};

// log2 of the runs a planar epilogue stores straight from registers (the
// destination's lowest bits are the tile's lowest column bits, full tiles),
// or 0 when it stages the tile through shared memory
int tc_planar_direct_run(const TcPlanarOut &o);
// true if a planar output that the epilogue would stage fits the box view of
// a TMA store (TcTmaOut; 16-bit planes of a four-product form)
bool tc_planar_tma_fits(const TcPlanarOut &o, TcTmaOut *out = nullptr);

// true if `form` has a tensor-core GEMM compiled into this library (and the
// driver entry point for TMA descriptors is reachable)
bool tc_form_available(tn_form form);

// bytes per plane element of a split form (2: bf16 / fp16, 4: tf32)
int tc_plane_bytes(tn_form form);

// planes per operand: 4 for the hi/lo split forms (re_hi, im_hi, re_lo,
// im_lo: BF16x3, TF32x3, FP16X3), 2 for FP16S (re, im); with products == 3
// (the 3M product of the hi/lo forms) 6 (re_hi, im_hi, s_hi, re_lo, im_lo,
// s_lo)
int tc_plane_count(tn_form form, int products = 4);

// true if the form has a 3M variant (the hi/lo split forms)
bool tc_form_has_3m(tn_form form);

// K bytes between accumulator read-outs when TcGemm::flush_bytes is 0: the
// largest interval that keeps the form's accuracy (the read-out interval
// bounds how many MMAs add into one truncating tensor-memory sum)
int tc_default_flush_bytes(tn_form form);

// Shapes the tensor-core kernel takes (smaller GEMMs stay on the FP32
// CUDA-core kernel).
bool tc_gemm_suitable(const GemmArgs &a);

// Encode the TMA descriptors of g (pointers and form filled in); false if the
// driver rejects them.
bool tc_prepare(TcGemm &g);

// A small step on the tensor cores, T split into pieces in shared memory (no
// split pass): for the split forms with K and N of 16 or 32 values, no batch
// bits, at least 2^16 rows, and the rows' 7 lowest bits at T's and C's 7
// lowest positions.  launch_small_tc returns cudaErrorMisalignedAddress when
// T is not 16-byte aligned (the caller then takes the CUDA-core kernel).
bool small_tc_suitable(const SmallArgs &a, tn_form form);
cudaError_t launch_small_tc(const SmallArgs &a, tn_form form, cudaStream_t s);

// K partitions for a GEMM whose tile grid alone would leave SMs idle.
int tc_choose_ksplit(const GemmArgs &a, tn_form form);

cudaError_t launch_gemm_tc(const TcGemm &g, cudaStream_t s);

// Read and clear the device error word of the tensor-core kernels (0 = ok,
// 1 = a bounded mbarrier wait expired); synchronises `s`.
int tc_read_error(cudaStream_t s);

}  // namespace tn
