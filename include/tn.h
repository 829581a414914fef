/*
 * libtn: sliced big-head tensor-network contraction on one GB300 (sm_103a).
 *
 * The operation (Pan & Zhang, "Simulating the Sycamore quantum supremacy
 * circuits", arXiv:2103.03074): a quantum circuit is a tensor network of bond
 * dimension 2 ("Big-head simulation" section, Fig. 1).  Some output qubits are
 * left open, the others are closed on a fixed bitstring s1, so one contraction
 * yields the 2^k amplitudes <s1; s2|U|0> for every assignment s2 of the k open
 * qubits.  A set of n_e bond labels is sliced ("Dynamic slicing" paragraph of
 * the appendix): slice id s holds sliced label j at bit j of s, every slice
 * runs the same pairwise contraction tree (Fig. 3: a pair sharing n_AB labels
 * with n_A, n_B outer labels costs 2^{n_A+n_B+n_AB} complex multiply-adds),
 * and the 2^{n_e} slice results sum to the full contraction.
 *
 * Conventions shared by every call:
 *  - Bond dimension is 2 for every label.  A tensor of rank r holds 2^r
 *    complex values; its first label is the most significant axis
 *    (row-major, like a C-ordered numpy array of shape (2,)*r).
 *  - Complex values are interleaved (re, im).
 *  - Labels are non-negative int32.  Every label is held by at most two
 *    tensors and at most once per tensor; a label held by one tensor must be
 *    open.
 *  - The amplitude tensor over the open labels has the open labels in the
 *    given order, first = most significant bit of the flat index.
 *  - Return value 0 = success; negative = error (TN_ERR_*), with a message
 *    for the calling thread in tn_last_error().
 *  - Device pointers are CUDA device memory of the current device; calls are
 *    ordered on the given stream (0 = legacy default stream).
 */
#ifndef TN_H
#define TN_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tn_plan *tn_plan_t; /* opaque, owned by the library */
typedef struct tn_costmodel *tn_costmodel_t; /* opaque learned step-cost model */
typedef struct tn_batch *tn_batch_t; /* opaque batch of plans run as one graph */
typedef struct CUstream_st *tn_stream_t; /* a cudaStream_t */

enum {
    TN_OK = 0,
    TN_ERR_ARG = -1,     /* bad labels, non-binary tree, sliced label that is open, ... */
    TN_ERR_OOM = -2,     /* device memory for the plan's arena cannot be had */
    TN_ERR_CUDA = -3,    /* a CUDA runtime call or kernel launch failed */
    TN_ERR_TIMEOUT = -4, /* a bounded device-side wait expired */
    TN_ERR_STATE = -5    /* call made on a plan in a failed state */
};

/* Arithmetic form of the pairwise contractions (the cross-slice sum and the
 * probability reduction are FP64 in every form). */
typedef enum {
    TN_FP32 = 0,   /* complex64 operands, FP32 CUDA-core complex products (reference form) */
    TN_BF16X3 = 1, /* operands split into bf16 hi/lo, three products per real product, tensor cores, FP32 accumulate */
    TN_TF32X3 = 2, /* tf32 hi/lo split, three products per real product, tensor cores */
    TN_FP16S = 3,  /* fp16 with per-tensor power-of-two scale, tensor cores */
    TN_FP16X3 = 4  /* per-tensor power-of-two scale, then an fp16 hi/lo split, three products per real
                      product, tensor cores, FP32 accumulate (about the TF32x3 precision at the fp16 rate) */
} tn_form;

typedef struct {
    /* slices executed together: 2^batch_log2 consecutive slice ids run as one
     * pass with the low sliced labels kept as batch labels; -1 = choose from
     * the memory budget */
    int32_t batch_log2;
    /* device bytes the plan may hold (arena + leaves); 0 = 60% of free memory */
    int64_t mem_budget;
    /* record per-step CUDA-event timings on every call (profiling mode) */
    int32_t profile;
    /* CUDA-graph replay: the first tn_contract_slices call runs eagerly, then
     * captures the slice-invariant prologue and the per-block body into two
     * graphs; later calls replay them (the slice extraction and the FP64 sum,
     * whose arguments change per block, stay ordinary launches) */
    int32_t use_graph;
    /* tensor-core GEMM tuning (0 = library default): K bytes per pipeline
     * stage and plane row (64 or 128; the 3M product takes 32, or 64 when
     * 64 is asked for), and K bytes between read-outs of the tensor-memory
     * accumulators into FP32 registers (a multiple of it) */
    int32_t tc_chunk_bytes;
    int32_t tc_flush_bytes;
    /* 0 (default) or 1: a tensor-core GEMM of the BF16x3 / TF32x3 forms whose
     * output feeds the next step's hi/lo split writes that split's planes
     * itself (in the next step's layout) when its epilogue writes stay
     * coalesced, instead of complex64 output plus a split pass; -1: off */
    int32_t tc_planar;
    /* CUDA-graph branches: the captured graphs order each step after the
     * steps it depends on and spread independent steps over this many
     * streams (0 = default 4; 1 = one chain in op order) */
    int32_t graph_branches;
    /* split forms: a step with a small operand (which would run on the
     * CUDA-core small-step kernel) goes to the tensor-core GEMM instead when
     * its K and N both have >= 3 bits, K + N has >= small_tc_bits bits and T
     * has >= 2^16 rows (0 = never, the default: on the 30-qubit workload the
     * extra split pass costs more than the tensor cores save) */
    int32_t small_tc_bits;
    /* small-step kernel: 0 (default) takes the tiled kernel (row tiles staged
     * through shared memory, register-blocked outputs) where K and N are
     * 4..32 wide and T has >= 2^12 rows, else one thread per row; -1: always
     * one thread per row */
    int32_t small_tiled;
    /* split forms BF16X3, TF32X3, FP16X3: real products per complex product on
     * the tensor cores.  0 or 4 (default): four, A_re [B_re|B_im] and
     * A_im [B_re|B_im]; 3: Gauss's 3M product, A_re B_re, A_im B_im and
     * (A_re + A_im)(B_re + B_im), re = T1 - T2, im = T3 - T1 - T2 (a quarter
     * fewer tensor-core flops; each operand then has six planes, the third
     * value s = re + im split like re and im) */
    int32_t tc_products;
    /* tiny small steps (T and C of at most 2^small_tasks elements each, at
     * most 2^7 K values; 0 = default 17): the ones whose inputs are leaves or
     * each other's outputs run as the tasks of one persistent launch, which
     * orders them by device-side completion counters (bounded waits) instead
     * of one kernel launch each; -1: off */
    int32_t small_tasks;
    /* split forms (TF32X3, FP16X3, BF16X3): 0 (default) runs a large small
     * step (K of 16 or 32 values, N of 8, 16 or 32, at least 2^16 rows, no batch labels,
     * its rows' 7 lowest bits lowest in T and C) on the tensor cores, T split
     * into pieces in shared memory (each 128-row tile of T scaled by its own
     * power of two in FP16X3) with the form's products; -1: CUDA cores */
    int32_t small_tc;
    /* split forms with 16-bit planes (BF16X3, FP16X3, FP16S, four products):
     * 0 (default) lets a GEMM whose planar output would be staged through
     * shared memory and stored by its epilogue warps write the planes to
     * shared memory in the order of a destination box instead, stored by TMA
     * (where the half tile's destination bits fit a five-dimensional box
     * view whose rows are 128 bytes, in GEMMs whose tiles have more than one
     * accumulator read-out); -1: off */
    int32_t tc_tma_store;
} tn_plan_opts;

/* Order search options (host-side planning). */
typedef struct {
    int32_t trials;     /* order trials, greedy or bipartition (method below; default 256) */
    uint64_t seed;      /* seed of the search's SplitMix64 stream */
    int32_t log2_cap;   /* slice until every intermediate has <= 2^log2_cap elements (-1: no cap) */
    int32_t n_sliced;   /* slice exactly this many labels (-1: as the cap needs) */
    int32_t threads;    /* host threads (0 = hardware concurrency) */
    /* learned ranking: with cost_model set and candidates > 1, the best
     * `candidates` trees by the analytic cost are compiled (for rank_form, with
     * 2^rank_batch_log2 slices per pass, -1 = all sliced labels) and the one
     * with the smallest predicted device time wins; otherwise the analytic
     * cost (total complex MACs over all slices) decides */
    int32_t candidates;
    int32_t rank_batch_log2;
    int32_t rank_form;
    tn_costmodel_t cost_model;
    /* trial kind: 0 randomised greedy (default); 1 hierarchical bipartition
     * (appendix, "Finding contraction order using hierarchical
     * partitioning": min-cut splits down to parts of a few dozen tensors,
     * greedy inside a part; trial 0 takes the paper's parts of <= 60
     * tensors, the others draw the balance window and part size); 2 both,
     * alternating.  Slicing and subtree reconfiguration follow either way. */
    int32_t method;
    /* what ranks the trials: 0 total complex MACs over all slices (default);
     * 1 the roofline time of the tree compiled for rank_form with
     * 2^rank_batch_log2 slices per block (-1: the largest block whose arena
     * fits 160 GiB), as tn_estimate_tree_ms prices it; 2 that time with each
     * tensor-core GEMM priced at no less than its output elements over the
     * rate its epilogue writes them (measured on GB300: ~2.2e11 elements/s
     * into split planes, ~4e11 as complex64), the bound of short-K GEMMs.
     * Either way the learned ranking (cost_model, candidates) then picks
     * among the best. */
    int32_t objective;
} tn_search_opts;

/* A circuit: gate g acts on gate_nq[g] (1 or 2) qubits gate_q[2g], gate_q[2g+1]
 * with the row-major 2^k x 2^k complex matrix at gate_m[32 g ...] (interleaved
 * re/im; 8 or 32 doubles used).  Qubit 0 is the first character of a
 * bitstring.  The initial state is |0...0>. */
typedef struct {
    int32_t n_qubits;
    int32_t n_gates;
    const int32_t *gate_nq;
    const int32_t *gate_q;
    const double *gate_m;
} tn_circuit;

/*
 * Build a plan for the sliced contraction of a tensor network
 * ("Dynamic slicing" paragraph; Fig. 3 pairwise steps).
 *   ranks[n_tensors]            rank of each tensor
 *   labels[sum ranks]           concatenated label lists (host)
 *   data[2 * sum 2^rank]        concatenated interleaved complex64 values (host, copied;
 *                               NULL: the leaves start as zeros and are set later
 *                               with tn_plan_update_data)
 *   n_labels, bond_dims         bond_dims[label] must be 2 for every label used (may be NULL)
 *   open_labels[n_open]         amplitude-tensor axis order, [0] = MSB
 *   sliced_labels[n_sliced]     slice id bit j -> sliced_labels[j]; must not be open
 *   tree[2 * n_steps]           n_steps = n_tensors - 1 pairs (i, j) of SSA node ids:
 *                               leaves are 0..n_tensors-1, step t makes node n_tensors + t
 * All host arrays are copied; the plan owns its device memory.
 * Errors: TN_ERR_ARG (malformed input), TN_ERR_OOM, TN_ERR_CUDA.
 */
int tn_plan_create(tn_plan_t *out, int n_tensors, const int32_t *ranks, const int32_t *labels,
                   const float *data, int n_labels, const int32_t *bond_dims, int n_open,
                   const int32_t *open_labels, int n_sliced, const int32_t *sliced_labels,
                   int n_steps, const int32_t *tree, tn_form form, const tn_plan_opts *opts);

/*
 * Contract slices [slice_begin, slice_end) and ADD their sum into d_amp
 * (device, complex128 interleaved, 2^n_open entries, caller-owned).  Additive,
 * so ranges compose; an empty range adds nothing.  The range must lie in
 * [0, 2^n_sliced).  Stream-ordered on `stream`; the call returns after
 * enqueueing (no host synchronisation) unless profiling is on.
 * Errors: TN_ERR_ARG (range), TN_ERR_CUDA, TN_ERR_TIMEOUT, TN_ERR_STATE.
 */
int tn_contract_slices(tn_plan_t plan, int64_t slice_begin, int64_t slice_end, double *d_amp,
                       tn_stream_t stream);

/*
 * The sliced contraction with host buffers ("Dynamic slicing": slices
 * [slice_begin, slice_end) summed in FP64), for callers that keep their data
 * on the host: copies new leaf values in (h_data, host complex64 interleaved
 * in tn_plan_create's concatenated layout, the plan's leaf count of values;
 * NULL keeps the current values), zeroes a plan-owned device amplitude
 * tensor, contracts the range into it, and when h_stats is given computes
 * the probabilities' sums of Eq. 1 on the device (h_stats[3] = {P(s1),
 * linear XEB, max p} for n_qubits qubits); then copies the amplitudes to
 * h_amp (host complex128, 2^n_open entries; may be NULL) and synchronises the
 * stream.  Pinned host memory makes the copies asynchronous to the host up to
 * that synchronisation.  The first call allocates the plan's device
 * amplitude tensor (2^n_open x 16 bytes + 24 bytes).
 * Errors: as tn_contract_slices, TN_ERR_ARG (n_qubits < n_open with
 * h_stats), TN_ERR_OOM.
 */
int tn_contract_slices_host(tn_plan_t plan, int64_t slice_begin, int64_t slice_end, const float *h_data,
                            int n_qubits, double *h_amp, double *h_stats, tn_stream_t stream);

/*
 * Amplitudes of a circuit over its open qubits (the big-head problem of the
 * "Big-head simulation" section): build the network (single-qubit gates
 * absorbed into two-qubit gates, boundary vectors absorbed), search an order
 * and a slice set (search may be NULL for defaults), plan, contract every
 * slice and OVERWRITE d_amp (device complex128, 2^n_open entries).
 *   fixed_bits[n_qubits]   the closed bits s1 (entries at open positions ignored)
 *   open_qubits[n_open]    amplitude axis order, [0] = MSB
 * Synchronises `stream` before returning.
 */
int tn_amplitudes(const tn_circuit *circuit, const uint8_t *fixed_bits, int n_open,
                  const int32_t *open_qubits, tn_form form, const tn_search_opts *search,
                  const tn_plan_opts *opts, double *d_amp, tn_stream_t stream);

/*
 * Probabilities and linear XEB (Eq. 1) of an amplitude tensor on the device, in
 * FP64 (marginal and conditional probabilities: appendix on P(s1), P(s2|s1)).
 * Writes d_prob[i] = |amp_i|^2 (may be NULL) and d_out[3] (device, required):
 * d_out[0] = sum_i p_i (the marginal P(s1)), d_out[1] = F_XEB = 2^n_qubits / L *
 * sum p - 1 with L = 2^n_open, d_out[2] = max p.  If `out` (host, 3 doubles) is
 * non-NULL the three values are copied there and `stream` is synchronised;
 * otherwise the call only enqueues work.
 */
int tn_probabilities_xeb(const double *d_amp, int n_open, int n_qubits, double *d_prob,
                         double *d_out, double *out, tn_stream_t stream);

/*
 * Post-selection ("Fidelity" paragraph, Eq. 1, Fig. 2 right): the
 * probabilities p_i = re_i^2 + im_i^2 (FP64, products and sum rounded
 * separately) of the amplitude tensor d_amp (device complex128, 2^n_open
 * entries, interleaved re/im) are sorted in decreasing order on the device,
 * and for each of the n_points counts N_j (host int64, 1 <= N_j <= 2^n_open)
 * out_xeb[j] (host) receives the XEB of the N_j most probable bitstrings,
 * F_j = 2^n_qubits / N_j * (sum of the N_j largest p) - 1.  d_order (device
 * int64 [2^n_open], may be NULL) receives the indices in that order (equal
 * probabilities in any order).  n_open <= 31, n_points <= 65535.  Device
 * scratch (12 bytes per entry plus small arrays) comes from the stream-ordered
 * allocator and is released before return; the call synchronises `stream`.
 * Errors: TN_ERR_ARG (bad sizes or counts), TN_ERR_OOM, TN_ERR_CUDA.
 */
int tn_postselect_xeb(const double *d_amp, int n_open, int n_qubits, int n_points, const int64_t *counts,
                      double *out_xeb, int64_t *d_order, tn_stream_t stream);

/*
 * Sampling from the conditional distribution P(s2|s1) = P(s1;s2) / P(s1)
 * (appendix on conditional and marginal probabilities) by inverse
 * transform: with the cumulative probabilities c_i = sum_{i' <= i} p_i' in
 * index order (FP64), sample j is the smallest index i with c_i > u_j * P(s1),
 * P(s1) = sum of all p.  The uniform numbers are inputs: d_u (device double
 * [n_samples], each in [0, 1)); d_out (device int64 [n_samples]) receives
 * amplitude indices (bit j of the index = open qubit j, MSB first).  Stream-
 * ordered; scratch of 8 bytes per entry from the stream-ordered allocator.
 * n_open <= 40.  Errors: TN_ERR_ARG, TN_ERR_OOM, TN_ERR_CUDA.
 */
int tn_conditional_sample(const double *d_amp, int n_open, int64_t n_samples, const double *d_u, int64_t *d_out,
                          tn_stream_t stream);

/*
 * Histogram of x_i = p_i * scale over n_bins equal bins of [0, x_max) plus an
 * overflow bin (Fig. 2 left with scale = 2^n_qubits; Fig. 5 with scale =
 * 2^n_open / P(s1)): bin b = floor(x / (x_max / n_bins)) computed in FP64
 * (clamped to n_bins - 1 below x_max), bin n_bins counts x >= x_max.
 * d_counts: device int64 [n_bins + 1], overwritten.  n_bins <= 4096.
 * Stream-ordered.  Errors: TN_ERR_ARG, TN_ERR_CUDA.
 */
int tn_probability_histogram(const double *d_amp, int n_open, double scale, int n_bins, double x_max,
                             int64_t *d_counts, tn_stream_t stream);

/*
 * Replace the leaf values of a plan (same layout as tn_plan_create's `data`,
 * host memory, pinned or pageable) with an asynchronous copy on `stream`; the
 * next tn_contract_slices on that stream sees the new values.  The host
 * buffer must stay valid until the copy completes.
 */
int tn_plan_update_data(tn_plan_t plan, const float *data, tn_stream_t stream);

/*
 * Step-timing recorder.  With tn_plan_opts.profile = 1 every kernel of a
 * tn_contract_slices call is bracketed by CUDA events and the call
 * synchronises; durations accumulate per op.  Writes up to max_rows rows of 12
 * doubles: {phase (0 slice-invariant prologue, 1 per slice block), op index,
 * kind (0 small step, 1 permute, 2 GEMM, 3 extract, 4 FP64 sum, 5 hi/lo split, 6 max-abs of a scaled form), tree step,
 * total ms, launches, complex MACs per launch, algorithmic bytes per launch,
 * shape[4]} with shape = {H, M, N, K} for a GEMM, {H, rows, 0, K} for a split,
 * {batch bits, rows, 2^N, 2^K} for a small step, {0, elements, 0, 0} for a permute
 * and returns the number of rows (negative on error).  reset != 0 clears the
 * totals after reading.
 */
int tn_plan_profile(tn_plan_t plan, int max_rows, double *rows, int reset);

void tn_plan_destroy(tn_plan_t plan);

/* Message of the calling thread's last error ("" if none). */
const char *tn_last_error(void);

/*
 * Host-side order search (first pairwise order, then slicing): randomised
 * greedy or hierarchical-bipartition trials (opts->method) scored by the
 * Fig. 3 cost 2^{n_A+n_B+n_AB} summed over steps, then greedy slicing to the
 * cap or count and subtree reconfiguration of the best trees.  TN_ERR_ARG
 * for an unknown method, or a network that breaks tn_plan_create's rules
 * (a label held by more than two tensors or twice by one, a label held once
 * that is not open, an open label held twice or listed twice).  Writes the tree (2*(n_tensors-1)
 * SSA ids), the sliced labels (up to max_sliced) and stats[4] =
 * {log2 total MACs over all slices, log2 largest intermediate per slice,
 *  n_sliced, log2 MACs per slice}.
 */
int tn_find_order(int n_tensors, const int32_t *ranks, const int32_t *labels, int n_open,
                  const int32_t *open_labels, const tn_search_opts *opts, int32_t *out_tree,
                  int max_sliced, int32_t *out_sliced, int *out_n_sliced, double *stats);

/*
 * Analytic time of a tree (the FLOP/memory fallback of the learned cost
 * model): the plan tn_plan_create would build for `form` is compiled on the
 * host (no CUDA call) and every op is priced at its roofline time, the
 * larger of its algorithmic bytes over 7 TB/s and its flops over its unit's
 * peak (FP32 CUDA cores 80 TFLOP/s, tensor cores 2.25 PFLOP/s, 1.125 for
 * TF32x3), plus 2 us per launch; the slice-invariant prologue counts once,
 * the per-block body once per block.  The block holds 2^batch_log2 slices
 * (capped at n_sliced); batch_log2 < 0 takes the largest block whose arena
 * and leaves fit arena_budget bytes (<= 0: 160 GiB), as tn_plan_create
 * sizes it.  Network, sliced labels, tree and opts (plan options, may be
 * NULL; their batch_log2 is ignored) as for tn_plan_create (same checks,
 * TN_ERR_ARG).  *out_ms: milliseconds for all 2^n_sliced slices,
 * = *out_prologue_ms + 2^(n_sliced - *out_batch_log2) * *out_block_ms;
 * out_batch_log2, out_arena (arena bytes), out_prologue_ms (the
 * slice-invariant ops) and out_block_ms (one block) may be NULL.
 */
int tn_estimate_tree_ms(int n_tensors, const int32_t *ranks, const int32_t *labels, int n_open,
                        const int32_t *open_labels, int n_sliced, const int32_t *sliced_labels, int n_steps,
                        const int32_t *tree, tn_form form, const tn_plan_opts *opts, int batch_log2,
                        int64_t arena_budget, double *out_ms, int *out_batch_log2, int64_t *out_arena,
                        double *out_prologue_ms, double *out_block_ms);

/*
 * The plan tn_estimate_tree_ms prices, as text: one line per compiled op as
 * tn_plan_describe writes it (phase, step, kind, shape, kernel variant,
 * plan-time notes), each with its roofline_ms; no CUDA call.  Arguments as
 * for tn_estimate_tree_ms.  Writes up to cap - 1 characters and a NUL to out
 * (cap 0: out may be NULL) and returns the full length, or a negative error.
 */
int tn_describe_tree(int n_tensors, const int32_t *ranks, const int32_t *labels, int n_open,
                     const int32_t *open_labels, int n_sliced, const int32_t *sliced_labels, int n_steps,
                     const int32_t *tree, tn_form form, const tn_plan_opts *opts, int batch_log2,
                     int64_t arena_budget, char *out, int cap);

/*
 * Slicing a given tree ("Dynamic slicing" paragraph): the search's greedy
 * slicing (two rules, the cheaper result that meets the cap wins) applied
 * to the caller's tree, until every intermediate has <= 2^log2_cap elements
 * (log2_cap < 0: no cap) or, with n_sliced >= 0, exactly n_sliced labels.
 * Network and tree as for tn_plan_create (same checks, TN_ERR_ARG).  Writes
 * the sliced labels (up to max_sliced; TN_ERR_ARG when more are needed),
 * their count and stats[4] as tn_find_order does.
 */
int tn_slice_tree(int n_tensors, const int32_t *ranks, const int32_t *labels, int n_open, const int32_t *open_labels,
                  int n_steps, const int32_t *tree, int log2_cap, int n_sliced, int max_sliced, int32_t *out_sliced,
                  int *out_n_sliced, double *stats);

/*
 * Branch merging (appendix, "Details of simulations"): in a tree, a large
 * tensor X met by two small ones in turn, ((X a) b), is rewritten as
 * (X (a b)) when a, b and their product have rank <= max_small_rank (0: 12)
 * and a per-step time estimate drops by at least 5% (the larger of the
 * step's bytes over 7 TB/s and its FP32 flops over 80 TFLOP/s, sliced labels
 * kept as batch labels); repeated until nothing improves.  The result is the
 * same contraction (pairwise contraction is associative).  tree_out receives
 * the rewritten SSA tree (2 * (n_tensors - 1) ids, may alias tree_in);
 * stats[3] = {rewrites, log2 MACs per block before, after}.
 */
int tn_merge_branches(int n_tensors, const int32_t *ranks, const int32_t *labels, int n_open,
                      const int32_t *open_labels, int n_sliced, const int32_t *sliced_labels, int n_steps,
                      const int32_t *tree_in, int max_small_rank, int32_t *tree_out, double *stats);

/*
 * Order search for the two-stage big-head form ("Big-head simulation"
 * section, Fig. 1; appendix on the first cut): the tail starts with every
 * tensor holding an open label and grows one neighbouring tensor at a time,
 * always the one leaving the smallest cut, up to tail_max tensors (0: half
 * the network); the prefix with the smallest cut is kept.  With
 * opts->method >= 1 (bipartition) that tail is then refined by
 * Fiduccia-Mattheyses passes, the open-leg tensors held in the tail and its
 * size kept within the limit.  Then the head's
 * order is searched with the cut labels as its open labels (sliced as opts'
 * cap or count asks; the sliced labels are internal to the head) and the
 * tail's with cut + open labels (not sliced), and the two trees are joined
 * at the root: out_tree (2 * (n_tensors - 1) SSA ids) has the cut at its
 * last step.  stats[7] = {log2 head MACs per slice, log2 head width,
 * head slices, log2 tail MACs, log2 tail width, cut bonds, log2 total MACs}.
 */
int tn_find_order_head_tail(int n_tensors, const int32_t *ranks, const int32_t *labels, int n_open,
                            const int32_t *open_labels, int tail_max, const tn_search_opts *opts, int32_t *out_tree,
                            int max_sliced, int32_t *out_sliced_head, int *out_n_sliced_head, double *stats);

/*
 * Open qubits chosen from the first cut ("Big-head simulation" section: the
 * open qubits are those whose last tensors fall in G_tail, a small region
 * behind a narrow cut; the appendix tries first cuts until the contraction's
 * cost is acceptable).  In the circuit's network with every qubit open
 * (gates absorbed as tn_circuit_network builds it), a connected tail grows
 * from each tensor holding a qubit's last wire segment, one neighbouring
 * tensor at a time, always the one leaving the smallest cut among those that
 * keep at most n_open qubit ends in the tail (ties: more qubit ends, then the
 * lower tensor id, or in 15 more growths per seed a random one from a fixed
 * SplitMix64 stream), up to half the network.  Every tail holding exactly
 * n_open ends is a candidate.  Without opts the smallest cut wins; with opts
 * the order search (opts as for tn_find_order) prices the network of each of
 * the 8 smallest-cut candidates and the cheapest wins.  Writes the open
 * qubits (n_open, increasing), the tail's tensor ids in the all-open network
 * (out_tail, room for its tensor count; may be NULL), their count, the cut
 * (bonds between tail and head) and *out_log2_cost (log2 total MACs of the
 * winner's search, or log2 of its plan's roofline (objective 1) or expected
 * (objective 2) ms: the measure the candidates are compared by; -1 without
 * opts; may be NULL).  TN_ERR_ARG unless
 * 1 <= n_open < n_qubits, or when no connected tail holds exactly n_open
 * ends.
 */
int tn_choose_open_qubits(const tn_circuit *circuit, int n_open, const tn_search_opts *opts, int32_t *out_open_qubits,
                          int32_t *out_tail, int *out_n_tail, int *out_cut, double *out_log2_cost);

/*
 * The candidate open sets of tn_choose_open_qubits, in the order it takes
 * them: every connected tail with exactly n_open qubit ends that its growths
 * reach, sorted by cut (ties in growth order); with search options the
 * chooser prices the first 8.  Writes min(max_out, count) candidates: open
 * qubits to out_qubits[i * n_open ...] (increasing) and the cut to
 * out_cuts[i]; *out_n = the full count.  Host memory only; no GPU needed.
 * TN_ERR_ARG unless 1 <= n_open < n_qubits, or when no tail qualifies.
 */
int tn_open_qubit_candidates(const tn_circuit *circuit, int n_open, int max_out, int32_t *out_qubits, int *out_cuts,
                             int *out_n);

/*
 * Stage-2 slicing for tn_head_tail_amplitudes: its stage-2 network (the
 * tail's tensors, then v_head over the cut as one more leaf, joined at the
 * root of the tail's subtree) sliced by tn_slice_tree until every
 * intermediate has <= 2^log2_cap elements.  The sliced labels are tail or
 * cut labels, never open ones, as sliced_tail must be.  Tree and network as
 * for tn_head_tail_amplitudes (the root step joins the head, without open
 * legs, and the tail); TN_ERR_ARG otherwise, or when more than max_sliced
 * labels are needed.  stats[4] as tn_find_order's.
 */
int tn_slice_stage2(int n_tensors, const int32_t *ranks, const int32_t *labels, int n_open, const int32_t *open_labels,
                    int n_steps, const int32_t *tree, int log2_cap, int max_sliced, int32_t *out_sliced_tail,
                    int *out_n_sliced, double *stats);

/*
 * Two-stage big-head contraction ("Big-head simulation" section): the
 * tree's last step must join the head (no open label) and the tail (every
 * open label); the labels they share are the first cut C.  Stage 1
 * contracts the head, summed over sliced_head (labels internal to the
 * head), into v_head over C (complex128, FP64 sum; axes C in increasing
 * label order, first = most significant).  Stage 2 contracts the tail with
 * v_head as one more leaf (rounded to complex64), summed over sliced_tail
 * (tail labels or cut labels, not open), into d_amp (device complex128
 * [2^n_open], overwritten).  v_head depends only on the closed bits, so one
 * head contraction serves every assignment of the open qubits; slicing cut
 * bonds in stage 2 bounds the tail's intermediates.  d_vhead (device
 * complex128 [2^|C|], may be NULL) receives v_head; *n_cut (may be NULL)
 * receives |C|.  Network arguments, forms and options as for
 * tn_plan_create; the two plans are built, run and released inside the
 * call, which synchronises `stream`.  Errors: TN_ERR_ARG when the root
 * step is not such a cut, a sliced label is on the wrong side or |C| > 40;
 * else as tn_plan_create and tn_contract_slices.
 */
int tn_head_tail_amplitudes(int n_tensors, const int32_t *ranks, const int32_t *labels, const float *data,
                            int n_open, const int32_t *open_labels, int n_steps, const int32_t *tree,
                            int n_sliced_head, const int32_t *sliced_head, int n_sliced_tail,
                            const int32_t *sliced_tail, tn_form form, const tn_plan_opts *opts, double *d_amp,
                            double *d_vhead, int *n_cut, tn_stream_t stream);

/*
 * The network tn_amplitudes contracts for a circuit (gate absorption and
 * boundary vectors applied), with bonds named by the wire-segment convention:
 * the segment after the t-th gate on qubit q is label offset_q + t,
 * offset_q = sum_{q'<q} (gates on q' + 1).  Two calls: first with
 * out_data == NULL to get *n_tensors and *total_rank, then with buffers of
 * ranks[n_tensors], labels[total_rank], data[2 * sum 2^rank] (complex64),
 * open_labels[n_open].
 */
int tn_circuit_network(const tn_circuit *circuit, const uint8_t *fixed_bits, int n_open,
                       const int32_t *open_qubits, int *n_tensors, int *total_rank,
                       int64_t *total_elems, int32_t *ranks, int32_t *labels, float *out_data,
                       int32_t *open_labels);

/*
 * Allocation-free split-precision complex GEMM (the paper has no counterpart;
 * this is a service of the library, not a step of the method).
 *
 * For callers that cannot allocate device memory where they need a product
 * (an allocator owned by another framework with a fixed budget, real-time
 * loops that must not enter the driver's allocator, code handed only device
 * buffers): C = A B with complex64 A [M][K], B [K][N], C [M][N], all row-major,
 * interleaved (re, im), device pointers owned by the caller; C is overwritten.
 * form must be TN_TF32X3 or TN_BF16X3 (the same tensor-core kernels as the
 * plan's GEMM steps).  M, N, K powers of two, M >= 64, N >= 32, K >= 32.
 *
 * Scratch: a fixed 32 MiB __device__ array inside the library, held by every
 * GPU that loads the library until process exit; the hi/lo planes need
 * 4 * e * (M + N) * K bytes (e = 4 for TF32X3, 2 for BF16X3) and larger
 * problems are rejected with TN_ERR_ARG.  No call allocates or frees memory.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the array and each call
 * overwrites the part it uses, so calls that overlap on the GPU (other
 * streams, other host threads) race; order them on one stream.
 * Synchronous: after launching, the call reads and clears the library's
 * device error word (the GEMM's pipeline waits are bounded), which waits for
 * the stream; C is complete when the call returns TN_OK.
 * Errors: TN_ERR_ARG (sizes, form, NULL), TN_ERR_CUDA, TN_ERR_TIMEOUT (a
 * bounded pipeline wait expired; C is then incomplete).
 */
int tn_gemm_split_noalloc(const float *d_A, const float *d_B, float *d_C, int64_t M, int64_t N, int64_t K,
                          tn_form form, tn_stream_t stream);

/*
 * Learned step-cost model: an MLP (16 features -> 64 -> 64 -> 1, ReLU, FP32)
 * that predicts, from the step features of tn_plan_op_features, log2 of a
 * step's device time over its roofline time (feature 14); the predicted time
 * in ms is 2^(output + 16 * feature 14).  Trained on the GPU by the library's own forward,
 * backward and Adam kernels on timings from tn_plan_profile.  Not a step of
 * the paper's method: it ranks candidate contraction trees for the search.
 *   create: seeded He-normal initialisation.
 *   params: copy the flat parameter vector out (get) and/or in (set), host
 *           memory, n_params floats (W1[64][16], b1, W2[64][64], b2, w3, b3).
 *   grad:   mean-squared-error loss and its gradient for device features
 *           d_X[n][16] and targets d_T[n]; gradient copied to d_grad (device,
 *           n_params floats, may be NULL); loss to host (synchronises).
 *   train:  `epochs` full-batch Adam steps (learning rate lr); final loss to
 *           host (synchronises).
 *   predict: d_Y[n] = model(d_X), stream-ordered.
 */
int tn_costmodel_create(tn_costmodel_t *out, uint64_t seed);
void tn_costmodel_destroy(tn_costmodel_t cm);
int tn_costmodel_params(tn_costmodel_t cm, float *get, const float *set, int *n_params);
int tn_costmodel_grad(tn_costmodel_t cm, const float *d_X, const float *d_T, int64_t n, float *d_grad,
                      double *loss, tn_stream_t stream);
int tn_costmodel_train(tn_costmodel_t cm, const float *d_X, const float *d_T, int64_t n, int epochs, float lr,
                       double *final_loss, tn_stream_t stream);
int tn_costmodel_predict(tn_costmodel_t cm, const float *d_X, float *d_Y, int64_t n, tn_stream_t stream);

/*
 * Step features (16 floats per kernel step, in the order of tn_plan_profile's
 * rows without the extraction and FP64-sum rows): kind one-hot {small step,
 * permute, FP32 GEMM, tensor-core GEMM, hi/lo split}, log2(MACs+1)/32,
 * log2(bytes+1)/32, log2 of the four shape entries /32, TF32 flag, BF16 flag,
 * log2(parallel work units, K partitions included)/32, log2(roofline ms)/16, 1.
 * The roofline time is max(bytes / 7 TB/s, flops / peak of the unit) + 2 us,
 * peaks 80 TFLOP/s FP32 (8 flops per complex MAC) and 2.25 (tf32: 1.125)
 * PFLOP/s tensor (24 flops per complex MAC, 8 for FP16S).  Returns the number
 * of steps written (at most max_ops) or a negative error.
 */
int tn_plan_op_features(tn_plan_t plan, float *out, int max_ops);

/*
 * Batch of independent plans (many circuits of uneven size, each with its own
 * slices) run together.  The batch borrows the plans and their amplitude
 * buffers (device complex128, 2^n_open each; plans and buffers must outlive
 * the batch).  tn_batch_run OVERWRITES each buffer with the sum over all of
 * that plan's slices.  The first run is eager on `stream` and synchronises it;
 * it then captures one CUDA graph in which the plans are spread over
 * n_streams concurrent branches (longest job first by complex MACs); later
 * runs are one graph launch on `stream`.
 */
int tn_batch_create(tn_batch_t *out, int n_plans, const tn_plan_t *plans, double *const *d_amps, int n_streams);
int tn_batch_run(tn_batch_t batch, tn_stream_t stream);
void tn_batch_destroy(tn_batch_t batch);

/*
 * Autotuner for the plan's tensor-core GEMM steps: times each of them under a
 * few (K chunk bytes, accumulator read-out bytes) configurations on the
 * plan's current buffers (reps timed launches each, CUDA events on `stream`)
 * and keeps the fastest.  Results are cached for the process by step
 * signature (form, H, M, N, K), so later plans with the same steps reuse
 * them without timing.  Synchronises `stream`; the GEMM outputs in the arena
 * are overwritten (call it before contracting, or contract again after).
 * Drops CUDA graphs captured before (they are recaptured on the next call).
 */
int tn_plan_autotune(tn_plan_t plan, int reps, tn_stream_t stream);

/* Per-plan statistics: out[0] MACs per slice batch, out[1] slices per batch,
 * out[2] arena bytes, out[3] number of steps, out[4] kernel launches per
 * batch, out[5] algorithmic HBM bytes per batch, out[6] MACs of the
 * slice-invariant prologue (computed once per call), out[7] its bytes,
 * out[8] its launches, out[9] log2 slices per batch, out[10] calls served by
 * CUDA-graph replay.  out must hold 11 doubles. */
int tn_plan_stats(tn_plan_t plan, double *out);

/*
 * Text description of a plan's compiled ops, one line each, in execution
 * order (slice-invariant prologue first, then the per-block body): step,
 * kind, shape and the kernel variant chosen (small-step kernel and store
 * mode, tensor-core or FP32 GEMM, split-K, planar outputs), with notes on
 * declined fusions.  Writes at most cap - 1 characters and a terminating
 * NUL to out (host, may be NULL when cap is 0); returns the full length.
 */
int tn_plan_describe(tn_plan_t plan, char *out, int cap);

#ifdef __cplusplus
}
#endif
#endif /* TN_H */
