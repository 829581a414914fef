// Internal host-side structures of libtn (not part of the C ABI).
#pragma once
#include <complex>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "tn.h"

namespace tn {

using cd = std::complex<double>;

// A dense tensor with bond dimension 2 on every axis; labels[0] is the most
// significant axis of the row-major value array.
struct Tensor {
    std::vector<int32_t> labels;
    std::vector<cd> data;  // 2^rank values
    int rank() const { return (int)labels.size(); }
};

struct Network {
    std::vector<Tensor> tensors;
    std::vector<int32_t> open;  // amplitude axis order
};

// SSA contraction tree: leaves 0..n-1, step t makes node n + t.
using Tree = std::vector<std::pair<int, int>>;

struct SearchResult {
    Tree tree;
    std::vector<int32_t> sliced;
    double log2_total = 0;   // log2 MACs over all slices
    double log2_width = 0;   // log2 largest intermediate per slice
    double log2_slice = 0;   // log2 MACs per slice
};

// error reporting (thread-local message)
void set_error(const std::string &msg);
int fail(int code, const std::string &msg);

// network.cpp: circuit -> network (single-qubit gates absorbed)
int build_circuit_network(const tn_circuit *c, const uint8_t *fixed_bits, int n_open,
                          const int32_t *open_qubits, Network &out);

// order.cpp: randomised greedy order + greedy slicing
int search_order(const std::vector<std::vector<int32_t>> &labels, const std::vector<int32_t> &open,
                 const tn_search_opts &opts, SearchResult &out);
// the k best distinct trials by the analytic key (over-cap width, total MACs)
int search_order_top(const std::vector<std::vector<int32_t>> &labels, const std::vector<int32_t> &open,
                     const tn_search_opts &opts, int k, std::vector<SearchResult> &out);

// plan.cpp: order search with learned ranking when opts.cost_model is set
int search_ranked(const std::vector<std::vector<int32_t>> &labels, const std::vector<int32_t> &open,
                  const tn_search_opts &opts, SearchResult &out);
// plan.cpp: learned ranking of candidate trees (index of the predicted
// fastest; predicted ms per candidate in pred_ms)
int rank_candidates(const std::vector<std::vector<int32_t>> &labels, const std::vector<int32_t> &open,
                    const std::vector<SearchResult> &cands, const tn_search_opts &opts, std::vector<double> &pred_ms,
                    int &best);

// evaluate a given tree + slice set (log2 costs); returns false on a malformed tree
bool evaluate_tree(const std::vector<std::vector<int32_t>> &labels, const std::vector<int32_t> &open,
                   const Tree &tree, const std::vector<int32_t> &sliced, SearchResult &out);

tn_search_opts default_search_opts();

// plan.cpp: roofline time (ms, all slices) of a tree compiled for `form`
// with batch_log2 batch bits (< 0: the largest batch whose arena fits
// `budget` bytes); negative when the tree does not compile.  With expected,
// a tensor-core GEMM is priced at no less than its epilogue's measured output
// rate (the search's expected-time objective).  Host only.
double tree_roofline_ms(const std::vector<std::vector<int32_t>> &labels, const std::vector<int32_t> &open,
                        const Tree &tree, const std::vector<int32_t> &sliced, tn_form form, int batch_log2,
                        double budget, bool expected = false);
// the arena budget the search and tn_estimate_tree_ms assume when none is
// given: 60% of a GB300's ~275 GiB of free HBM, as tn_plan_create's default
// budget gives on an idle device
constexpr double kNominalArenaBytes = 160.0 * 1073741824.0;

// order.cpp: the network rules tn_plan_create also enforces (each label held
// by one or two tensors, at most once by each; the labels held once are
// exactly the open ones, each listed once); nullptr if they hold, else what
// is wrong
const char *check_network(const std::vector<std::vector<int32_t>> &labels, const std::vector<int32_t> &open);

// order.cpp: Fiduccia-Mattheyses refinement of a two-way split of a graph
// (nb: one entry per shared bond; side: 0/1 per vertex, refined in place;
// the side-0 count stays in [lo, hi]; vertices marked in fixed never move);
// returns the cut
int fm_refine(const std::vector<std::vector<int>> &nb, std::vector<int> &side, const std::vector<char> *fixed, int lo,
              int hi, int max_passes);

// plan.cpp: replace a plan leaf's values by complex128 device data (rounded
// to complex64), stream-ordered
int plan_load_leaf_c128(tn_plan_t plan, int leaf, const double *d_src, CUstream_st *stream);
// plan.cpp: replace a plan leaf's values by host complex64 data, stream-ordered
int plan_load_leaf_host(tn_plan_t plan, int leaf, const float *src, CUstream_st *stream);

}  // namespace tn
