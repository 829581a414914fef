// C-ABI entry points that need no GPU: errors, order search, circuit network.
#include <cstring>
#include <string>

#include "tn_internal.h"

namespace tn {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

const char *last_error_cstr() { return g_err.c_str(); }

}  // namespace tn

using namespace tn;

extern "C" const char *tn_last_error(void) { return last_error_cstr(); }

extern "C" int tn_find_order(int n_tensors, const int32_t *ranks, const int32_t *labels, int n_open,
                             const int32_t *open_labels, const tn_search_opts *opts, int32_t *out_tree,
                             int max_sliced, int32_t *out_sliced, int *out_n_sliced, double *stats) {
    if (n_tensors <= 0 || !ranks || (n_open > 0 && !open_labels) || n_open < 0)
        return fail(TN_ERR_ARG, "tn_find_order: bad arguments");
    std::vector<std::vector<int32_t>> labs(n_tensors);
    size_t off = 0;
    for (int i = 0; i < n_tensors; i++) {
        if (ranks[i] < 0 || ranks[i] > 62) return fail(TN_ERR_ARG, "tn_find_order: rank out of range");
        labs[i].assign(labels + off, labels + off + ranks[i]);
        off += ranks[i];
    }
    std::vector<int32_t> open(open_labels, open_labels + n_open);
    tn_search_opts o = opts ? *opts : default_search_opts();
    SearchResult r;
    int rc = search_ranked(labs, open, o, r);
    if (rc) return rc;
    if ((int)r.sliced.size() > max_sliced) return fail(TN_ERR_ARG, "tn_find_order: max_sliced too small");
    if (out_tree)
        for (size_t t = 0; t < r.tree.size(); t++) {
            out_tree[2 * t] = r.tree[t].first;
            out_tree[2 * t + 1] = r.tree[t].second;
        }
    if (out_sliced)
        for (size_t j = 0; j < r.sliced.size(); j++) out_sliced[j] = r.sliced[j];
    if (out_n_sliced) *out_n_sliced = (int)r.sliced.size();
    if (stats) {
        stats[0] = r.log2_total;
        stats[1] = r.log2_width;
        stats[2] = (double)r.sliced.size();
        stats[3] = r.log2_slice;
    }
    return TN_OK;
}

extern "C" int tn_circuit_network(const tn_circuit *circuit, const uint8_t *fixed_bits, int n_open,
                                  const int32_t *open_qubits, int *n_tensors, int *total_rank,
                                  int64_t *total_elems, int32_t *ranks, int32_t *labels, float *out_data,
                                  int32_t *open_labels) {
    Network net;
    int rc = build_circuit_network(circuit, fixed_bits, n_open, open_qubits, net);
    if (rc) return rc;
    int tr = 0;
    int64_t te = 0;
    for (auto &t : net.tensors) {
        tr += t.rank();
        te += (int64_t)t.data.size();
    }
    if (n_tensors) *n_tensors = (int)net.tensors.size();
    if (total_rank) *total_rank = tr;
    if (total_elems) *total_elems = te;
    if (!out_data) return TN_OK;
    size_t lo = 0, dof = 0;
    for (size_t i = 0; i < net.tensors.size(); i++) {
        const Tensor &t = net.tensors[i];
        if (ranks) ranks[i] = t.rank();
        for (int a = 0; a < t.rank(); a++) labels[lo++] = t.labels[a];
        for (const cd &v : t.data) {
            out_data[dof++] = (float)v.real();
            out_data[dof++] = (float)v.imag();
        }
    }
    if (open_labels)
        for (size_t j = 0; j < net.open.size(); j++) open_labels[j] = net.open[j];
    return TN_OK;
}
