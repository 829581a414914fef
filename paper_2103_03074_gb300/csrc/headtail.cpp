// Two-stage big-head contraction ("Big-head simulation" section, Fig. 1).
//
// A first cut C splits the network into a head (every closed qubit, no open
// leg) and a tail (every open leg).  Stage 1 contracts the head into
// v_head over C, summed over the head's own sliced bonds in FP64; stage 2
// contracts the tail with v_head as one more leaf into the amplitudes of
// every assignment of the open qubits.  Both stages are ordinary plans, so
// every step runs in the library's kernels.
//
// The order search for this form grows the tail from the tensors holding
// open legs, one neighbouring tensor at a time, always the one that leaves
// the smallest cut, and keeps the prefix with the smallest cut (the paper
// partitions with a clustering algorithm under size constraints; this is a
// greedy stand-in); then it searches each side's pairwise order separately
// and joins them at the root.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <set>
#include <unordered_map>
#include <vector>

#include "tn.h"
#include "tn_internal.h"

namespace tn {
namespace {

std::vector<std::vector<int32_t>> parse_labels(int n, const int32_t *ranks, const int32_t *labels) {
    std::vector<std::vector<int32_t>> out(n);
    size_t off = 0;
    for (int i = 0; i < n; i++) {
        out[i].assign(labels + off, labels + off + ranks[i]);
        off += ranks[i];
    }
    return out;
}

// an SSA tree over n leaves: every id in range, every node used once
bool valid_tree(int n, const Tree &tree) {
    std::vector<char> used(n + tree.size(), 0);
    for (size_t t = 0; t < tree.size(); t++) {
        const int lim = n + (int)t, a = tree[t].first, b = tree[t].second;
        if (a < 0 || b < 0 || a >= lim || b >= lim || a == b || used[a] || used[b]) return false;
        used[a] = used[b] = 1;
    }
    return true;
}

void mark_subtree(int node, int n, const Tree &tree, std::vector<char> &in) {
    std::vector<int> st{node};
    while (!st.empty()) {
        const int x = st.back();
        st.pop_back();
        in[x] = 1;
        if (x >= n) {
            st.push_back(tree[x - n].first);
            st.push_back(tree[x - n].second);
        }
    }
}

// The steps of the subtree rooted at `root`, renumbered for a network whose
// leaves are `leaves` in that order (leaf ids become positions; steps keep
// their original order).  Returns the new id of the root.
int sub_tree(int root, int n, const Tree &tree, const std::vector<int> &leaves, Tree &out) {
    std::vector<char> in(n + tree.size(), 0);
    mark_subtree(root, n, tree, in);
    std::unordered_map<int, int> id;
    for (size_t i = 0; i < leaves.size(); i++) id[leaves[i]] = (int)i;
    int next = (int)leaves.size();
    for (size_t t = 0; t < tree.size(); t++) {
        const int node = n + (int)t;
        if (!in[node]) continue;
        out.push_back({id.at(tree[t].first), id.at(tree[t].second)});
        id[node] = next++;
    }
    return id.at(root);
}

std::set<int32_t> labels_of(const std::vector<std::vector<int32_t>> &labs, const std::vector<int> &leaves) {
    std::set<int32_t> s;
    for (int i : leaves) s.insert(labs[i].begin(), labs[i].end());
    return s;
}

// flatten (ranks, labels, data) of a sub-network
void gather_net(const std::vector<std::vector<int32_t>> &labs, const float *data, const std::vector<int64_t> &off,
                const std::vector<int> &leaves, std::vector<int32_t> &ranks, std::vector<int32_t> &flat,
                std::vector<float> &vals) {
    for (int i : leaves) {
        ranks.push_back((int32_t)labs[i].size());
        flat.insert(flat.end(), labs[i].begin(), labs[i].end());
        const int64_t n = (int64_t)2 << labs[i].size();
        vals.insert(vals.end(), data + off[i], data + off[i] + n);
    }
}

struct PlanGuard {
    tn_plan_t p = nullptr;
    ~PlanGuard() {
        if (p) tn_plan_destroy(p);
    }
};

}  // namespace
}  // namespace tn

using namespace tn;

extern "C" int tn_head_tail_amplitudes(int n_tensors, const int32_t *ranks, const int32_t *labels, const float *data,
                                       int n_open, const int32_t *open_labels, int n_steps, const int32_t *tree_in,
                                       int n_sliced_head, const int32_t *sliced_head, int n_sliced_tail,
                                       const int32_t *sliced_tail, tn_form form, const tn_plan_opts *opts,
                                       double *d_amp, double *d_vhead, int *n_cut, tn_stream_t stream) {
    if (n_tensors < 2 || !ranks || !labels || !data || !tree_in || n_steps != n_tensors - 1 || !d_amp ||
        n_open < 0 || (n_open > 0 && !open_labels) || n_sliced_head < 0 || n_sliced_tail < 0 ||
        (n_sliced_head > 0 && !sliced_head) || (n_sliced_tail > 0 && !sliced_tail) || n_sliced_head > 62 ||
        n_sliced_tail > 62)
        return fail(TN_ERR_ARG, "tn_head_tail_amplitudes: bad arguments");
    for (int i = 0; i < n_tensors; i++)
        if (ranks[i] < 0 || ranks[i] > 62) return fail(TN_ERR_ARG, "tn_head_tail_amplitudes: rank out of range");
    const auto labs = parse_labels(n_tensors, ranks, labels);
    std::vector<int64_t> off(n_tensors);
    int64_t acc = 0;
    for (int i = 0; i < n_tensors; i++) {
        off[i] = acc;
        acc += (int64_t)2 << labs[i].size();
    }
    Tree tree(n_steps);
    for (int t = 0; t < n_steps; t++) tree[t] = {tree_in[2 * t], tree_in[2 * t + 1]};
    if (!valid_tree(n_tensors, tree)) return fail(TN_ERR_ARG, "tn_head_tail_amplitudes: malformed tree");
    // the two sides of the root step
    const int n = n_tensors;
    std::vector<int> side[2];
    for (int k = 0; k < 2; k++) {
        std::vector<char> in(n + tree.size(), 0);
        mark_subtree(k == 0 ? tree.back().first : tree.back().second, n, tree, in);
        for (int i = 0; i < n; i++)
            if (in[i]) side[k].push_back(i);
    }
    const std::set<int32_t> open(open_labels, open_labels + n_open);
    int open_side[2] = {0, 0};
    for (int k = 0; k < 2; k++)
        for (int32_t x : labels_of(labs, side[k])) open_side[k] += (int)open.count(x);
    if (open_side[0] && open_side[1])
        return fail(TN_ERR_ARG, "tn_head_tail_amplitudes: open legs on both sides of the root step (no big-head cut)");
    const int h = open_side[0] ? 1 : 0;  // head side: no open leg
    const std::vector<int> &head = side[h], &tail = side[1 - h];
    const int head_root = h == 0 ? tree.back().first : tree.back().second;
    const int tail_root = h == 0 ? tree.back().second : tree.back().first;
    const std::set<int32_t> lh = labels_of(labs, head), lt = labels_of(labs, tail);
    std::vector<int32_t> cut;
    for (int32_t x : lh)
        if (lt.count(x)) cut.push_back(x);
    if (cut.size() > 40) return fail(TN_ERR_ARG, "tn_head_tail_amplitudes: cut of more than 40 bonds");
    const std::set<int32_t> cutset(cut.begin(), cut.end());
    for (int j = 0; j < n_sliced_head; j++)
        if (!lh.count(sliced_head[j]) || cutset.count(sliced_head[j]) || lt.count(sliced_head[j]))
            return fail(TN_ERR_ARG, "tn_head_tail_amplitudes: a head sliced label is not internal to the head");
    for (int j = 0; j < n_sliced_tail; j++)
        if (!lt.count(sliced_tail[j]) || open.count(sliced_tail[j]))
            return fail(TN_ERR_ARG, "tn_head_tail_amplitudes: a tail sliced label is not in the tail or is open");
    if (n_cut) *n_cut = (int)cut.size();
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    // stage 1: the head into v_head over the cut (first cut label = MSB)
    Tree ht;
    sub_tree(head_root, n, tree, head, ht);
    std::vector<int32_t> hr, hl, htree;
    std::vector<float> hv;
    gather_net(labs, data, off, head, hr, hl, hv);
    for (const auto &st : ht) {
        htree.push_back(st.first);
        htree.push_back(st.second);
    }
    PlanGuard A, B;
    int rc = tn_plan_create(&A.p, (int)head.size(), hr.data(), hl.data(), hv.data(), 0, nullptr, (int)cut.size(),
                            cut.data(), n_sliced_head, sliced_head, (int)ht.size(), htree.data(), form, opts);
    if (rc) return rc;
    const int64_t nv = (int64_t)1 << cut.size();
    double *v = d_vhead;
    bool own_v = false;
    if (!v) {
        if (cudaMalloc(&v, sizeof(double) * 2 * nv) != cudaSuccess) return fail(TN_ERR_OOM, "tn_head_tail_amplitudes: v_head");
        own_v = true;
    }
    struct Free {
        double *p;
        bool own;
        ~Free() {
            if (own) cudaFree(p);
        }
    } fv{v, own_v};
    if (cudaMemsetAsync(v, 0, sizeof(double) * 2 * nv, s) != cudaSuccess)
        return fail(TN_ERR_CUDA, "tn_head_tail_amplitudes: memset");
    rc = tn_contract_slices(A.p, 0, (int64_t)1 << n_sliced_head, v, stream);
    if (rc) return rc;

    // stage 2: the tail with v_head as its last leaf, joined at the root
    Tree tt;
    const int tr = sub_tree(tail_root, n, tree, tail, tt);
    const int vleaf = (int)tail.size();
    std::vector<int32_t> tr_ranks, tl, ttree;
    for (int i : tail) {
        tr_ranks.push_back((int32_t)labs[i].size());
        tl.insert(tl.end(), labs[i].begin(), labs[i].end());
    }
    tr_ranks.push_back((int32_t)cut.size());
    tl.insert(tl.end(), cut.begin(), cut.end());
    for (auto &st : tt) {  // shift step ids past the extra leaf
        const int a = st.first >= vleaf ? st.first + 1 : st.first;
        const int b = st.second >= vleaf ? st.second + 1 : st.second;
        ttree.push_back(a);
        ttree.push_back(b);
    }
    ttree.push_back(tr >= vleaf ? tr + 1 : tr);
    ttree.push_back(vleaf);
    // leaves: the tail's from the caller's host data, v_head from the device
    rc = tn_plan_create(&B.p, vleaf + 1, tr_ranks.data(), tl.data(), nullptr, 0, nullptr, n_open, open_labels,
                        n_sliced_tail, sliced_tail, (int)ttree.size() / 2, ttree.data(), form, opts);
    if (rc) return rc;
    for (int k = 0; k < vleaf && rc == 0; k++) rc = plan_load_leaf_host(B.p, k, data + off[tail[k]], s);
    if (rc == 0) rc = plan_load_leaf_c128(B.p, vleaf, v, s);
    if (rc) return rc;
    if (cudaMemsetAsync(d_amp, 0, sizeof(double) * ((size_t)2 << n_open), s) != cudaSuccess)
        return fail(TN_ERR_CUDA, "tn_head_tail_amplitudes: memset");
    rc = tn_contract_slices(B.p, 0, (int64_t)1 << n_sliced_tail, d_amp, stream);
    if (rc) return rc;
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(TN_ERR_CUDA, "tn_head_tail_amplitudes: stream");
    return TN_OK;
}

extern "C" int tn_find_order_head_tail(int n_tensors, const int32_t *ranks, const int32_t *labels, int n_open,
                                       const int32_t *open_labels, int tail_max, const tn_search_opts *opts,
                                       int32_t *out_tree, int max_sliced, int32_t *out_sliced_head,
                                       int *out_n_sliced_head, double *stats) {
    if (n_tensors < 2 || !ranks || !labels || n_open < 0 || (n_open > 0 && !open_labels) || tail_max < 0)
        return fail(TN_ERR_ARG, "tn_find_order_head_tail: bad arguments");
    for (int i = 0; i < n_tensors; i++)
        if (ranks[i] < 0 || ranks[i] > 62) return fail(TN_ERR_ARG, "tn_find_order_head_tail: rank out of range");
    const int n = n_tensors;
    const auto labs = parse_labels(n, ranks, labels);
    if (const char *bad = check_network(labs, std::vector<int32_t>(open_labels, open_labels + n_open)))
        return fail(TN_ERR_ARG, std::string("tn_find_order_head_tail: ") + bad);
    const std::set<int32_t> open(open_labels, open_labels + n_open);
    std::unordered_map<int32_t, std::vector<int>> holders;
    for (int i = 0; i < n; i++)
        for (int32_t x : labs[i]) holders[x].push_back(i);
    // the tail starts with every tensor holding an open leg
    std::vector<char> in_tail(n, 0);
    std::vector<int> order;
    for (int i = 0; i < n; i++)
        for (int32_t x : labs[i])
            if (open.count(x) && !in_tail[i]) {
                in_tail[i] = 1;
                order.push_back(i);
            }
    if (order.empty()) return fail(TN_ERR_ARG, "tn_find_order_head_tail: no open legs");
    if ((int)order.size() >= n) return fail(TN_ERR_ARG, "tn_find_order_head_tail: every tensor holds an open leg");
    // cut = bonds with exactly one end in the tail
    auto cut_size = [&](const std::vector<char> &t) {
        int c = 0;
        for (const auto &kv : holders)
            if (kv.second.size() == 2 && t[kv.second[0]] != t[kv.second[1]]) c++;
        return c;
    };
    const int limit = tail_max > 0 ? std::min(tail_max, n - 1) : n / 2;
    int best_cut = cut_size(in_tail);
    size_t best_len = order.size();
    while ((int)order.size() < limit) {
        int pick = -1, pick_cut = 1 << 30;
        for (int i = 0; i < n; i++) {
            if (in_tail[i]) continue;
            bool adj = false;
            for (int32_t x : labs[i])
                for (int j : holders[x])
                    if (in_tail[j]) adj = true;
            if (!adj) continue;
            in_tail[i] = 1;
            const int c = cut_size(in_tail);
            in_tail[i] = 0;
            if (c < pick_cut) {
                pick_cut = c;
                pick = i;
            }
        }
        if (pick < 0) break;
        in_tail[pick] = 1;
        order.push_back(pick);
        if (pick_cut < best_cut) {
            best_cut = pick_cut;
            best_len = order.size();
        }
    }
    std::fill(in_tail.begin(), in_tail.end(), 0);
    for (size_t k = 0; k < best_len; k++) in_tail[order[k]] = 1;
    if (opts && opts->method >= 1) {
        // the partition step of the first cut: Fiduccia-Mattheyses passes
        // from the grown tail, the open-leg tensors held in the tail and
        // the tail kept between them and the size limit
        std::vector<std::vector<int>> nb(n);
        std::vector<char> fixed(n, 0);
        std::vector<int> side(n);
        for (int i = 0; i < n; i++) {
            side[i] = in_tail[i] ? 0 : 1;
            for (int32_t x : labs[i]) {
                if (open.count(x)) fixed[i] = 1;
                const auto &h = holders[x];
                if (h.size() == 2 && h[0] != h[1]) nb[i].push_back(h[0] == i ? h[1] : h[0]);
            }
        }
        int n_fixed = 0;
        for (char f : fixed) n_fixed += f;
        fm_refine(nb, side, &fixed, n_fixed, std::max(limit, (int)best_len), 16);
        for (int i = 0; i < n; i++) in_tail[i] = side[i] == 0;
    }
    std::vector<int> head, tail;
    for (int i = 0; i < n; i++) (in_tail[i] ? tail : head).push_back(i);
    std::vector<int32_t> cut;
    for (const auto &kv : holders)
        if (kv.second.size() == 2 && in_tail[kv.second[0]] != in_tail[kv.second[1]]) cut.push_back(kv.first);
    std::sort(cut.begin(), cut.end());
    // each side's order: the head into the cut (sliced to the options' cap
    // or count), the tail into cut + open legs (not sliced)
    tn_search_opts o = opts ? *opts : default_search_opts();
    std::vector<std::vector<int32_t>> hl, tl;
    for (int i : head) hl.push_back(labs[i]);
    for (int i : tail) tl.push_back(labs[i]);
    SearchResult hr, trr;
    int rc = search_ranked(hl, cut, o, hr);
    if (rc) return rc;
    tn_search_opts ot = o;
    ot.n_sliced = 0;
    ot.log2_cap = -1;
    ot.cost_model = nullptr;
    std::vector<int32_t> topen(cut);
    topen.insert(topen.end(), open_labels, open_labels + n_open);
    rc = search_order(tl, topen, ot, trr);
    if (rc) return rc;
    if ((int)hr.sliced.size() > max_sliced) return fail(TN_ERR_ARG, "tn_find_order_head_tail: max_sliced too small");
    // join: head steps, tail steps, root step, in the original leaf ids
    std::vector<int> idh(head.size() + hr.tree.size()), idt(tail.size() + trr.tree.size());
    for (size_t i = 0; i < head.size(); i++) idh[i] = head[i];
    for (size_t i = 0; i < tail.size(); i++) idt[i] = tail[i];
    int next = n;
    Tree full;
    for (size_t t = 0; t < hr.tree.size(); t++) {
        full.push_back({idh[hr.tree[t].first], idh[hr.tree[t].second]});
        idh[head.size() + t] = next++;
    }
    for (size_t t = 0; t < trr.tree.size(); t++) {
        full.push_back({idt[trr.tree[t].first], idt[trr.tree[t].second]});
        idt[tail.size() + t] = next++;
    }
    full.push_back({idh.back(), idt.back()});
    if (out_tree)
        for (size_t t = 0; t < full.size(); t++) {
            out_tree[2 * t] = full[t].first;
            out_tree[2 * t + 1] = full[t].second;
        }
    if (out_sliced_head)
        for (size_t j = 0; j < hr.sliced.size(); j++) out_sliced_head[j] = hr.sliced[j];
    if (out_n_sliced_head) *out_n_sliced_head = (int)hr.sliced.size();
    if (stats) {
        // head per slice, head width, head slices, tail, tail width, cut,
        // total = head over all slices + tail + the root inner product
        const double root = std::exp2((double)cut.size() + n_open);
        stats[0] = hr.log2_slice;
        stats[1] = hr.log2_width;
        stats[2] = (double)hr.sliced.size();
        stats[3] = trr.log2_total;
        stats[4] = trr.log2_width;
        stats[5] = (double)cut.size();
        stats[6] = std::log2(std::exp2(hr.log2_total) + std::exp2(trr.log2_total) + root);
    }
    return TN_OK;
}

namespace {

// A candidate first cut for tn_choose_open_qubits: the tail's open qubits,
// its cut and its tensors (in the all-open network).
struct OpenCand {
    int cut;
    std::vector<int32_t> qubits;
    std::vector<char> in;
};

// Every connected tail holding exactly n_open qubit ends that the growths
// reach, sorted by cut (stable: growth order breaks ties).  n_tensors gets the
// all-open network's tensor count.
int open_candidates(const tn_circuit *circuit, int n_open, std::vector<OpenCand> &cands, int &n_tensors) {
    using Cand = OpenCand;
    cands.clear();
    const int nq = circuit->n_qubits;
    std::vector<int32_t> all(nq);
    for (int q = 0; q < nq; q++) all[q] = q;
    Network net;
    int rc = build_circuit_network(circuit, nullptr, nq, all.data(), net);
    if (rc) return rc;
    const int n = (int)net.tensors.size();
    std::unordered_map<int32_t, std::vector<int>> holders;
    for (int i = 0; i < n; i++)
        for (int32_t x : net.tensors[i].labels) holders[x].push_back(i);
    // the tensor holding each qubit's last wire segment (an open leg here)
    std::vector<std::vector<int>> qubits_of(n);
    for (int q = 0; q < nq; q++) qubits_of[holders[net.open[q]][0]].push_back(q);
    // bonds between tensors (one per shared label)
    std::vector<std::vector<int>> nb(n);
    for (const auto &kv : holders)
        if (kv.second.size() == 2 && kv.second[0] != kv.second[1]) {
            nb[kv.second[0]].push_back(kv.second[1]);
            nb[kv.second[1]].push_back(kv.second[0]);
        }
    // candidate tails: (cut, open qubits) -> the tail that reached it first
    auto record = [&](int cut, const std::vector<char> &in) {
        std::vector<int32_t> qs;
        for (int q = 0; q < nq; q++)
            if (in[holders[net.open[q]][0]]) qs.push_back(q);
        for (auto &c : cands)
            if (c.qubits == qs) {
                if (cut < c.cut) { c.cut = cut; c.in = in; }
                return;
            }
        cands.push_back({cut, qs, in});
    };
    std::vector<char> in(n);
    std::vector<int> conn(n);
    // equal cuts are frequent and the order they are taken in steers the
    // growth: every seed tensor grows kRuns times, the first with ties to
    // the lower index, the others to a random one (SplitMix64, fixed seed)
    constexpr int kRuns = 16;
    uint64_t rs = 0x2103030740ull;
    auto next_u64 = [&rs]() {
        rs += 0x9E3779B97F4A7C15ull;
        uint64_t z = rs;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    for (int run = 0; run < n * kRuns; run++) {
        const int seed = run / kRuns;
        const bool random_ties = run % kRuns != 0;
        if (qubits_of[seed].empty() || (int)qubits_of[seed].size() > n_open) continue;
        std::fill(in.begin(), in.end(), 0);
        std::fill(conn.begin(), conn.end(), 0);
        int v = seed, cut = 0, n_in = 0, n_q = 0;
        for (;;) {
            // add v to the tail
            in[v] = 1;
            n_in++;
            n_q += (int)qubits_of[v].size();
            cut += (int)nb[v].size() - 2 * conn[v];
            for (int u : nb[v]) conn[u]++;
            if (n_q == n_open) record(cut, in);
            if (n_in >= n / 2) break;
            // the neighbour leaving the smallest cut without exceeding n_open
            // open qubits (ties: more open qubits, then the lower index or a
            // random one); the tail stays connected, which keeps the open
            // qubits together (a tail of scattered last-layer tensors reaches
            // the same cut for any open set)
            int pick = -1, pick_cut = 0, pick_q = 0, ties = 0;
            for (int u = 0; u < n; u++) {
                if (in[u] || conn[u] == 0) continue;
                const int uq = (int)qubits_of[u].size();
                if (n_q + uq > n_open) continue;
                const int c = cut + (int)nb[u].size() - 2 * conn[u];
                if (pick < 0 || c < pick_cut || (c == pick_cut && uq > pick_q)) {
                    pick = u;
                    pick_cut = c;
                    pick_q = uq;
                    ties = 1;
                } else if (random_ties && c == pick_cut && uq == pick_q && next_u64() % (uint64_t)(++ties) == 0) {
                    pick = u;
                }
            }
            if (pick < 0) break;
            v = pick;
        }
    }
    if (cands.empty()) return fail(TN_ERR_ARG, "no connected tail holds exactly n_open qubit ends");
    std::stable_sort(cands.begin(), cands.end(), [](const Cand &a, const Cand &b) { return a.cut < b.cut; });
    n_tensors = n;
    return TN_OK;
}

}  // namespace

extern "C" int tn_choose_open_qubits(const tn_circuit *circuit, int n_open, const tn_search_opts *opts,
                                     int32_t *out_open_qubits, int32_t *out_tail, int *out_n_tail, int *out_cut,
                                     double *out_log2_cost) {
    if (!circuit || !out_open_qubits || circuit->n_qubits < 2 || n_open < 1 || n_open >= circuit->n_qubits)
        return fail(TN_ERR_ARG, "tn_choose_open_qubits: need a circuit and 1 <= n_open < n_qubits");
    const int nq = circuit->n_qubits;
    std::vector<OpenCand> cands;
    int n = 0;
    int rc = open_candidates(circuit, n_open, cands, n);
    if (rc) return fail(rc, std::string("tn_choose_open_qubits: ") + tn_last_error());
    // with search options: of the kPick smallest cuts, the open set whose
    // network the order search contracts most cheaply (the paper tries
    // first cuts until the contraction's complexity is acceptable)
    constexpr int kPick = 8;
    int best = 0;
    bool priced = false;      // a candidate's cost has been taken
    double best_cost = -1.0;  // reported as -1 without search options
    if (opts) {
        const int m = std::min<int>(kPick, (int)cands.size());
        for (int i = 0; i < m; i++) {
            Network sub;
            std::vector<uint8_t> zeros(nq, 0);
            rc = build_circuit_network(circuit, zeros.data(), n_open, cands[i].qubits.data(), sub);
            if (rc) return rc;
            std::vector<std::vector<int32_t>> labs;
            for (const auto &t : sub.tensors) labs.push_back(t.labels);
            SearchResult r;
            rc = search_order(labs, sub.open, *opts, r);
            if (rc) return rc;
            // the search's own measure: total MACs, or with the roofline
            // objective the compiled plan's roofline time
            double cost = r.log2_total;
            if (opts->objective >= 1) {
                const tn_form f = (opts->rank_form >= TN_FP32 && opts->rank_form <= TN_FP16X3) ? (tn_form)opts->rank_form
                                                                                               : TN_FP32;
                const double ms = tree_roofline_ms(labs, sub.open, r.tree, r.sliced, f, opts->rank_batch_log2,
                                                   kNominalArenaBytes, opts->objective == 2);
                cost = ms > 0 ? std::log2(ms) : INFINITY;
            }
            if (!priced || cost < best_cost) {
                priced = true;
                best_cost = cost;
                best = i;
            }
        }
    }
    const OpenCand &c = cands[best];
    for (int k = 0; k < n_open; k++) out_open_qubits[k] = c.qubits[k];
    int nt = 0;
    for (int i = 0; i < n; i++)
        if (c.in[i]) {
            if (out_tail) out_tail[nt] = i;
            nt++;
        }
    if (out_n_tail) *out_n_tail = nt;
    if (out_cut) *out_cut = c.cut;
    if (out_log2_cost) *out_log2_cost = best_cost;
    return TN_OK;
}

extern "C" int tn_open_qubit_candidates(const tn_circuit *circuit, int n_open, int max_out, int32_t *out_qubits,
                                        int *out_cuts, int *out_n) {
    if (!circuit || !out_n || circuit->n_qubits < 2 || n_open < 1 || n_open >= circuit->n_qubits || max_out < 0 ||
        (max_out > 0 && (!out_qubits || !out_cuts)))
        return fail(TN_ERR_ARG, "tn_open_qubit_candidates: need a circuit, 1 <= n_open < n_qubits and output room");
    std::vector<OpenCand> cands;
    int n = 0;
    int rc = open_candidates(circuit, n_open, cands, n);
    if (rc) return fail(rc, std::string("tn_open_qubit_candidates: ") + tn_last_error());
    const int m = std::min<int>(max_out, (int)cands.size());
    for (int i = 0; i < m; i++) {
        for (int k = 0; k < n_open; k++) out_qubits[(size_t)i * n_open + k] = cands[i].qubits[k];
        out_cuts[i] = cands[i].cut;
    }
    *out_n = (int)cands.size();
    return TN_OK;
}

extern "C" int tn_slice_stage2(int n_tensors, const int32_t *ranks, const int32_t *labels, int n_open,
                               const int32_t *open_labels, int n_steps, const int32_t *tree_in, int log2_cap,
                               int max_sliced, int32_t *out_sliced_tail, int *out_n_sliced, double *stats) {
    if (n_tensors < 2 || !ranks || !labels || n_open < 1 || !open_labels || n_steps != n_tensors - 1 || !tree_in ||
        log2_cap < 0)
        return fail(TN_ERR_ARG, "tn_slice_stage2: bad arguments");
    for (int i = 0; i < n_tensors; i++)
        if (ranks[i] < 0 || ranks[i] > 62) return fail(TN_ERR_ARG, "tn_slice_stage2: rank out of range");
    const int n = n_tensors;
    const auto labs = parse_labels(n, ranks, labels);
    Tree tree(n_steps);
    for (int t = 0; t < n_steps; t++) tree[t] = {tree_in[2 * t], tree_in[2 * t + 1]};
    if (!valid_tree(n, tree)) return fail(TN_ERR_ARG, "tn_slice_stage2: malformed tree");
    // head and tail: the two sides of the root step, the tail holding the open legs
    const std::set<int32_t> open(open_labels, open_labels + n_open);
    std::vector<int> side[2];
    int open_side[2] = {0, 0};
    for (int k = 0; k < 2; k++) {
        std::vector<char> in(n + tree.size(), 0);
        mark_subtree(k == 0 ? tree.back().first : tree.back().second, n, tree, in);
        for (int i = 0; i < n; i++)
            if (in[i]) side[k].push_back(i);
        for (int32_t x : labels_of(labs, side[k])) open_side[k] += (int)open.count(x);
    }
    if (open_side[0] && open_side[1])
        return fail(TN_ERR_ARG, "tn_slice_stage2: open legs on both sides of the root step (no big-head cut)");
    const int h = open_side[0] ? 1 : 0;
    const std::vector<int> &head = side[h], &tail = side[1 - h];
    const int tail_root = h == 0 ? tree.back().second : tree.back().first;
    const std::set<int32_t> lh = labels_of(labs, head), lt = labels_of(labs, tail);
    std::vector<int32_t> cut;
    for (int32_t x : lh)
        if (lt.count(x)) cut.push_back(x);
    // stage 2 as tn_head_tail_amplitudes builds it: the tail's leaves, then
    // v_head over the cut (increasing labels) as the last leaf, joined at the root
    Tree tt;
    const int tr = sub_tree(tail_root, n, tree, tail, tt);
    const int vleaf = (int)tail.size();
    std::vector<int32_t> r2, l2, t2;
    for (int i : tail) {
        r2.push_back((int32_t)labs[i].size());
        l2.insert(l2.end(), labs[i].begin(), labs[i].end());
    }
    r2.push_back((int32_t)cut.size());
    l2.insert(l2.end(), cut.begin(), cut.end());
    for (const auto &st : tt) {
        t2.push_back(st.first >= vleaf ? st.first + 1 : st.first);
        t2.push_back(st.second >= vleaf ? st.second + 1 : st.second);
    }
    t2.push_back(tr >= vleaf ? tr + 1 : tr);
    t2.push_back(vleaf);
    return tn_slice_tree(vleaf + 1, r2.data(), l2.data(), n_open, open_labels, (int)t2.size() / 2, t2.data(), log2_cap,
                         -1, max_sliced, out_sliced_tail, out_n_sliced, stats);
}
