// Host-side contraction-order search and slicing.
//
// Cost model (Fig. 3): contracting a pair that shares n_AB labels, with n_A and
// n_B outer labels, costs 2^{n_A + n_B + n_AB} complex multiply-adds; its
// space cost is the size of the result.  A tree's cost is the sum over its
// steps; its width is its largest tensor.
//
// Order: randomised greedy.  Each trial repeatedly merges the connected pair
// with the smallest key, key = slog2(2^{|out|} - alpha (2^{|A|} + 2^{|B|}))
// minus temperature x Gumbel noise (trial 0 is the plain greedy alpha = 1,
// no noise).  Or (method 1, or every other trial with method 2) hierarchical
// bipartition as in the paper's appendix: min-cut splits down to parts of a
// few dozen tensors, greedy inside a part (bipartition_trial below).
//
// Slicing ("Dynamic slicing" paragraph): labels are sliced one at a time
// under two greedy rules (lower the widest intermediate first; or, among the
// widest intermediates' labels, the smallest total cost 2^{n_e} x sum_steps
// 2^{|step labels \ sliced|}); the cheaper result that meets the cap is kept.
//
// Subtree reconfiguration: the best few trees are then improved locally.
// Every internal node's subtree, cut at up to 11 frontier tensors, is
// re-ordered optimally by dynamic programming over frontier subsets under
// the current slice set; slicing is redone and the cycle repeats.  On the
// 53-qubit 20-cycle circuit this lowers the sliced total from 2^73 to 2^61
// (the paper's own instance: about 2^62).
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <queue>
#include <thread>
#include <unordered_map>

#include "tn_internal.h"

namespace tn {

namespace {

struct Rng {  // SplitMix64
    uint64_t s;
    explicit Rng(uint64_t seed) : s(seed) {}
    uint64_t next() {
        s += 0x9E3779B97F4A7C15ull;
        uint64_t z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

// Dense label sets over remapped label ids.
struct Sets {
    int W = 0;
    std::vector<uint64_t> bits;
    void init(int n_sets, int n_labels) {
        W = (n_labels + 63) / 64;
        if (W == 0) W = 1;
        bits.assign((size_t)n_sets * W, 0);
    }
    uint64_t *at(int i) { return bits.data() + (size_t)i * W; }
    const uint64_t *at(int i) const { return bits.data() + (size_t)i * W; }
};

inline int popc(const uint64_t *a, int W) {
    int c = 0;
    for (int i = 0; i < W; i++) c += __builtin_popcountll(a[i]);
    return c;
}

struct Problem {
    int n = 0;          // leaves
    int L = 0;          // labels (remapped)
    Sets leaf;          // leaf label sets
    std::vector<uint64_t> open;  // open mask
    std::vector<int32_t> id2label;
    std::vector<std::vector<int>> leaf_labels;  // remapped ids per leaf
};

// Builds the search's view of a network; returns nullptr, or what is wrong
// with it (a label is a bond between at most two tensors, each holding it
// once; every kept label is held by some tensor).
const char *make_problem(const std::vector<std::vector<int32_t>> &labels, const std::vector<int32_t> &open,
                         Problem &p) {
    std::unordered_map<int32_t, int> remap;
    std::vector<int> holders;
    for (auto &l : labels) {
        for (int32_t x : l) {
            auto it = remap.find(x);
            if (it == remap.end()) {
                it = remap.emplace(x, (int)remap.size()).first;
                p.id2label.push_back(x);
                holders.push_back(0);
            }
            if (++holders[it->second] > 2) return "label held by more than two tensors";
        }
        for (size_t a = 0; a < l.size(); a++)
            for (size_t b = a + 1; b < l.size(); b++)
                if (l[a] == l[b]) return "label repeated within a tensor";
    }
    for (int32_t x : open)
        if (!remap.count(x)) return "open label held by no tensor";
    p.n = (int)labels.size();
    p.L = (int)remap.size();
    p.leaf.init(p.n, p.L);
    p.open.assign(p.leaf.W, 0);
    p.leaf_labels.resize(p.n);
    for (int i = 0; i < p.n; i++)
        for (int32_t x : labels[i]) {
            int id = remap[x];
            p.leaf.at(i)[id >> 6] |= 1ull << (id & 63);
            p.leaf_labels[i].push_back(id);
        }
    for (int32_t x : open) {
        int id = remap[x];
        p.open[id >> 6] |= 1ull << (id & 63);
    }
    return nullptr;
}

// All node label sets of a tree (leaves, then one per step) and step unions.
struct TreeSets {
    Sets node;   // 2n-1 sets
    Sets uni;    // n-1 step unions (labels of A u B)
};

bool tree_sets(const Problem &p, const Tree &tree, TreeSets &ts) {
    const int n = p.n, W = p.leaf.W;
    if ((int)tree.size() != std::max(n - 1, 0)) return false;
    ts.node.init(2 * n - 1 > 0 ? 2 * n - 1 : 1, p.L);
    ts.uni.init(n - 1 > 0 ? n - 1 : 1, p.L);
    std::memcpy(ts.node.at(0), p.leaf.at(0), sizeof(uint64_t) * W * n);
    std::vector<char> used(2 * n, 0);
    for (int t = 0; t < n - 1; t++) {
        int a = tree[t].first, b = tree[t].second;
        if (a < 0 || b < 0 || a >= n + t || b >= n + t || a == b || used[a] || used[b]) return false;
        used[a] = used[b] = 1;
        const uint64_t *sa = ts.node.at(a), *sb = ts.node.at(b);
        uint64_t *so = ts.node.at(n + t), *su = ts.uni.at(t);
        for (int w = 0; w < W; w++) {
            su[w] = sa[w] | sb[w];
            so[w] = su[w] & ~(sa[w] & sb[w] & ~p.open[w]);
        }
    }
    return true;
}

struct SliceEval {
    std::vector<int> sliced;  // remapped ids
    double log2_slice_cost = 0, log2_width = 0, log2_total = 0;
};

double log2_sum_pow2(const std::vector<double> &e) {  // log2(sum 2^e)
    if (e.empty()) return -INFINITY;
    double m = *std::max_element(e.begin(), e.end());
    double s = 0;
    for (double x : e) s += std::exp2(x - m);
    return m + std::log2(s);
}

// Greedy slicing.  n_sliced >= 0: exactly that many; else slice until width <= cap.
// Greedy slicing of one tree until the widest intermediate fits 2^log2_cap
// (or n_sliced labels are sliced).  rule 0: the label that lowers the widest
// intermediate most, then the smallest total cost; rule 1: among the labels
// of the widest intermediates, the one in the most expensive steps (the
// smallest total cost after slicing), then the width.
void slice_tree(const Problem &p, const TreeSets &ts, int n_nodes, int n_steps, int log2_cap,
                int n_sliced, int rule, SliceEval &ev) {
    const int W = p.leaf.W;
    std::vector<uint64_t> smask(W, 0);
    std::vector<int> wv(n_nodes), wu(n_steps);
    auto recount = [&]() {
        for (int v = 0; v < n_nodes; v++) {
            const uint64_t *s = ts.node.at(v);
            int c = 0;
            for (int w = 0; w < W; w++) c += __builtin_popcountll(s[w] & ~smask[w]);
            wv[v] = c;
        }
        for (int t = 0; t < n_steps; t++) {
            const uint64_t *s = ts.uni.at(t);
            int c = 0;
            for (int w = 0; w < W; w++) c += __builtin_popcountll(s[w] & ~smask[w]);
            wu[t] = c;
        }
    };
    recount();
    ev.sliced.clear();
    for (int iter = 0; iter < p.L; iter++) {
        int wmax = n_nodes ? *std::max_element(wv.begin(), wv.end()) : 0;
        if (n_sliced >= 0) {
            if ((int)ev.sliced.size() >= n_sliced) break;
        } else if (log2_cap < 0 || wmax <= log2_cap) {
            break;
        }
        // per-label: reduction of the step-cost sum and the new width
        std::vector<double> drop(p.L, 0.0);
        double base = 0;
        double m = 0;
        for (int t = 0; t < n_steps; t++) m = std::max(m, (double)wu[t]);
        for (int t = 0; t < n_steps; t++) {
            double c = std::exp2(wu[t] - m);
            base += c;
            const uint64_t *s = ts.uni.at(t);
            for (int w = 0; w < W; w++) {
                uint64_t x = s[w] & ~smask[w] & ~p.open[w];
                while (x) {
                    int b = __builtin_ctzll(x);
                    x &= x - 1;
                    drop[w * 64 + b] += 0.5 * c;
                }
            }
        }
        // slicing label l lowers the widest intermediate only when every
        // widest node holds l (to wmax - 1: the others are narrower
        // already), so the new width follows from how many widest nodes
        // hold l
        std::vector<int> in_widest_cnt(p.L, 0);
        int n_widest = 0;
        for (int v = 0; v < n_nodes; v++) {
            if (wv[v] != wmax) continue;
            n_widest++;
            const uint64_t *sv = ts.node.at(v);
            for (int w = 0; w < W; w++) {
                uint64_t x = sv[w];
                while (x) {
                    in_widest_cnt[w * 64 + __builtin_ctzll(x)]++;
                    x &= x - 1;
                }
            }
        }
        int best = -1;
        int best_w = 0;
        double best_c = 0;
        for (int l = 0; l < p.L; l++) {
            if ((p.open[l >> 6] >> (l & 63)) & 1) continue;
            if ((smask[l >> 6] >> (l & 63)) & 1) continue;
            if (drop[l] <= 0) continue;  // label in no step
            const bool in_widest = in_widest_cnt[l] > 0;
            const int nw = (n_widest > 0 && in_widest_cnt[l] == n_widest) ? wmax - 1 : wmax;
            double c = base - drop[l];
            if (rule == 1) {
                if (!in_widest) continue;
                if (best < 0 || c < best_c || (c == best_c && nw < best_w)) {
                    best = l;
                    best_w = nw;
                    best_c = c;
                }
                continue;
            }
            if (best < 0 || nw < best_w || (nw == best_w && c < best_c)) {
                best = l;
                best_w = nw;
                best_c = c;
            }
        }
        if (best < 0) break;
        smask[best >> 6] |= 1ull << (best & 63);
        ev.sliced.push_back(best);
        recount();
    }
    std::vector<double> e(wu.begin(), wu.end());
    ev.log2_slice_cost = n_steps ? log2_sum_pow2(e) : 0.0;
    ev.log2_width = n_nodes ? *std::max_element(wv.begin(), wv.end()) : 0;
    ev.log2_total = ev.log2_slice_cost + (double)ev.sliced.size();
}

inline double slog2(double x) { return x >= 0 ? std::log2(1.0 + x) : -std::log2(1.0 - x); }

// One randomised greedy trial.
Tree greedy_trial(const Problem &p, uint64_t seed, bool plain) {
    const int n = p.n, W = p.leaf.W;
    Rng rng(seed);
    double alpha = plain ? 1.0 : rng.uniform();
    double temp = plain ? 0.0 : std::exp2(-7.0 + 7.0 * rng.uniform());
    Sets s;
    s.init(2 * n, p.L);
    std::memcpy(s.at(0), p.leaf.at(0), sizeof(uint64_t) * W * n);
    std::vector<int> size(2 * n, 0);
    for (int i = 0; i < n; i++) size[i] = popc(s.at(i), W);
    std::vector<std::array<int, 2>> holders(p.L, {-1, -1});
    for (int i = 0; i < n; i++)
        for (int id : p.leaf_labels[i]) {
            auto &h = holders[id];
            if (h[0] < 0) h[0] = i; else h[1] = i;
        }
    std::vector<char> alive(2 * n, 0);
    for (int i = 0; i < n; i++) alive[i] = 1;
    struct Item { double key; int a, b; };
    auto cmp = [](const Item &x, const Item &y) {
        if (x.key != y.key) return x.key > y.key;
        if (x.a != y.a) return x.a > y.a;
        return x.b > y.b;
    };
    std::priority_queue<Item, std::vector<Item>, decltype(cmp)> pq(cmp);
    std::vector<uint64_t> tmp(W);
    auto out_size = [&](int a, int b) {
        const uint64_t *sa = s.at(a), *sb = s.at(b);
        int c = 0;
        for (int w = 0; w < W; w++) c += __builtin_popcountll((sa[w] | sb[w]) & ~(sa[w] & sb[w] & ~p.open[w]));
        return c;
    };
    auto push = [&](int a, int b) {
        if (a > b) std::swap(a, b);
        int o = out_size(a, b);
        double cost = std::exp2((double)o) - alpha * (std::exp2((double)size[a]) + std::exp2((double)size[b]));
        double key = slog2(cost);
        if (temp > 0) {
            double u = rng.uniform();
            if (u < 1e-300) u = 1e-300;
            key -= temp * (-std::log(-std::log(u)));
        }
        pq.push({key, a, b});
    };
    for (int l = 0; l < p.L; l++)
        if (holders[l][0] >= 0 && holders[l][1] >= 0) push(holders[l][0], holders[l][1]);
    Tree tree;
    int nxt = n, n_alive = n;
    while (n_alive > 1) {
        int a = -1, b = -1;
        while (!pq.empty()) {
            Item it = pq.top();
            pq.pop();
            if (alive[it.a] && alive[it.b]) {
                a = it.a;
                b = it.b;
                break;
            }
        }
        if (a < 0) {  // disconnected: join the two smallest alive nodes
            int s1 = -1, s2 = -1;
            for (int i = 0; i < nxt; i++) {
                if (!alive[i]) continue;
                if (s1 < 0 || size[i] < size[s1]) { s2 = s1; s1 = i; }
                else if (s2 < 0 || size[i] < size[s2]) s2 = i;
            }
            a = std::min(s1, s2);
            b = std::max(s1, s2);
        }
        uint64_t *sa = s.at(a), *sb = s.at(b), *so = s.at(nxt);
        for (int w = 0; w < W; w++) so[w] = (sa[w] | sb[w]) & ~(sa[w] & sb[w] & ~p.open[w]);
        size[nxt] = popc(so, W);
        alive[a] = alive[b] = 0;
        alive[nxt] = 1;
        tree.push_back({a, b});
        // holders update and new candidate pairs
        for (int w = 0; w < W; w++) {
            uint64_t x = sa[w] | sb[w];
            while (x) {
                int l = w * 64 + __builtin_ctzll(x);
                x &= x - 1;
                auto &h = holders[l];
                bool kept = (so[l >> 6] >> (l & 63)) & 1;
                for (int k = 0; k < 2; k++)
                    if (h[k] == a || h[k] == b) h[k] = kept ? nxt : -1;
                if (h[0] == nxt && h[1] == nxt) h[1] = -1;  // open label held by both operands (cannot happen)
            }
        }
        for (int w = 0; w < W; w++) {
            uint64_t x = so[w];
            while (x) {
                int l = w * 64 + __builtin_ctzll(x);
                x &= x - 1;
                auto &h = holders[l];
                int other = h[0] == nxt ? h[1] : h[0];
                if (other >= 0 && other != nxt && alive[other]) push(nxt, other);
            }
        }
        nxt++;
        n_alive--;
    }
    return tree;
}

}  // namespace

// Fiduccia-Mattheyses refinement of a two-way split (nb: one entry per
// shared bond, side: 0 or 1 per vertex).  Each pass moves, one at a time,
// the unlocked vertex whose move lowers the cut most while the count of
// side-0 vertices stays in [lo, hi], locks it, and keeps the best prefix of
// the pass (ties: the more even split); vertices marked in `fixed` never
// move.  Passes repeat while the cut drops, at most max_passes.  Returns
// the cut.
int fm_refine(const std::vector<std::vector<int>> &nb, std::vector<int> &side, const std::vector<char> *fixed, int lo,
              int hi, int max_passes) {
    const int m = (int)side.size();
    std::vector<int> gain(m);
    std::vector<char> locked(m);
    int cut = 0, n0 = 0;
    for (int i = 0; i < m; i++) {
        gain[i] = 0;
        for (int j : nb[i]) gain[i] += side[j] != side[i] ? 1 : -1;
        if (side[i] == 0) {
            n0++;
            for (int j : nb[i]) cut += side[j] == 1;
        }
    }
    for (int pass = 0; pass < max_passes; pass++) {
        for (int i = 0; i < m; i++) locked[i] = fixed ? (*fixed)[i] : 0;
        std::vector<int> moves;
        int cur = cut, c0 = n0, pbest = cut, pbest_len = 0;
        int pbest_imb = std::abs(2 * n0 - m);
        for (int s = 0; s < m; s++) {
            int bi = -1;
            for (int i = 0; i < m; i++) {
                if (locked[i]) continue;
                const int nc0 = c0 + (side[i] == 0 ? -1 : 1);
                if (nc0 < lo || nc0 > hi) continue;
                if (bi < 0 || gain[i] > gain[bi]) bi = i;
            }
            if (bi < 0) break;
            cur -= gain[bi];
            c0 += side[bi] == 0 ? -1 : 1;
            for (int j : nb[bi]) gain[j] += side[j] == side[bi] ? 2 : -2;
            gain[bi] = -gain[bi];
            side[bi] ^= 1;
            locked[bi] = 1;
            moves.push_back(bi);
            const int imb = std::abs(2 * c0 - m);
            if (cur < pbest || (cur == pbest && imb < pbest_imb)) {
                pbest = cur;
                pbest_imb = imb;
                pbest_len = (int)moves.size();
            }
        }
        // undo the moves past the best prefix
        for (int s = (int)moves.size() - 1; s >= pbest_len; s--) {
            const int i = moves[s];
            c0 += side[i] == 0 ? -1 : 1;
            for (int j : nb[i]) gain[j] += side[j] == side[i] ? 2 : -2;
            gain[i] = -gain[i];
            side[i] ^= 1;
        }
        const bool better = pbest < cut;
        cut = pbest;
        n0 = c0;
        if (!better) break;
    }
    return cut;
}

namespace {

// Hierarchical bipartition (appendix, "Finding contraction order using
// hierarchical partitioning"; Fig. 3 gives the cost of each split): the
// network is split in two parts sharing few bonds, each part again, until a
// part holds at most leaf_max tensors; such a part is contracted in greedy
// order, and the parts are joined in the order of the splits (the split at
// the top is the tree's last step).  One split: a region grown from a random
// tensor, always taking the outside tensor with the most bonds into the
// region, to a random size inside the balance window; then fm_refine
// inside the window; the best of `restarts` such splits is kept.
// The paper's clustering partitioner is not public; this is a plain
// min-cut bisection in its place.
struct Bisector {
    const Problem &p;
    Rng rng;
    double eps;
    int leaf_max, restarts;
    bool plain_leaves;
    std::vector<std::array<int, 2>> holders;  // the (up to) two leaves holding each label
    std::vector<int> where;                   // leaf -> index in the current part, or -1
    Tree tree;
    int nxt;

    Bisector(const Problem &pr, uint64_t seed, double e, int lm, int rs, bool plain)
        : p(pr), rng(seed), eps(e), leaf_max(lm), restarts(rs), plain_leaves(plain), holders(pr.L, {-1, -1}),
          where(pr.n, -1), nxt(pr.n) {
        for (int i = 0; i < p.n; i++)
            for (int id : p.leaf_labels[i]) {
                auto &h = holders[id];
                if (h[0] < 0) h[0] = i; else if (h[0] != i) h[1] = i;
            }
    }

    int other(int id, int v) const { return holders[id][0] == v ? holders[id][1] : holders[id][0]; }

    // greedy order inside part S, the labels leaving S taken as open
    int greedy_part(const std::vector<int> &S) {
        const int m = (int)S.size(), W = p.leaf.W;
        Problem sub;
        sub.n = m;
        sub.L = p.L;
        sub.leaf.init(m, p.L);
        sub.open = p.open;
        sub.leaf_labels.resize(m);
        for (int i = 0; i < m; i++) where[S[i]] = i;
        for (int i = 0; i < m; i++) {
            std::memcpy(sub.leaf.at(i), p.leaf.at(S[i]), sizeof(uint64_t) * W);
            sub.leaf_labels[i] = p.leaf_labels[S[i]];
            for (int id : p.leaf_labels[S[i]]) {
                const int o = other(id, S[i]);
                if (o < 0 || where[o] < 0) sub.open[id >> 6] |= 1ull << (id & 63);
            }
        }
        for (int v : S) where[v] = -1;
        const Tree t = greedy_trial(sub, rng.next(), plain_leaves);
        std::vector<int> map(2 * m - 1);
        for (int i = 0; i < m; i++) map[i] = S[i];
        for (int s = 0; s < (int)t.size(); s++) {
            tree.push_back({map[t[s].first], map[t[s].second]});
            map[m + s] = nxt++;
        }
        return map[2 * m - 2];
    }

    // split S into two parts inside the balance window with a small cut
    void split(const std::vector<int> &S, std::vector<int> &A, std::vector<int> &B) {
        const int m = (int)S.size();
        for (int i = 0; i < m; i++) where[S[i]] = i;
        std::vector<std::vector<int>> nb(m);  // one entry per shared label
        for (int i = 0; i < m; i++)
            for (int id : p.leaf_labels[S[i]]) {
                const int o = other(id, S[i]);
                if (o >= 0 && where[o] >= 0) nb[i].push_back(where[o]);
            }
        for (int v : S) where[v] = -1;
        int lo = (int)std::ceil(0.5 * (1.0 - eps) * m), hi = (int)std::floor(0.5 * (1.0 + eps) * m);
        lo = std::max(lo, 1);
        hi = std::min(hi, m - 1);
        if (lo > hi) lo = hi = m / 2;
        std::vector<int> best_side;
        int best_cut = -1, best_imb = 0;
        std::vector<int> side(m), conn(m);
        for (int r = 0; r < restarts; r++) {
            // region growth from a random tensor to a random size in [lo, hi]
            const int target = lo + (int)(rng.next() % (uint64_t)(hi - lo + 1));
            std::fill(side.begin(), side.end(), 1);
            std::fill(conn.begin(), conn.end(), 0);
            int n0 = 0;
            int v = (int)(rng.next() % (uint64_t)m);
            for (;;) {
                side[v] = 0;
                n0++;
                for (int j : nb[v]) conn[j]++;
                if (n0 >= target) break;
                int bv = -1, bc = -1, ties = 0;
                for (int j = 0; j < m; j++) {
                    if (side[j] == 0) continue;
                    if (conn[j] > bc) { bc = conn[j]; bv = j; ties = 1; }
                    else if (conn[j] == bc && rng.next() % (uint64_t)(++ties) == 0) bv = j;
                }
                v = bv;
            }
            const int cut = fm_refine(nb, side, nullptr, lo, hi, 12);
            n0 = 0;
            for (int i = 0; i < m; i++) n0 += side[i] == 0;
            const int imb = std::abs(2 * n0 - m);
            if (best_cut < 0 || cut < best_cut || (cut == best_cut && imb < best_imb)) {
                best_cut = cut;
                best_imb = imb;
                best_side = side;
            }
        }
        A.clear();
        B.clear();
        for (int i = 0; i < m; i++) (best_side[i] == 0 ? A : B).push_back(S[i]);
    }

    int build(const std::vector<int> &S) {
        if (S.size() == 1) return S[0];
        if ((int)S.size() <= leaf_max) return greedy_part(S);
        std::vector<int> A, B;
        split(S, A, B);
        const int a = build(A), b = build(B);
        tree.push_back({std::min(a, b), std::max(a, b)});
        return nxt++;
    }
};

// One hierarchical-bipartition trial.  plain: the balance window +-10%,
// parts of <= 60 tensors (the paper's setting) and plain greedy inside;
// else the window, the part size and the greedy noise are drawn from seed.
Tree bipartition_trial(const Problem &p, uint64_t seed, bool plain) {
    Rng rng(seed);
    double eps = 0.1;
    int leaf_max = 60, restarts = 4;
    if (!plain) {
        eps = 0.02 + 0.58 * rng.uniform();
        leaf_max = (int)std::lround(std::exp2(1.0 + 5.0 * rng.uniform()));
        restarts = 1 + (int)(rng.next() % 4);
    }
    Bisector bs(p, rng.next(), eps, std::max(leaf_max, 2), restarts, plain);
    std::vector<int> all(p.n);
    for (int i = 0; i < p.n; i++) all[i] = i;
    bs.build(all);
    return bs.tree;
}

// Subtree reconfiguration.  For each internal node v, the subtree below v is
// cut at a frontier of up to kmax tensors (expanding the costliest step
// first) and the frontier is re-contracted in the cheapest order, found by
// dynamic programming over subsets: a subset's tensor has the XOR of the
// frontier label sets (a label held by two frontier tensors is contracted),
// and merging subsets Y, Z costs 2^{|labels(Y) u labels(Z)| minus sliced}.
// v keeps its output, so the rest of the tree is unchanged.
Tree reconfigure(const Problem &p, const Tree &tree, const std::vector<uint64_t> &smask, int kmax, int passes,
                 uint64_t seed) {
    const int n = p.n, W = p.leaf.W, N = 2 * n - 1;
    if (n < 3) return tree;
    std::vector<int> c0(N, -1), c1(N, -1), parent(N, -1);
    Sets set;
    set.init(N, p.L);
    std::memcpy(set.at(0), p.leaf.at(0), sizeof(uint64_t) * W * n);
    for (int t = 0; t < n - 1; t++) {
        const int v = n + t, a = tree[t].first, b = tree[t].second;
        c0[v] = a;
        c1[v] = b;
        parent[a] = parent[b] = v;
        for (int w = 0; w < W; w++) set.at(v)[w] = set.at(a)[w] ^ set.at(b)[w];
    }
    const int root = N - 1;
    auto step_cost = [&](int v) {
        int c = 0;
        for (int w = 0; w < W; w++) c += __builtin_popcountll((set.at(c0[v])[w] | set.at(c1[v])[w]) & ~smask[w]);
        return std::exp2((double)c);
    };
    Rng rng(seed);
    std::vector<int> order;
    for (int v = n; v < N; v++) order.push_back(v);
    for (int pass = 0; pass < passes; pass++) {
        for (int i = (int)order.size() - 1; i > 0; i--) std::swap(order[i], order[rng.next() % (uint64_t)(i + 1)]);
        for (int v : order) {
            std::vector<int> fr{v}, inner;
            while ((int)fr.size() < kmax) {
                int bi = -1;
                double bc = -1;
                for (int i = 0; i < (int)fr.size(); i++)
                    if (c0[fr[i]] >= 0) {
                        const double c = step_cost(fr[i]);
                        if (c > bc) { bc = c; bi = i; }
                    }
                if (bi < 0) break;
                const int u = fr[bi];
                inner.push_back(u);
                fr[bi] = c0[u];
                fr.push_back(c1[u]);
            }
            const int k = (int)fr.size();
            if (k < 3) continue;
            // local label index over the frontier's labels
            std::vector<int> lab;
            for (int f : fr)
                for (int w = 0; w < W; w++) {
                    uint64_t x = set.at(f)[w];
                    while (x) {
                        const int l = w * 64 + __builtin_ctzll(x);
                        x &= x - 1;
                        if (std::find(lab.begin(), lab.end(), l) == lab.end()) lab.push_back(l);
                    }
                }
            const int LW = ((int)lab.size() + 63) / 64;
            if (LW > 16) continue;
            const int S = 1 << k;
            std::vector<uint64_t> L((size_t)S * LW, 0), sl(LW, 0);
            for (int j = 0; j < (int)lab.size(); j++) {
                const int l = lab[j];
                if ((smask[l >> 6] >> (l & 63)) & 1) sl[j >> 6] |= 1ull << (j & 63);
                for (int i = 0; i < k; i++)
                    if ((set.at(fr[i])[l >> 6] >> (l & 63)) & 1) L[(size_t)(1 << i) * LW + (j >> 6)] |= 1ull << (j & 63);
            }
            for (int X = 1; X < S; X++) {
                const int low = X & -X;
                if (X == low) continue;
                for (int w = 0; w < LW; w++) L[(size_t)X * LW + w] = L[(size_t)low * LW + w] ^ L[(size_t)(X ^ low) * LW + w];
            }
            std::vector<double> best(S, 0.0);
            std::vector<int> split(S, 0);
            for (int X = 1; X < S; X++) {
                const int low = X & -X;
                if (X == low) continue;
                best[X] = INFINITY;
                for (int Y = (X - 1) & X; Y > 0; Y = (Y - 1) & X) {
                    if (!(Y & low)) continue;
                    const int Z = X ^ Y;
                    int c = 0;
                    for (int w = 0; w < LW; w++)
                        c += __builtin_popcountll((L[(size_t)Y * LW + w] | L[(size_t)Z * LW + w]) & ~sl[w]);
                    const double tot = best[Y] + best[Z] + std::exp2((double)c);
                    if (tot < best[X]) { best[X] = tot; split[X] = Y; }
                }
            }
            double cur = step_cost(v);
            for (int u : inner) cur += step_cost(u);
            if (!(best[S - 1] < cur * (1.0 - 1e-9))) continue;
            // rebuild the subtree on the same node ids, v stays its root
            std::vector<int> ids = inner;
            std::vector<std::pair<int, int>> stack{{S - 1, v}};
            while (!stack.empty()) {
                const int X = stack.back().first, id = stack.back().second;
                stack.pop_back();
                const int Y = split[X], Z = X ^ Y;
                int ch[2];
                for (int q = 0; q < 2; q++) {
                    const int part = q ? Z : Y;
                    if ((part & (part - 1)) == 0) {
                        ch[q] = fr[__builtin_ctz(part)];
                    } else {
                        ch[q] = ids.back();
                        ids.pop_back();
                        stack.push_back({part, ch[q]});
                    }
                    parent[ch[q]] = id;
                }
                c0[id] = ch[0];
                c1[id] = ch[1];
            }
            // label sets of the rebuilt internal nodes, children first
            std::vector<int> post, st2{v};
            while (!st2.empty()) {
                const int u = st2.back();
                st2.pop_back();
                post.push_back(u);
                for (int c : {c0[u], c1[u]})
                    if (c >= n && std::find(fr.begin(), fr.end(), c) == fr.end()) st2.push_back(c);
            }
            for (int i = (int)post.size() - 1; i >= 0; i--) {
                const int u = post[i];
                for (int w = 0; w < W; w++) set.at(u)[w] = set.at(c0[u])[w] ^ set.at(c1[u])[w];
            }
        }
    }
    // serialise: post-order from the root, internal nodes renumbered n + t
    Tree out;
    std::vector<int> ssa(N, -1);
    for (int i = 0; i < n; i++) ssa[i] = i;
    std::vector<std::pair<int, int>> st{{root, 0}};
    while (!st.empty()) {
        auto &top = st.back();
        const int u = top.first;
        if (u < n) { st.pop_back(); continue; }
        if (top.second == 0) { top.second = 1; st.push_back({c0[u], 0}); continue; }
        if (top.second == 1) { top.second = 2; st.push_back({c1[u], 0}); continue; }
        out.push_back({ssa[c0[u]], ssa[c1[u]]});
        ssa[u] = n + (int)out.size() - 1;
        st.pop_back();
    }
    return out;
}

}  // namespace

const char *check_network(const std::vector<std::vector<int32_t>> &labels, const std::vector<int32_t> &open) {
    std::unordered_map<int32_t, int> cnt;
    for (const auto &l : labels) {
        for (size_t a = 0; a < l.size(); a++) {
            for (size_t b = a + 1; b < l.size(); b++)
                if (l[a] == l[b]) return "label repeated within a tensor";
            if (++cnt[l[a]] > 2) return "label held by more than two tensors";
        }
    }
    std::unordered_map<int32_t, int> seen;
    for (int32_t x : open) {
        auto it = cnt.find(x);
        if (it == cnt.end()) return "open label held by no tensor";
        if (it->second == 2) return "open label held by two tensors";
        if (++seen[x] > 1) return "open label repeated";
    }
    for (const auto &kv : cnt)
        if (kv.second == 1 && !seen.count(kv.first)) return "label held by one tensor must be open";
    return nullptr;
}

tn_search_opts default_search_opts() {
    tn_search_opts o;
    std::memset(&o, 0, sizeof o);
    o.trials = 256;
    o.seed = 0x2103030740ull;
    o.log2_cap = -1;
    o.n_sliced = -1;
    o.threads = 0;
    o.candidates = 0;
    o.rank_batch_log2 = -1;
    o.rank_form = TN_FP32;
    o.cost_model = nullptr;
    return o;
}

bool evaluate_tree(const std::vector<std::vector<int32_t>> &labels, const std::vector<int32_t> &open,
                   const Tree &tree, const std::vector<int32_t> &sliced, SearchResult &out) {
    Problem p;
    if (make_problem(labels, open, p)) return false;
    TreeSets ts;
    if (!tree_sets(p, tree, ts)) return false;
    std::unordered_map<int32_t, int> remap;
    for (int i = 0; i < p.L; i++) remap[p.id2label[i]] = i;
    std::vector<uint64_t> smask(p.leaf.W, 0);
    for (int32_t x : sliced) {
        auto it = remap.find(x);
        if (it == remap.end()) return false;
        smask[it->second >> 6] |= 1ull << (it->second & 63);
    }
    int n_nodes = 2 * p.n - 1, n_steps = p.n - 1;
    std::vector<double> e;
    double width = 0;
    for (int v = 0; v < n_nodes; v++) {
        int c = 0;
        for (int w = 0; w < p.leaf.W; w++) c += __builtin_popcountll(ts.node.at(v)[w] & ~smask[w]);
        width = std::max(width, (double)c);
    }
    for (int t = 0; t < n_steps; t++) {
        int c = 0;
        for (int w = 0; w < p.leaf.W; w++) c += __builtin_popcountll(ts.uni.at(t)[w] & ~smask[w]);
        e.push_back(c);
    }
    out.tree = tree;
    out.sliced = sliced;
    out.log2_slice = n_steps ? log2_sum_pow2(e) : 0.0;
    out.log2_width = width;
    out.log2_total = out.log2_slice + (double)sliced.size();
    return true;
}

int search_order_top(const std::vector<std::vector<int32_t>> &labels, const std::vector<int32_t> &open,
                     const tn_search_opts &opts_in, int k, std::vector<SearchResult> &out) {
    tn_search_opts opts = opts_in;
    if (opts.trials <= 0) opts.trials = 256;
    if (k < 1) k = 1;
    out.clear();
    Problem p;
    if (const char *bad = check_network(labels, open)) return fail(TN_ERR_ARG, std::string("order search: ") + bad);
    if (const char *bad = make_problem(labels, open, p)) return fail(TN_ERR_ARG, std::string("order search: ") + bad);
    if (p.n == 0) return fail(TN_ERR_ARG, "empty network");
    if (opts.method < 0 || opts.method > 2) return fail(TN_ERR_ARG, "unknown order-search method");
    if (opts.objective < 0 || opts.objective > 2) return fail(TN_ERR_ARG, "unknown order-search objective");
    const tn_form rform =
        (opts.rank_form >= TN_FP32 && opts.rank_form <= TN_FP16X3) ? (tn_form)opts.rank_form : TN_FP32;
    // the trials' score: log2 of total MACs, or of the compiled plan's roofline time
    const auto score = [&](const Tree &tree, const SliceEval &ev) {
        if (opts.objective == 0) return ev.log2_total;
        std::vector<int32_t> sl;
        for (int id : ev.sliced) sl.push_back(p.id2label[id]);
        const double ms = tree_roofline_ms(labels, open, tree, sl, rform, opts.rank_batch_log2, kNominalArenaBytes,
                                           opts.objective == 2);
        return ms > 0 ? std::log2(ms) : (double)INFINITY;
    };
    if (p.n == 1) {
        SearchResult r;
        r.log2_width = (double)labels[0].size();
        out.push_back(r);
        return TN_OK;
    }
    int threads = opts.threads > 0 ? opts.threads : (int)std::max(1u, std::thread::hardware_concurrency());
    threads = std::min(threads, opts.trials);
    // total: the score the candidates are ranked by; rl: the roofline score
    // (objective 1 only)
    struct Cand { double key_w, total, width; int trial; Tree tree; SliceEval ev; double rl = 0; };
    // order: smaller over-cap width, then the smaller score (log2 MACs or log2
    // roofline ms), then lower trial
    auto better = [](const Cand &a, const Cand &b) {
        if (a.key_w != b.key_w) return a.key_w < b.key_w;
        if (a.total != b.total) return a.total < b.total;
        return a.trial < b.trial;
    };
    // every thread keeps its kk best, so the union holds the global kk best
    // whatever the thread count (the search is deterministic in the seed)
    // bipartition trees change more under reconfiguration, so more of them
    // are reconfigured (greedy keeps its measured 4)
    const int kk = std::max(k, opts.method == 0 ? 4 : 16);
    std::vector<std::vector<Cand>> keep(threads), keep_m(threads);
    std::atomic<int> next{0};
    const auto insert = [&](std::vector<Cand> &mine, Cand &&c) {
        if ((int)mine.size() < kk) {
            mine.push_back(std::move(c));
            std::sort(mine.begin(), mine.end(), better);
        } else if (better(c, mine.back())) {
            mine.back() = std::move(c);
            std::sort(mine.begin(), mine.end(), better);
        }
    };
    auto worker = [&](int tid) {
        TreeSets ts;
        auto &mine = keep[tid];
        for (;;) {
            int t = next.fetch_add(1);
            if (t >= opts.trials) break;
            const uint64_t ts_seed = opts.seed + 0x9E3779B97F4A7C15ull * (uint64_t)(t + 1);
            const bool bip = opts.method == 1 || (opts.method == 2 && (t & 1));
            Tree tree = bip ? bipartition_trial(p, ts_seed, t == (opts.method == 2 ? 1 : 0))
                            : greedy_trial(p, ts_seed, t == 0);
            if (!tree_sets(p, tree, ts)) continue;
            SliceEval ev;
            // both slicing rules; the cheaper result that meets the cap wins
            SliceEval ev1;
            slice_tree(p, ts, 2 * p.n - 1, p.n - 1, opts.log2_cap, opts.n_sliced, 0, ev);
            slice_tree(p, ts, 2 * p.n - 1, p.n - 1, opts.log2_cap, opts.n_sliced, 1, ev1);
            const auto key = [&](const SliceEval &e) {
                const bool over = opts.log2_cap >= 0 && e.log2_width > opts.log2_cap;
                return std::make_pair(over ? e.log2_width : 0.0, e.log2_total);
            };
            if (key(ev1) < key(ev)) ev = std::move(ev1);
            const bool over = opts.log2_cap >= 0 && ev.log2_width > opts.log2_cap;
            const double sc = score(tree, ev);
            // the roofline objective also keeps the best trials by MACs:
            // reconfiguration reshapes a tree, so its time before says
            // little about its time after
            if (opts.objective >= 1)
                insert(keep_m[tid], Cand{over ? ev.log2_width : 0.0, ev.log2_total, ev.log2_width, t, tree, ev, sc});
            insert(mine, Cand{over ? ev.log2_width : 0.0, sc, ev.log2_width, t, std::move(tree), ev, sc});
        }
    };
    std::vector<std::thread> pool;
    for (int i = 1; i < threads; i++) pool.emplace_back(worker, i);
    worker(0);
    for (auto &th : pool) th.join();
    std::vector<Cand> all;
    for (auto &v : keep)
        for (auto &c : v) all.push_back(std::move(c));
    std::sort(all.begin(), all.end(), better);
    if (all.empty()) return fail(TN_ERR_ARG, "order search produced no tree");
    if ((int)all.size() > kk) all.resize(kk);
    if (opts.objective >= 1) {
        // the MAC-ranked candidates first, in the order (and so with the
        // reconfiguration seeds) a MAC-ranked search gives them, then the
        // time-ranked ones it lacks: the time-ranked pick can only improve
        // on the MAC-ranked one; all ranked by roofline time from here on
        std::vector<Cand> bym;
        for (auto &v : keep_m)
            for (auto &c : v) bym.push_back(std::move(c));
        std::sort(bym.begin(), bym.end(), better);
        if ((int)bym.size() > kk) bym.resize(kk);
        for (auto &c : all) {
            bool dup = false;
            for (const auto &b : bym) dup = dup || b.trial == c.trial;
            if (!dup) bym.push_back(std::move(c));
        }
        all = std::move(bym);
        for (auto &c : all) c.total = c.rl;
    }
    // subtree reconfiguration of the best few trees, under their slicing,
    // then slicing again and a second round under the new slice set
    if (opts.trials > 1) {
        const int R = (int)all.size();
        std::vector<Cand> extra(R);
        std::vector<std::thread> pool2;
        auto improve = [&](int i) {
            const Cand &c = all[i];
            Tree t = c.tree;
            SliceEval ev = c.ev;
            TreeSets ts;
            for (int round = 0; round < 4; round++) {
                std::vector<uint64_t> sm(p.leaf.W, 0);
                for (int id : ev.sliced) sm[id >> 6] |= 1ull << (id & 63);
                t = reconfigure(p, t, sm, 11, 4, opts.seed + 0x51ED27u * (uint64_t)(i * 2 + round + 1));
                if (!tree_sets(p, t, ts)) return;
                SliceEval e0, e1;
                slice_tree(p, ts, 2 * p.n - 1, p.n - 1, opts.log2_cap, opts.n_sliced, 0, e0);
                slice_tree(p, ts, 2 * p.n - 1, p.n - 1, opts.log2_cap, opts.n_sliced, 1, e1);
                const auto key = [&](const SliceEval &e) {
                    const bool over = opts.log2_cap >= 0 && e.log2_width > opts.log2_cap;
                    return std::make_pair(over ? e.log2_width : 0.0, e.log2_total);
                };
                ev = key(e1) < key(e0) ? std::move(e1) : std::move(e0);
            }
            const bool over = opts.log2_cap >= 0 && ev.log2_width > opts.log2_cap;
            const double sc = score(t, ev);
            extra[i] = Cand{over ? ev.log2_width : 0.0, sc, ev.log2_width, c.trial, std::move(t), ev};
        };
        for (int i = 1; i < R; i++) pool2.emplace_back(improve, i);
        improve(0);
        for (auto &th : pool2) th.join();
        for (auto &c : extra)
            if (!c.tree.empty()) all.push_back(std::move(c));
    }
    std::sort(all.begin(), all.end(), better);
    for (auto &c : all) {
        if ((int)out.size() >= k) break;
        bool dup = false;
        for (auto &o : out)
            if (o.tree == c.tree) { dup = true; break; }
        if (dup) continue;
        SearchResult r;
        r.tree = c.tree;
        for (int id : c.ev.sliced) r.sliced.push_back(p.id2label[id]);
        r.log2_total = c.ev.log2_total;
        r.log2_width = c.ev.log2_width;
        r.log2_slice = c.ev.log2_slice_cost;
        out.push_back(std::move(r));
    }
    if (out.empty()) return fail(TN_ERR_ARG, "order search produced no tree");
    return TN_OK;
}

int search_order(const std::vector<std::vector<int32_t>> &labels, const std::vector<int32_t> &open,
                 const tn_search_opts &opts, SearchResult &out) {
    std::vector<SearchResult> top;
    int rc = search_order_top(labels, open, opts, 1, top);
    if (rc) return rc;
    out = top[0];
    return TN_OK;
}

}  // namespace tn

// ---------------------------------------------------------------- branch merging
// A big tensor X met by two small ones in turn, ((X a) b), streams X through
// memory twice; (X (a b)) merges the small ones first and streams X once, at
// the price of more arithmetic when a and b share no bond ("Details of
// simulations": merging branches balances the pairwise contractions).  The
// rewrite is kept where a per-step time estimate drops: the larger of the
// step's bytes over 7 TB/s and its FP32 flops over 80 TFLOP/s, with sliced
// labels kept as batch labels (as the executor runs a block of slices).
namespace tn {
namespace {

struct BNode {
    int l = -1, r = -1;  // children (internal nodes); -1 for leaves
};

double step_time(int ra, int rb, int rc, int ru) {
    const double bytes = 8.0 * (std::exp2(ra) + std::exp2(rb) + std::exp2(rc));
    const double flops = 8.0 * std::exp2(ru);
    return std::max(bytes / 7.0e12, flops / 80.0e12);
}

}  // namespace
}  // namespace tn

extern "C" int tn_merge_branches(int n_tensors, const int32_t *ranks, const int32_t *labels, int n_open,
                                 const int32_t *open_labels, int n_sliced, const int32_t *sliced_labels,
                                 int n_steps, const int32_t *tree_in, int max_small_rank, int32_t *tree_out,
                                 double *stats) {
    using namespace tn;
    if (n_tensors < 1 || !ranks || !labels || n_steps != n_tensors - 1 || (n_steps > 0 && (!tree_in || !tree_out)) ||
        n_open < 0 || (n_open > 0 && !open_labels) || n_sliced < 0 || (n_sliced > 0 && !sliced_labels))
        return fail(TN_ERR_ARG, "tn_merge_branches: bad arguments");
    const int n = n_tensors;
    std::vector<std::vector<int32_t>> labs(n);
    size_t off = 0;
    for (int i = 0; i < n; i++) {
        if (ranks[i] < 0 || ranks[i] > 62) return fail(TN_ERR_ARG, "tn_merge_branches: rank out of range");
        labs[i].assign(labels + off, labels + off + ranks[i]);
        off += ranks[i];
    }
    // sliced labels stay in the tensors (batch labels), like open labels
    std::vector<int32_t> kept(open_labels, open_labels + n_open);
    kept.insert(kept.end(), sliced_labels, sliced_labels + n_sliced);
    Problem p;
    if (const char *bad = make_problem(labs, kept, p)) return fail(TN_ERR_ARG, std::string("tn_merge_branches: ") + bad);
    Tree tree(n_steps);
    for (int t = 0; t < n_steps; t++) tree[t] = {tree_in[2 * t], tree_in[2 * t + 1]};
    TreeSets ts;
    if (!tree_sets(p, tree, ts)) return fail(TN_ERR_ARG, "tn_merge_branches: malformed tree");
    if (n_steps == 0) {
        if (stats) stats[0] = stats[1] = stats[2] = 0;
        return TN_OK;
    }
    const int W = p.leaf.W, nn = 2 * n - 1;
    std::vector<BNode> node(nn);
    for (int t = 0; t < n_steps; t++) node[n + t] = {tree[t].first, tree[t].second};
    const int root = nn - 1;
    // label sets bottom-up (children before parents: any post-order)
    Sets set;
    set.init(nn, p.L);
    std::vector<int> order;
    auto post = [&]() {
        order.clear();
        std::vector<std::pair<int, bool>> st{{root, false}};
        while (!st.empty()) {
            auto [x, done] = st.back();
            st.pop_back();
            if (x < n || done) {
                order.push_back(x);
                continue;
            }
            st.push_back({x, true});
            st.push_back({node[x].r, false});
            st.push_back({node[x].l, false});
        }
    };
    auto compute = [&](int x) {
        uint64_t *so = set.at(x);
        if (x < n) {
            std::memcpy(so, p.leaf.at(x), sizeof(uint64_t) * W);
            return;
        }
        const uint64_t *sa = set.at(node[x].l), *sb = set.at(node[x].r);
        for (int w = 0; w < W; w++) so[w] = (sa[w] | sb[w]) & ~(sa[w] & sb[w] & ~p.open[w]);
    };
    auto rank_of = [&](int x) { return popc(set.at(x), W); };
    auto union_rank = [&](int a, int b) {
        int c = 0;
        for (int w = 0; w < W; w++) c += __builtin_popcountll(set.at(a)[w] | set.at(b)[w]);
        return c;
    };
    auto out_rank = [&](int a, int b) {  // rank of the contraction of a and b
        int c = 0;
        for (int w = 0; w < W; w++) {
            const uint64_t sa = set.at(a)[w], sb = set.at(b)[w];
            c += __builtin_popcountll((sa | sb) & ~(sa & sb & ~p.open[w]));
        }
        return c;
    };
    auto log2_macs = [&]() {
        std::vector<double> e;
        for (int x = n; x < nn; x++) e.push_back((double)union_rank(node[x].l, node[x].r));
        return log2_sum_pow2(e);
    };
    post();
    for (int x : order) compute(x);
    const double before = log2_macs();
    const int small = max_small_rank > 0 ? max_small_rank : 12;
    int rewrites = 0;
    for (int pass = 0; pass < 64; pass++) {
        bool changed = false;
        post();
        for (int P : order) {
            if (P < n) continue;
            for (int side = 0; side < 2; side++) {
                const int Q = side == 0 ? node[P].l : node[P].r, b = side == 0 ? node[P].r : node[P].l;
                if (Q < n || rank_of(b) > small) continue;
                // X: the larger child of Q, a: the smaller
                int X = node[Q].l, a = node[Q].r;
                if (rank_of(a) > rank_of(X)) std::swap(X, a);
                if (rank_of(a) > small) continue;
                const int rm = out_rank(a, b);
                if (rm > small) continue;
                const double t_old = step_time(rank_of(X), rank_of(a), rank_of(Q), union_rank(X, a)) +
                                     step_time(rank_of(Q), rank_of(b), rank_of(P), union_rank(Q, b));
                // after: M = (a b), P = (X M); P's labels are unchanged
                const int rp = rank_of(P);
                int ru = 0;  // |X u M|
                for (int w = 0; w < W; w++) {
                    const uint64_t sa = set.at(a)[w], sb = set.at(b)[w];
                    const uint64_t sm = (sa | sb) & ~(sa & sb & ~p.open[w]);
                    ru += __builtin_popcountll(set.at(X)[w] | sm);
                }
                const double t_new = step_time(rank_of(a), rank_of(b), rm, union_rank(a, b)) +
                                     step_time(rank_of(X), rm, rp, ru);
                if (t_new < 0.95 * t_old) {
                    node[Q] = {a, b};
                    node[P] = {X, Q};
                    compute(Q);
                    compute(P);
                    rewrites++;
                    changed = true;
                    break;
                }
            }
        }
        if (!changed) break;
    }
    // re-linearise: post-order, leaves keep their ids, steps numbered anew
    post();
    std::vector<int> id(nn, -1);
    for (int i = 0; i < n; i++) id[i] = i;
    int next = n, t = 0;
    for (int x : order) {
        if (x < n) continue;
        tree_out[2 * t] = id[node[x].l];
        tree_out[2 * t + 1] = id[node[x].r];
        id[x] = next++;
        t++;
    }
    if (stats) {
        stats[0] = rewrites;
        stats[1] = before;
        stats[2] = log2_macs();
    }
    return TN_OK;
}

// ---------------------------------------------------------------- slicing a given tree
// The slicing step of the search ("Dynamic slicing": bonds fixed one at a
// time until every intermediate fits) applied to a tree the caller already
// has: both greedy rules run and the cheaper result that meets the cap wins,
// as in the search.
namespace tn {

extern "C" int tn_slice_tree(int n_tensors, const int32_t *ranks, const int32_t *labels, int n_open,
                             const int32_t *open_labels, int n_steps, const int32_t *tree, int log2_cap,
                             int n_sliced, int max_sliced, int32_t *out_sliced, int *out_n_sliced,
                             double *stats) {
    if (n_tensors < 1 || !ranks || !labels || n_steps != n_tensors - 1 || (n_steps > 0 && !tree) || n_open < 0 ||
        (n_open > 0 && !open_labels) || (log2_cap < 0 && n_sliced < 0) || max_sliced < 0 ||
        (max_sliced > 0 && !out_sliced))
        return fail(TN_ERR_ARG, "tn_slice_tree: bad arguments");
    std::vector<std::vector<int32_t>> labs(n_tensors);
    size_t off = 0;
    for (int i = 0; i < n_tensors; i++) {
        if (ranks[i] < 0 || ranks[i] > 62) return fail(TN_ERR_ARG, "tn_slice_tree: rank out of range");
        labs[i].assign(labels + off, labels + off + ranks[i]);
        off += ranks[i];
    }
    const std::vector<int32_t> open(open_labels, open_labels + n_open);
    if (const char *bad = check_network(labs, open)) return fail(TN_ERR_ARG, std::string("tn_slice_tree: ") + bad);
    Problem p;
    if (const char *bad = make_problem(labs, open, p)) return fail(TN_ERR_ARG, std::string("tn_slice_tree: ") + bad);
    Tree t(n_steps);
    for (int i = 0; i < n_steps; i++) t[i] = {tree[2 * i], tree[2 * i + 1]};
    TreeSets ts;
    if (!tree_sets(p, t, ts)) return fail(TN_ERR_ARG, "tn_slice_tree: malformed tree");
    SliceEval e0, e1;
    slice_tree(p, ts, 2 * p.n - 1, p.n - 1, log2_cap, n_sliced, 0, e0);
    slice_tree(p, ts, 2 * p.n - 1, p.n - 1, log2_cap, n_sliced, 1, e1);
    const auto key = [&](const SliceEval &e) {
        const bool over = log2_cap >= 0 && e.log2_width > log2_cap;
        return std::make_pair(over ? e.log2_width : 0.0, e.log2_total);
    };
    const SliceEval &ev = key(e1) < key(e0) ? e1 : e0;
    if ((int)ev.sliced.size() > max_sliced) return fail(TN_ERR_ARG, "tn_slice_tree: max_sliced too small");
    for (size_t j = 0; j < ev.sliced.size(); j++) out_sliced[j] = p.id2label[ev.sliced[j]];
    if (out_n_sliced) *out_n_sliced = (int)ev.sliced.size();
    if (stats) {
        stats[0] = ev.log2_total;
        stats[1] = ev.log2_width;
        stats[2] = (double)ev.sliced.size();
        stats[3] = ev.log2_slice_cost;
    }
    return TN_OK;
}

}  // namespace tn
