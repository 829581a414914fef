// Plan compiler and the device-side C-ABI calls.
//
// A plan turns (network, open labels, sliced labels, tree) into a fixed
// sequence of kernel launches over a static device arena:
//
//  * Slices run in aligned blocks of 2^nb consecutive slice ids.  Within a
//    block the nb lowest sliced labels stay in the network as batch labels
//    (never summed, carried to the root); the other sliced labels are fixed
//    at the leaves from the block's base id (slice extraction).  The root then
//    holds one partial amplitude tensor per slice of the block, and the
//    cross-slice FP64 sum adds the slices of the requested range into the
//    caller's amplitude tensor ("Dynamic slicing": the sum over slices is the
//    unsliced contraction).
//  * Nodes whose subtree holds no fixed sliced label are slice-invariant: they
//    are computed once per call (prologue), not once per block.
//  * Each pairwise step (Fig. 3: H batch labels, M / N outer labels, K shared
//    labels, cost 2^{H+M+N+K} complex MACs) is either a "small" step (one
//    operand <= 2^12 values, staged in shared memory, the other read once with
//    bit-scatter addressing, output written in the big operand's layout with
//    K labels replaced by N labels) or a strided batched GEMM whose operands
//    are permuted first when their H/M/K label groups are not contiguous.
//  * Buffers are placed in one arena by first-fit over their live intervals.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <set>
#include <string>
#include <unordered_map>
#include <unordered_set>

#include <cuda_runtime.h>

#include "costmodel.h"
#include "kernels.h"
#include "tc_gemm.h"
#include "tn_internal.h"

namespace tn {

namespace {

// values double as the step-timing recorder's kind codes (3 = extract, 4 = sum)
enum OpKind { OP_SMALL = 0, OP_PERMUTE = 1, OP_GEMM = 2, OP_SPLIT = 5, OP_MAXABS = 6, OP_TASKS = 7 };

struct Operand {  // where an op reads or writes: static leaf or arena buffer
    int buf = -1;        // arena buffer id, or -1
    int64_t leaf_off = -1;  // element offset in the leaf buffer
};

struct Op {
    OpKind kind;
    int step = -1;
    bool dep = false;
    Operand in0, in1, out;
    Operand aux;    // scaled forms: the pair of max-abs slots (read by splits and the GEMM)
    int aux_idx = 0;  // slot index used by a max-abs op or a scaled split
    // tensor-core GEMM of a scaled form whose output feeds a scaled split: the
    // epilogue also writes max |re|, |im| of the output into this slot, in
    // place of a separate max-abs pass over the output
    Operand maxout;
    int maxout_idx = 0;
    SmallArgs small;
    MaxAbsArgs mx;
    BitPermArgs bp;  // permute (mode 0) or fused permute + hi/lo split (OP_SPLIT)
    GemmArgs gemm;
    TcGemm tc;  // tensor-core GEMM (gemm_variant 1), resolved after arena allocation
    double macs = 0, bytes = 0;
    int gemm_variant = 0;  // 0: FP32 CUDA cores, 1: tensor-core split form
    std::string note;      // plan-time decisions, for tn_plan_describe
    // OP_TASKS: small steps run as the tasks of one persistent launch, in
    // dependency order; the longest chain of members that feed each other;
    // the device task table (resolved after arena allocation, owned by the
    // plan)
    std::vector<Op> members;
    int task_levels = 0;
    std::vector<SmallTask> tasks;
    std::vector<int> unit_task;
    SmallTask *d_tasks = nullptr;
    int *d_unit_task = nullptr, *d_ctr = nullptr;
};

// f(operand, written) for every operand an op reads or writes (an OP_TASKS
// op: those of its members)
template <typename F>
void for_each_operand(const Op &op, F &&f) {
    if (op.kind == OP_TASKS) {
        for (const Op &m : op.members) for_each_operand(m, f);
        return;
    }
    f(op.in0, false);
    f(op.in1, false);
    f(op.aux, false);
    f(op.out, true);
    f(op.maxout, true);
}

struct Buf {
    int64_t elems = 0;
    int t0 = 0, t1 = 0;
    int64_t off = 0;  // bytes
};

struct NodeRec {
    std::vector<int32_t> lay;
    bool dep = false;
    bool extracted = false;
    int leaf = -1;
    Operand where;
    int t_prod = -1;
};

inline int pos_of(const std::vector<int32_t> &lay, int32_t x) {
    for (size_t i = 0; i < lay.size(); i++)
        if (lay[i] == x) return (int)(lay.size() - 1 - i);
    return -1;
}

struct Groups {
    bool ok = false;
    std::vector<int32_t> order[3];
    int lowpos[3] = {0, 0, 0};
};

// Are the labels of `lay` in contiguous runs per group (gid: label -> 0..2)?
Groups group_layout(const std::vector<int32_t> &lay, const std::unordered_map<int32_t, int> &gid) {
    Groups g;
    int r = (int)lay.size();
    int last = -1;
    bool seen[3] = {false, false, false};
    for (int i = 0; i < r; i++) {
        int id = gid.at(lay[i]);
        if (id != last) {
            if (seen[id]) return g;  // group split in two runs
            seen[id] = true;
            last = id;
        }
        g.order[id].push_back(lay[i]);
        g.lowpos[id] = r - 1 - i;
    }
    g.ok = true;
    return g;
}

// Tiled bit permutation from layout `src` to layout `dst` (same label set).
// The shared-memory tile takes the labels at the lowest positions of both
// layouts, alternating, up to kTileMaxBits, so that both the reads and the
// writes of a tile are runs of consecutive addresses.
BitPermArgs make_bitperm(const std::vector<int32_t> &src, const std::vector<int32_t> &dst, int mode) {
    BitPermArgs a;
    std::memset(&a, 0, sizeof a);
    const int r = (int)dst.size();
    a.rank = r;
    a.mode = mode;
    a.plane_stride = (int64_t)1 << r;
    std::vector<int> src_pos(r), dst_of_src(r);
    for (int p = 0; p < r; p++) {
        src_pos[p] = pos_of(src, dst[r - 1 - p]);
        dst_of_src[src_pos[p]] = p;
    }
    const int nt = std::min(kTileMaxBits, r);
    std::vector<char> in_tile(r, 0);
    int cnt = 0;
    auto add = [&](int p) {
        if (p < r && cnt < nt && !in_tile[p]) { in_tile[p] = 1; cnt++; }
    };
    // first the low destination bits of a 128-byte store run per plane (16
    // elements of complex64, 32 of a 32-bit plane, 64 of a 16-bit plane) and
    // the low source bits of a 128-byte load run (16 complex64 elements),
    // then destination and source bits alternately
    const int d_need = mode == 0 ? 4 : (mode_word(mode) ? 5 : 6), s_need = 4;
    int i_d = 0, i_s = 0;
    while (cnt < nt && (i_d < d_need || i_s < s_need)) {
        if (i_d < d_need) add(i_d++);
        if (i_s < s_need && i_s < r) add(dst_of_src[i_s++]);
        else if (i_s < s_need) i_s = s_need;
    }
    for (; cnt < nt && (i_d < r || i_s < r);) {
        if (i_d < r) add(i_d++);
        if (i_s < r) add(dst_of_src[i_s++]);
    }
    std::vector<int> tile;
    for (int p = 0; p < r; p++) {
        if (in_tile[p]) tile.push_back(p);
        else {
            a.rest_dst[a.n_rest] = p;
            a.rest_src[a.n_rest] = src_pos[p];
            a.n_rest++;
        }
    }
    a.n_tile = (int)tile.size();
    for (int j = 0; j < a.n_tile; j++) a.tile_dst[j] = tile[j];
    std::vector<int> order(a.n_tile);
    for (int j = 0; j < a.n_tile; j++) order[j] = j;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return src_pos[tile[x]] < src_pos[tile[y]]; });
    for (int j = 0; j < a.n_tile; j++) {
        a.rd_w[j] = order[j];
        a.rd_src[j] = src_pos[tile[order[j]]];
    }
    return a;
}

}  // namespace

}  // namespace tn

struct tn_plan {
    int device = 0;
    tn_form form = TN_FP32;
    int n_tensors = 0, n_open = 0, n_sliced = 0, nb = 0;
    std::vector<int32_t> open, sliced;
    // host copies
    std::vector<std::vector<int32_t>> labels;
    std::vector<int64_t> leaf_off;  // element offsets of leaves in d_leaves
    tn::Tree tree;
    // compiled
    std::vector<tn::Op> prologue, batch;
    std::vector<tn::Buf> bufs;
    std::vector<tn::ExtractEntry> extract;  // host copy (pointers resolved)
    int extract_max_out = 0;
    tn::AccumArgs accum;
    tn::Operand root;
    int64_t arena_bytes = 0;
    // device
    float2 *d_leaves = nullptr;
    char *d_arena = nullptr;
    double *d_host_amp = nullptr;  // tn_contract_slices_host: amplitudes + 3 statistics
    tn::ExtractEntry *d_extract = nullptr;
    std::vector<void *> task_mem;  // device task tables of OP_TASKS ops
    bool failed = false;
    // stats
    double macs_batch = 0, macs_prologue = 0, bytes_batch = 0, bytes_prologue = 0;
    int launches_batch = 0, launches_prologue = 0;
    tn_plan_opts opts = {};
    // step-timing recorder (profile mode)
    struct ProfRow {
        int phase, idx, kind, step;
        double ms;
        int64_t calls;
        double macs, bytes;
        double shape[4];  // GEMM / split: H, M (rows), N, K; other kinds: output rank
    };
    std::vector<ProfRow> prof;
    std::vector<cudaEvent_t> prof_ev;  // two per row
    int64_t leaf_bytes = 0;
    // CUDA-graph replay (opts.use_graph): the slice-invariant prologue and the
    // per-block body, captured once after the first eager call
    bool graphs_ready = false;
    cudaGraphExec_t g_pro = nullptr, g_body = nullptr;
    int64_t graph_calls = 0;
};

namespace tn {

namespace {

constexpr int kSmallMaxRank = 12;

// The op of `ops` that writes buffer w.buf (nullptr for a leaf or none).
Op *producer_of(std::vector<Op> &ops, const Operand &w) {
    if (w.buf < 0) return nullptr;
    for (auto &o : ops)
        if (o.out.buf == w.buf) return &o;
    return nullptr;
}

// Is w written by a tensor-core GEMM that could split its own output into
// the next step's planes (no split K, plain output so far)?
bool planar_candidate(std::vector<Op> &ops, const Operand &w) {
    const Op *p = producer_of(ops, w);
    return p && p->kind == OP_GEMM && p->gemm_variant == 1 && p->tc.ksplit == 1 && p->tc.out.mode == 0;
}

// Planar epilogue of a producer GEMM whose output (layout src, bit groups
// h | m | n of nH, nM, nN bits from the top) is written as split planes in
// layout dst.  Returns false when fewer than min_run low destination bits
// come from the epilogue's half tile (its writes would not be coalesced).
bool make_planar(const std::vector<int32_t> &src, const std::vector<int32_t> &dst, int nH, int nM, int nN, int mode,
                 int min_run, TcPlanarOut &o) {
    const int r = (int)src.size();
    if (r != (int)dst.size() || r != nH + nM + nN || nM < 6 || r > kMaxRank) return false;
    std::memset(&o, 0, sizeof o);
    o.mode = mode;
    o.plane_stride = (int64_t)1 << r;
    o.nH = nH;
    o.nM = nM;
    o.nN = nN;
    std::vector<int> dpos(r);
    for (int sp = 0; sp < r; sp++) {
        dpos[sp] = pos_of(dst, src[r - 1 - sp]);
        if (dpos[sp] < 0) return false;
    }
    for (int j = 0; j < nN; j++) o.npos[j] = (int8_t)dpos[j];
    for (int j = 0; j < nM; j++) o.mpos[j] = (int8_t)dpos[nN + j];
    for (int j = 0; j < nH; j++) o.hpos[j] = (int8_t)dpos[nN + nM + j];
    std::vector<std::pair<int, int>> bits;  // (destination position, tile bit)
    for (int b = 0; b < std::min(6, nN); b++) bits.push_back({o.npos[b], b});
    for (int b = 0; b < 6; b++) bits.push_back({o.mpos[b], 6 + b});
    std::sort(bits.begin(), bits.end());
    // the kernel's offsets inside a half tile are 32-bit (the tile base is
    // 64-bit), so every tile bit must land below destination bit 32
    if (bits.back().first >= 32) return false;
    o.ntb = (int)bits.size();
    int run = 0;
    for (int k = 0; k < o.ntb; k++) {
        o.tb[k] = (int8_t)bits[k].second;
        o.tpos[k] = (int8_t)bits[k].first;
        if (bits[k].first == k && run == k) run++;
    }
    return run >= min_run;
}

// Small steps whose T and C each hold at most 2^bits elements (and whose K
// has at most 2^kTaskMaxK values) run as the tasks of one persistent launch
// (OP_TASKS) instead of one launch each.  Scanning the op list in order, such
// a step joins the latest task group when each of its inputs comes from a
// member of that group or from an op before the group's position; otherwise
// it opens a new group at its own position.  A group runs where its first
// member stood, all members in one launch, so the timeline gives every member
// that one time (no member's buffer shares arena bytes with another's).
constexpr int kDefaultTaskBits = 17;

void group_tasks(std::vector<Op> &ops, int bits) {
    const int n = (int)ops.size();
    std::unordered_map<int, int> prod;  // arena buffer -> producing op
    for (int i = 0; i < n; i++)
        if (ops[i].out.buf >= 0) prod[ops[i].out.buf] = i;
    auto eligible = [&](const Op &op) {
        // (a step set up for the tiled kernel keeps its one-thread-per-row
        // fields; one that stores the next step's planes does not qualify)
        if (op.kind != OP_SMALL || op.small.tiled == 3 || op.small.nK > kTaskMaxK || op.maxout.buf >= 0) return false;
        const double elems = (double)op.small.rows * std::exp2((double)std::max(op.small.nK, op.small.nN));
        return elems <= std::exp2((double)bits);
    };
    std::vector<int> group(n, -1), level(n, 0), gpos, count;
    for (int i = 0; i < n; i++) {
        if (!eligible(ops[i])) continue;
        int p[2] = {-1, -1};
        const Operand *in[2] = {&ops[i].in0, &ops[i].in1};
        for (int q = 0; q < 2; q++)
            if (in[q]->buf >= 0) {
                auto it = prod.find(in[q]->buf);
                if (it != prod.end()) p[q] = it->second;
            }
        int g = (int)gpos.size() - 1;
        bool join = g >= 0;
        for (int q = 0; q < 2 && join; q++)
            if (p[q] >= 0 && !(p[q] < gpos[g] || group[p[q]] == g)) join = false;
        if (!join) {
            gpos.push_back(i);
            count.push_back(0);
            g = (int)gpos.size() - 1;
        }
        group[i] = g;
        count[g]++;
        for (int q = 0; q < 2; q++)
            if (p[q] >= 0 && group[p[q]] == g) level[i] = std::max(level[i], level[p[q]] + 1);
    }
    std::vector<Op> out;
    out.reserve(n);
    std::vector<int> gop(gpos.size(), -1);  // index in `out` of group g's op
    for (int i = 0; i < n; i++) {
        const int g = group[i];
        if (g < 0 || count[g] < 2) {
            out.push_back(std::move(ops[i]));
            continue;
        }
        if (gop[g] < 0) {
            Op t;
            t.kind = OP_TASKS;
            t.step = ops[i].step;
            t.dep = ops[i].dep;
            gop[g] = (int)out.size();
            out.push_back(std::move(t));
        }
        Op &t = out[gop[g]];
        t.task_levels = std::max(t.task_levels, level[i] + 1);
        t.macs += ops[i].macs;
        t.bytes += ops[i].bytes;
        t.members.push_back(std::move(ops[i]));
    }
    ops.swap(out);
}

// Compile the op lists for batch width nb.  Returns the arena size or -1 on
// a malformed input (message set).
int64_t compile(tn_plan &P, int nb) {
    P.nb = nb;
    P.prologue.clear();
    P.batch.clear();
    P.bufs.clear();
    P.extract.clear();
    const int n = P.n_tensors;
    std::unordered_set<int32_t> kept(P.open.begin(), P.open.end());
    std::unordered_map<int32_t, int> fixed_bit;  // fixed sliced label -> slice-id bit
    for (int j = 0; j < P.n_sliced; j++) {
        if (j < nb) kept.insert(P.sliced[j]);
        else fixed_bit[P.sliced[j]] = j;
    }
    std::vector<NodeRec> nodes(2 * n - 1 > 0 ? 2 * n - 1 : 1);
    // ops are first collected per step with dependency flags, buffers get
    // times afterwards
    struct PendingOp { Op op; };
    std::vector<Op> ops;  // in tree order
    auto new_buf = [&](int64_t elems) {
        Buf b;
        b.elems = elems;
        P.bufs.push_back(b);
        return (int)P.bufs.size() - 1;
    };
    // leaves
    for (int i = 0; i < n; i++) {
        NodeRec &nd = nodes[i];
        nd.leaf = i;
        std::vector<int> fpos;
        for (int32_t x : P.labels[i]) {
            if (fixed_bit.count(x)) nd.extracted = true;
            else nd.lay.push_back(x);
        }
        nd.dep = nd.extracted;
        if (nd.extracted) {
            nd.where.buf = new_buf((int64_t)1 << nd.lay.size());
            ExtractEntry e;
            std::memset(&e, 0, sizeof e);
            e.n_out = 1 << nd.lay.size();
            const int r = (int)P.labels[i].size();
            std::vector<int> fp;
            for (int a = 0; a < r; a++) {
                int32_t x = P.labels[i][a];
                auto it = fixed_bit.find(x);
                if (it == fixed_bit.end()) continue;
                e.fpos[e.nf] = r - 1 - a;
                e.sbit[e.nf] = it->second;
                fp.push_back(r - 1 - a);
                e.nf++;
            }
            std::sort(fp.begin(), fp.end());
            for (size_t q = 0; q < fp.size(); q++) e.fpos_sorted[q] = fp[q];
            // src/dst resolved later: stash leaf index / buffer id in pointers
            e.src = reinterpret_cast<const float2 *>((intptr_t)i);
            e.dst = reinterpret_cast<float2 *>((intptr_t)nd.where.buf);
            P.extract.push_back(e);
            P.extract_max_out = std::max(P.extract_max_out, e.n_out);
        } else {
            nd.where.leaf_off = P.leaf_off[i];
        }
    }
    // label sets of every node, and for each node the labels its parent step
    // contracts (shared with the sibling, not kept): a tensor-core step puts
    // those lowest in its output so that the parent's operand split (or this
    // step's planar epilogue) moves contiguous runs
    std::vector<std::unordered_set<int32_t>> lset(nodes.size());
    for (int i = 0; i < n; i++) lset[i].insert(nodes[i].lay.begin(), nodes[i].lay.end());
    std::vector<std::unordered_set<int32_t>> parentK(nodes.size());
    for (int t = 0; t < (int)P.tree.size(); t++) {
        const int ia = P.tree[t].first, ib = P.tree[t].second;
        std::unordered_set<int32_t> &o = lset[n + t];
        for (int32_t x : lset[ia])
            if (!lset[ib].count(x) || kept.count(x)) o.insert(x);
        for (int32_t x : lset[ib])
            if (!lset[ia].count(x)) o.insert(x);
        for (int32_t x : lset[ia])
            if (lset[ib].count(x) && !kept.count(x)) {
                parentK[ia].insert(x);
                parentK[ib].insert(x);
            }
    }
    // steps
    for (int t = 0; t < (int)P.tree.size(); t++) {
        const int ia = P.tree[t].first, ib = P.tree[t].second;
        NodeRec &na = nodes[ia], &nb_ = nodes[ib];
        NodeRec &nc = nodes[n + t];
        std::unordered_set<int32_t> sa(na.lay.begin(), na.lay.end()), sb(nb_.lay.begin(), nb_.lay.end());
        std::vector<int32_t> H, K;
        for (int32_t x : na.lay)
            if (sb.count(x)) (kept.count(x) ? H : K).push_back(x);
        nc.dep = na.dep || nb_.dep;
        const int ra = (int)na.lay.size(), rb = (int)nb_.lay.size();
        const bool a_big = ra >= rb;
        NodeRec &T = a_big ? na : nb_;
        NodeRec &S = a_big ? nb_ : na;
        const std::unordered_set<int32_t> &sT = a_big ? sa : sb;
        const std::unordered_set<int32_t> &sS = a_big ? sb : sa;
        std::vector<int32_t> Nl;  // free labels of S, S order
        for (int32_t x : S.lay)
            if (!sT.count(x)) Nl.push_back(x);
        std::vector<int32_t> Ml;  // free labels of T, T order
        for (int32_t x : T.lay)
            if (!sS.count(x)) Ml.push_back(x);
        const int nH = (int)H.size(), nK = (int)K.size(), nN = (int)Nl.size(), nM = (int)Ml.size();
        const double macs = std::exp2((double)(nH + nM + nK + nN));
        // a small step with enough arithmetic per T element goes to the
        // tensor cores in the split forms (the CUDA-core kernel is bound by
        // FP32 issue there, not by memory)
        const bool small_to_tc = P.opts.small_tc_bits > 0 && P.form != TN_FP32 && nK >= 3 && nN >= 3 &&
                                 nK + nN >= P.opts.small_tc_bits && (int)T.lay.size() - nK >= 16;
        if ((int)S.lay.size() <= kSmallMaxRank && nK <= 10 && nN <= 10 && nH <= kMaxHBits && !small_to_tc) {
            // ---- small step: C = T layout with K labels replaced by N labels
            Op op;
            std::memset(&op.small, 0, sizeof op.small);
            op.kind = OP_SMALL;
            op.step = t;
            op.dep = nc.dep;
            std::vector<int32_t> cl = T.lay;
            std::vector<int> kslots;
            std::unordered_set<int32_t> Kset(K.begin(), K.end());
            for (int i = 0; i < (int)cl.size(); i++)
                if (Kset.count(cl[i])) kslots.push_back(i);
            std::vector<char> del(cl.size(), 0);
            for (int i = 0; i < (int)kslots.size(); i++) {
                if (i < nN) cl[kslots[i]] = Nl[i];
                else del[kslots[i]] = 1;
            }
            std::vector<int32_t> c2;
            for (int i = nN - 1; i >= (int)kslots.size(); i--) c2.push_back(Nl[i]);
            std::reverse(c2.begin(), c2.end());
            for (int i = 0; i < (int)cl.size(); i++)
                if (!del[i]) c2.push_back(cl[i]);
            nc.lay = c2;
            if ((int)nc.lay.size() > kMaxRank || (int)T.lay.size() > kMaxRank) {
                set_error("tensor rank exceeds the kernel limit");
                return -1;
            }
            SmallArgs &s = op.small;
            s.nK = nK;
            s.nN = nN;
            s.nH = nH;
            s.s_rank = (int)S.lay.size();
            s.rows = (int64_t)1 << (T.lay.size() - nK);
            // K bits: ascending T positions
            std::vector<int> tk;
            for (int32_t x : K) tk.push_back(pos_of(T.lay, x));
            std::vector<int32_t> Ksorted = K;
            std::sort(Ksorted.begin(), Ksorted.end(),
                      [&](int32_t x, int32_t y) { return pos_of(T.lay, x) < pos_of(T.lay, y); });
            for (int j = 0; j < nK; j++) {
                s.kposT[j] = pos_of(T.lay, Ksorted[j]);
                s.kposS[j] = pos_of(S.lay, Ksorted[j]);
                s.tins[j] = s.kposT[j];
            }
            s.n_tins = nK;
            std::vector<int> cn;
            for (int j = 0; j < nN; j++) {
                s.nposC[j] = pos_of(nc.lay, Nl[j]);
                s.nposS[j] = pos_of(S.lay, Nl[j]);
                cn.push_back(s.nposC[j]);
            }
            std::sort(cn.begin(), cn.end());
            for (int j = 0; j < nN; j++) s.cins[j] = cn[j];
            s.n_cins = nN;
            for (int j = 0; j < nH; j++) {
                int pt = pos_of(T.lay, H[j]);
                int below = 0;
                for (int q = 0; q < nK; q++)
                    if (s.kposT[q] < pt) below++;
                s.hbitR[j] = pt - below;
                s.hposS[j] = pos_of(S.lay, H[j]);
            }
            if (P.opts.small_tiled >= 0) prepare_small_tiled(s);
            if (P.opts.small_tc >= 0 && small_tc_suitable(s, P.form)) s.tc_form = (int)P.form;
            op.in0 = T.where;  // T
            op.in1 = S.where;  // S
            nc.where.buf = new_buf((int64_t)1 << nc.lay.size());
            op.out = nc.where;
            op.macs = macs;
            op.bytes = 8.0 * (std::exp2((double)T.lay.size()) + std::exp2((double)S.lay.size()) +
                              std::exp2((double)nc.lay.size()));
            ops.push_back(op);
            continue;
        }
        // ---- GEMM step: A = bigger operand (rows M), B = smaller (cols N)
        NodeRec &A = T, &B = S;
        GemmArgs shape;
        std::memset(&shape, 0, sizeof shape);
        shape.H = (int64_t)1 << nH;
        shape.M = (int64_t)1 << nM;
        shape.N = (int64_t)1 << nN;
        shape.K = (int64_t)1 << nK;
        const bool use_tc = P.form != TN_FP32 && tc_gemm_suitable(shape);
        std::vector<int32_t> hord, kord, mord, nord;
        Operand wA = A.where, wB = B.where;
        std::unordered_map<int32_t, int> gA, gB;
        for (int32_t x : H) { gA[x] = 0; gB[x] = 0; }
        for (int32_t x : K) { gA[x] = 2; gB[x] = 1; }
        for (int32_t x : Ml) gA[x] = 1;
        for (int32_t x : Nl) gB[x] = 2;
        Groups GA, GB;
        if (use_tc) {
            // the split pass reads each operand in whatever label order it has
            // (a fused bit permutation), so the group orders are free.  K
            // follows the operand a tensor-core GEMM will write in planar
            // form (its lowest labels are this step's K labels), else A;
            // rows and columns put the parent step's K labels lowest.
            const NodeRec &kref = (!planar_candidate(ops, A.where) && planar_candidate(ops, B.where)) ? B : A;
            const std::unordered_set<int32_t> Kset(K.begin(), K.end());
            for (int32_t x : A.lay)
                if (gA[x] == 0) hord.push_back(x);
            for (int32_t x : kref.lay)
                if (Kset.count(x)) kord.push_back(x);
            const std::unordered_set<int32_t> &pk = parentK[n + t];
            for (int pass = 0; pass < 2; pass++) {
                for (int32_t x : Ml)
                    if ((pk.count(x) != 0) == (pass == 1)) mord.push_back(x);
                for (int32_t x : Nl)
                    if ((pk.count(x) != 0) == (pass == 1)) nord.push_back(x);
            }
        } else {
            GA = group_layout(A.lay, gA);
            GB = group_layout(B.lay, gB);
            bool permA = false, permB = false;
            if (GA.ok && GB.ok && GA.order[0] == GB.order[0] && GA.order[2] == GB.order[1]) {
            } else if (GA.ok) {
                permB = true;
            } else if (GB.ok) {
                permA = true;
            } else {
                permA = permB = true;
            }
            if (GA.ok && !permA) {
                hord = GA.order[0];
                kord = GA.order[2];
            } else if (GB.ok && !permB) {
                hord = GB.order[0];
                kord = GB.order[1];
            } else {
                for (int32_t x : A.lay)
                    if (gA[x] == 0) hord.push_back(x);
                for (int32_t x : A.lay)
                    if (gA[x] == 2) kord.push_back(x);
            }
            auto emit_permute = [&](const NodeRec &src, const std::vector<int32_t> &new_lay, Operand &dst) {
                Op op;
                op.kind = OP_PERMUTE;
                op.step = t;
                op.dep = nc.dep;
                op.bp = make_bitperm(src.lay, new_lay, 0);
                op.in0 = src.where;
                dst.buf = new_buf((int64_t)1 << new_lay.size());
                dst.leaf_off = -1;
                op.out = dst;
                op.bytes = 16.0 * std::exp2((double)new_lay.size());
                ops.push_back(op);
            };
            std::vector<int32_t> layA = A.lay, layB = B.lay;
            if (permA) {
                std::vector<int32_t> nl = hord;
                nl.insert(nl.end(), Ml.begin(), Ml.end());
                nl.insert(nl.end(), kord.begin(), kord.end());
                emit_permute(A, nl, wA);
                layA = nl;
            }
            if (permB) {
                std::vector<int32_t> nl = hord;
                nl.insert(nl.end(), kord.begin(), kord.end());
                nl.insert(nl.end(), Nl.begin(), Nl.end());
                emit_permute(B, nl, wB);
                layB = nl;
            }
            GA = group_layout(layA, gA);
            GB = group_layout(layB, gB);
            if (!GA.ok || !GB.ok || GA.order[0] != GB.order[0] || GA.order[2] != GB.order[1]) {
                set_error("internal: GEMM layout grouping failed");
                return -1;
            }
            mord = GA.order[1];
            nord = GB.order[2];
        }
        nc.lay = hord;
        nc.lay.insert(nc.lay.end(), mord.begin(), mord.end());
        nc.lay.insert(nc.lay.end(), nord.begin(), nord.end());
        if ((int)nc.lay.size() > kMaxRank) {
            set_error("tensor rank exceeds the kernel limit");
            return -1;
        }
        Op op;
        op.kind = OP_GEMM;
        std::memset(&op.tc, 0, sizeof op.tc);
        op.tc.tma_out_ok = P.opts.tc_tma_store >= 0 ? 1 : 0;
        op.step = t;
        op.dep = nc.dep;
        GemmArgs &g = op.gemm;
        g = shape;
        g.sCn = 1;
        g.sCm = (int64_t)1 << nN;
        g.sCh = (int64_t)1 << (nM + nN);
        op.macs = macs;
        if (use_tc) {
            // split both operands into hi/lo planes [q][h][row][k] (fused with
            // their permutation); the tensor-core GEMM reads the planes by TMA.
            // scaled forms (FP16S, FP16X3): a max-abs pass per operand first
            // picks its power-of-two scale, and the split writes scaled fp16
            // planes {re, im} or {re_hi, im_hi, re_lo, im_lo}
            // the 3M product (tc_products 3, hi/lo forms): six planes per
            // operand, the split modes' 3M variants
            const int products = (P.opts.tc_products == 3 && tc_form_has_3m(P.form)) ? 3 : 4;
            const int es = tc_plane_bytes(P.form), np = tc_plane_count(P.form, products);
            const bool scaled = P.form == TN_FP16S || P.form == TN_FP16X3;
            const int mode4 = P.form == TN_FP16S ? 3 : P.form == TN_FP16X3 ? 4 : (es == 2 ? 1 : 2);
            const int mode = products == 3 ? mode_to_3m(mode4) : mode4;
            op.tc.products = products;
            Operand slots;
            if (scaled) {
                // four uint32 slots: the A and B operands' plane scales (max
                // |re|, |im|, or a planar producer's bound-derived value), then
                // a planar producer's true max of each (0 otherwise)
                slots.buf = new_buf(2);
                int idx = 0;
                for (const NodeRec *src : {&A, &B}) {
                    // an operand written by a tensor-core GEMM without split K
                    // gets its max from that GEMM's epilogue
                    Op *prod = nullptr;
                    if (src->where.buf >= 0)
                        for (auto &o : ops)
                            if (o.out.buf == src->where.buf) prod = &o;
                    if (prod && prod->kind == OP_GEMM && prod->gemm_variant == 1 && prod->tc.ksplit == 1) {
                        prod->maxout = slots;
                        prod->maxout_idx = idx++;
                        continue;
                    }
                    // likewise a small step (it keeps a running max of the
                    // values it stores)
                    if (prod && prod->kind == OP_SMALL && prod->small.tiled != 3 && prod->maxout.buf < 0) {
                        prod->maxout = slots;
                        prod->maxout_idx = idx++;
                        continue;
                    }
                    Op mo;
                    mo.kind = OP_MAXABS;
                    mo.step = t;
                    mo.dep = nc.dep;
                    std::memset(&mo.mx, 0, sizeof mo.mx);
                    mo.mx.n = (int64_t)1 << src->lay.size();
                    mo.in0 = src->where;
                    mo.out = slots;
                    mo.aux_idx = idx++;
                    mo.bytes = 8.0 * (double)mo.mx.n;
                    ops.push_back(mo);
                }
            }
            int split_idx = 0;
            // planes [q][h][K_high][row][K_low]: K cut into runs of 128 bytes
            // (K_low = its lowest 6 labels for 16-bit pieces, 5 for tf32),
            // so that a TMA box of a K run over 128 rows is one contiguous
            // block of memory (long-K operands otherwise read rows of
            // 128-byte pieces scattered by the row length)
            const int klo_bits = es == 2 ? 6 : 5;
            const bool chunked = (int)kord.size() > klo_bits;
            op.tc.k_low_bits = chunked ? klo_bits : 0;
            auto emit_split = [&](const NodeRec &src, const std::vector<int32_t> &rows) {
                std::vector<int32_t> dl = hord;
                const size_t nk_hi = chunked ? kord.size() - klo_bits : 0;
                dl.insert(dl.end(), kord.begin(), kord.begin() + nk_hi);
                dl.insert(dl.end(), rows.begin(), rows.end());
                dl.insert(dl.end(), kord.begin() + nk_hi, kord.end());
                const int64_t elems = (int64_t)1 << dl.size();
                // the GEMM that wrote src splits its own output into these
                // planes when its epilogue writes can be coalesced (runs of
                // at least 64 bytes per plane).  Not for the scaled forms:
                // their plane scale is the max of the whole output, known
                // only after the producer's last tile.
                // likewise a tiled small step: its store phase writes the
                // planes in destination runs
                if (P.opts.tc_planar >= 0 && !scaled && (mode == 1 || mode == 2) && src.lay.size() == dl.size()) {
                    Op *prod = producer_of(ops, src.where);
                    if (prod && prod->kind == OP_SMALL && prod->small.tiled && !prod->small.tc_form) {
                        const int r = (int)dl.size();
                        std::vector<int> cdest(r, -1);
                        for (int q = 0; q < r; q++) {
                            const int di = pos_of(dl, src.lay[r - 1 - q]);
                            cdest[q] = di;  // pos_of gives the bit position (first label = MSB)
                        }
                        SmallArgs sa = prod->small;
                        int run_bits = -1;
                        const int why = prepare_small_planar(sa, cdest.data(), mode, elems, &run_bits);
                        prod->note = why == 0 ? "planar store" : "planar store declined: reason " + std::to_string(why) +
                                                                     ", destination run bits " + std::to_string(run_bits);
                        if (why == 0) {
                            Operand dst;
                            dst.buf = new_buf((np * elems * es + 7) / 8);
                            prod->small = sa;
                            prod->out = dst;
                            prod->bytes += (double)np * es * (double)elems - 8.0 * (double)elems;
                            split_idx++;
                            return dst;
                        }
                    }
                }
                if (P.opts.tc_planar >= 0 && planar_candidate(ops, src.where) &&
                    (!scaled || producer_of(ops, src.where)->maxout.buf >= 0)) {
                    Op *prod = producer_of(ops, src.where);
                    TcPlanarOut o;
                    const int nHp = __builtin_ctzll((uint64_t)prod->gemm.H);
                    const int nMp = __builtin_ctzll((uint64_t)prod->gemm.M);
                    const int nNp = __builtin_ctzll((uint64_t)prod->gemm.N);
                    if (make_planar(src.lay, dl, nHp, nMp, nNp, mode, es == 2 ? 5 : 4, o)) {
                        Operand dst;
                        dst.buf = new_buf((np * elems * es + 7) / 8);
                        prod->tc.out = o;
                        prod->out = dst;
                        prod->bytes += (double)np * es * (double)elems - 8.0 * (double)elems;
                        split_idx++;
                        return dst;
                    }
                }
                Op sp;
                sp.kind = OP_SPLIT;
                sp.step = t;
                sp.dep = nc.dep;
                sp.bp = make_bitperm(src.lay, dl, mode);
                sp.in0 = src.where;
                if (scaled) {
                    sp.aux = slots;
                    sp.aux_idx = split_idx;
                }
                split_idx++;
                Operand dst;
                dst.buf = new_buf((np * elems * es + 7) / 8);
                sp.out = dst;
                sp.bytes = 8.0 * (double)elems + (double)np * es * (double)elems;
                ops.push_back(sp);
                return dst;
            };
            op.in0 = emit_split(A, mord);
            op.in1 = emit_split(B, nord);
            op.gemm_variant = 1;
            op.tc.ksplit = tc_choose_ksplit(g, P.form);
            if (scaled) op.aux = slots;
            op.bytes = (double)(np * es) * (double)(g.H * (g.M + g.N) * g.K) + 8.0 * (double)(g.H * g.M * g.N);
        } else {
            g.sAh = (int64_t)1 << GA.lowpos[0];
            g.sAm = (int64_t)1 << GA.lowpos[1];
            g.sAk = (int64_t)1 << GA.lowpos[2];
            g.sBh = (int64_t)1 << GB.lowpos[0];
            g.sBk = (int64_t)1 << GB.lowpos[1];
            g.sBn = (int64_t)1 << GB.lowpos[2];
            op.in0 = wA;
            op.in1 = wB;
            op.gemm_variant = 0;
            op.bytes = 8.0 * (std::exp2((double)A.lay.size()) + std::exp2((double)B.lay.size()) +
                              std::exp2((double)nc.lay.size()));
        }
        nc.where.buf = new_buf((int64_t)1 << nc.lay.size());
        op.out = nc.where;
        ops.push_back(op);
    }
    // root
    const int root_id = P.tree.empty() ? 0 : n + (int)P.tree.size() - 1;
    NodeRec &rt = nodes[root_id];
    {
        std::set<int32_t> want(P.open.begin(), P.open.end());
        for (int j = 0; j < nb; j++) want.insert(P.sliced[j]);
        std::set<int32_t> have(rt.lay.begin(), rt.lay.end());
        if (want != have) {
            set_error("root labels differ from open + batch labels (disconnected or malformed tree?)");
            return -1;
        }
    }
    std::memset(&P.accum, 0, sizeof P.accum);
    P.accum.n_open = P.n_open;
    P.accum.n_batch = nb;
    for (int j = 0; j < P.n_open; j++) P.accum.opos[j] = pos_of(rt.lay, P.open[P.n_open - 1 - j]);
    for (int j = 0; j < nb; j++) P.accum.bpos[j] = pos_of(rt.lay, P.sliced[j]);
    P.root = rt.where;
    const bool root_dep = rt.dep;

    // split into prologue (slice-invariant) and per-block ops; the tiny
    // small steps of each become tasks of persistent launches; timeline
    for (auto &op : ops) (op.dep ? P.batch : P.prologue).push_back(op);
    const int task_bits = P.opts.small_tasks == 0 ? kDefaultTaskBits : P.opts.small_tasks;
    if (task_bits > 0) {
        group_tasks(P.prologue, task_bits);
        group_tasks(P.batch, task_bits);
    }
    const int T_pro = (int)P.prologue.size();
    const int T_ext = T_pro;                       // extraction at the start of a block
    const int T_acc = T_pro + 1 + (int)P.batch.size();
    const int T_end = T_acc;
    // producer / consumer times per buffer
    std::vector<int> first(P.bufs.size(), INT32_MAX), last(P.bufs.size(), -1);
    auto touch = [&](const Operand &w, int time) {
        if (w.buf < 0) return;
        first[w.buf] = std::min(first[w.buf], time);
        last[w.buf] = std::max(last[w.buf], time);
    };
    std::vector<char> buf_dep(P.bufs.size(), 0), buf_pro(P.bufs.size(), 0);
    for (auto &e : P.extract) {
        int b = (int)(intptr_t)e.dst;
        touch(Operand{b, -1}, T_ext);
        buf_dep[b] = 1;
    }
    for (int i = 0; i < T_pro; i++)
        for_each_operand(P.prologue[i], [&](const Operand &w, bool written) {
            touch(w, i);
            if (written && w.buf >= 0) buf_pro[w.buf] = 1;
        });
    for (int i = 0; i < (int)P.batch.size(); i++) {
        const int time = T_pro + 1 + i;
        for_each_operand(P.batch[i], [&](const Operand &w, bool written) {
            touch(w, time);
            if (written && w.buf >= 0) buf_dep[w.buf] = 1;
        });
    }
    touch(P.root, T_acc);
    // an invariant buffer read inside the block loop lives to the loop's end
    for (size_t b = 0; b < P.bufs.size(); b++) {
        // (also a max-abs slot pair written by a prologue GEMM for one operand
        // and inside the block for the other: the prologue's value must
        // survive every block)
        if ((!buf_dep[b] || buf_pro[b]) && last[b] > T_pro) last[b] = T_end;
        if (first[b] == INT32_MAX) {  // never used (a GEMM output replaced by its planar form)
            first[b] = 0;
            last[b] = 0;
            P.bufs[b].elems = 0;
        }
        P.bufs[b].t0 = first[b];
        P.bufs[b].t1 = last[b];
    }
    (void)root_dep;
    // first-fit placement, largest first
    std::vector<int> idx(P.bufs.size());
    for (size_t i = 0; i < idx.size(); i++) idx[i] = (int)i;
    std::sort(idx.begin(), idx.end(), [&](int x, int y) {
        if (P.bufs[x].elems != P.bufs[y].elems) return P.bufs[x].elems > P.bufs[y].elems;
        return x < y;
    });
    std::vector<int> placed;
    int64_t arena = 0;
    for (int bi : idx) {
        Buf &b = P.bufs[bi];
        const int64_t bytes = ((b.elems * 8 + 255) / 256) * 256;
        std::vector<std::pair<int64_t, int64_t>> busy;
        for (int pj : placed) {
            const Buf &o = P.bufs[pj];
            if (o.t1 < b.t0 || b.t1 < o.t0) continue;
            busy.push_back({o.off, o.off + ((o.elems * 8 + 255) / 256) * 256});
        }
        std::sort(busy.begin(), busy.end());
        int64_t off = 0;
        for (auto &iv : busy) {
            if (off + bytes <= iv.first) break;
            off = std::max(off, iv.second);
        }
        b.off = off;
        arena = std::max(arena, off + bytes);
        placed.push_back(bi);
    }
    P.macs_batch = P.macs_prologue = P.bytes_batch = P.bytes_prologue = 0;
    for (auto &op : P.prologue) { P.macs_prologue += op.macs; P.bytes_prologue += op.bytes; }
    for (auto &op : P.batch) { P.macs_batch += op.macs; P.bytes_batch += op.bytes; }
    P.launches_prologue = (int)P.prologue.size();
    P.launches_batch = (int)P.batch.size() + (P.extract.empty() ? 0 : 1) + 1;
    return arena;
}

float2 *resolve(tn_plan &P, const Operand &w) {
    if (w.buf >= 0) return reinterpret_cast<float2 *>(P.d_arena + P.bufs[w.buf].off);
    return P.d_leaves + w.leaf_off;
}

// The device-side table of an OP_TASKS op (host copy): one SmallTask per
// member with resolved pointers, units of up to kTaskUnitItems items, and
// each member's producers among the earlier members.
void build_task_table(Op &op) {
    op.tasks.clear();
    op.unit_task.clear();
    std::unordered_map<int, int> prod;  // arena buffer -> member
    for (int i = 0; i < (int)op.members.size(); i++) {
        const Op &m = op.members[i];
        SmallTask t = make_small_task(m.small);
        const int nc_bits = t.nc == 32 ? 5 : (t.nc == 16 ? 4 : 3);
        const int64_t items = m.small.rows << (m.small.nN > nc_bits ? m.small.nN - nc_bits : 0);
        t.first_unit = (int)op.unit_task.size();
        t.n_units = (int)((items + kTaskUnitItems - 1) / kTaskUnitItems);
        for (const Operand *w : {&m.in0, &m.in1})
            if (w->buf >= 0) {
                auto it = prod.find(w->buf);
                if (it != prod.end() && t.n_deps < 2 && (t.n_deps == 0 || t.dep[0] != it->second))
                    t.dep[t.n_deps++] = it->second;
            }
        for (int u = 0; u < t.n_units; u++) op.unit_task.push_back(i);
        op.tasks.push_back(t);
        if (m.out.buf >= 0) prod[m.out.buf] = i;
    }
}

void resolve_all(tn_plan &P) {
    auto fix = [&](Op &op) {
        switch (op.kind) {
        case OP_TASKS:
            for (Op &m : op.members) {
                m.small.T = resolve(P, m.in0);
                m.small.S = resolve(P, m.in1);
                m.small.C = resolve(P, m.out);
            }
            build_task_table(op);
            break;
        case OP_SMALL:
            op.small.T = resolve(P, op.in0);
            op.small.S = resolve(P, op.in1);
            op.small.C = resolve(P, op.out);
            op.small.max_slot = op.maxout.buf >= 0
                                    ? reinterpret_cast<unsigned *>(resolve(P, op.maxout)) + op.maxout_idx
                                    : nullptr;
            break;
        case OP_PERMUTE:
        case OP_SPLIT:
            op.bp.in = resolve(P, op.in0);
            op.bp.out = resolve(P, op.out);
            if (op.aux.buf >= 0) op.bp.scale = reinterpret_cast<const unsigned *>(resolve(P, op.aux)) + op.aux_idx;
            break;
        case OP_MAXABS:
            op.mx.in = resolve(P, op.in0);
            op.mx.slot = reinterpret_cast<unsigned *>(resolve(P, op.out)) + op.aux_idx;
            op.mx.companion = op.mx.slot + 2;  // the operand's true-max slot
            break;
        case OP_GEMM:
            if (op.gemm_variant == 1) {
                op.tc.a = op.gemm;
                op.tc.a.C = resolve(P, op.out);
                op.tc.form = P.form;
                op.tc.planesA = resolve(P, op.in0);
                op.tc.planesB = resolve(P, op.in1);
                if (op.tc.ksplit < 1) op.tc.ksplit = 1;
                op.tc.chunk_bytes = P.opts.tc_chunk_bytes;
                op.tc.flush_bytes = P.opts.tc_flush_bytes;
                op.tc.scales = op.aux.buf >= 0 ? reinterpret_cast<const unsigned *>(resolve(P, op.aux)) : nullptr;
                if (op.tc.out.mode != 0) op.tc.out.planes = resolve(P, op.out);
                op.tc.max_slot = op.maxout.buf >= 0
                                     ? reinterpret_cast<unsigned *>(resolve(P, op.maxout)) + op.maxout_idx
                                     : nullptr;
            } else {
                op.gemm.A = resolve(P, op.in0);
                op.gemm.B = resolve(P, op.in1);
                op.gemm.C = resolve(P, op.out);
            }
            break;
        }
    };
    for (auto &op : P.prologue) fix(op);
    for (auto &op : P.batch) fix(op);

    for (auto &e : P.extract) {
        int leaf = (int)(intptr_t)e.src;
        int buf = (int)(intptr_t)e.dst;
        e.src = P.d_leaves + P.leaf_off[leaf];
        e.dst = reinterpret_cast<float2 *>(P.d_arena + P.bufs[buf].off);
    }
    P.accum.R = resolve(P, P.root);
}

cudaError_t run_op(const tn_plan &P, const Op &op, cudaStream_t s) {
    switch (op.kind) {
    case OP_SMALL:
        if (op.small.tc_form) {
            // T not 16-byte aligned (a leaf at an odd offset): the CUDA-core kernel
            const cudaError_t e = launch_small_tc(op.small, (tn_form)op.small.tc_form, s);
            if (e != cudaErrorMisalignedAddress) return e;
        }
        return launch_small(op.small, s);
    case OP_PERMUTE: return launch_bitperm(op.bp, s);
    case OP_GEMM:
        if (op.gemm_variant == 1) return launch_gemm_tc(op.tc, s);
        return launch_gemm_f32(op.gemm, s);
    case OP_SPLIT: return launch_bitperm(op.bp, s);
    case OP_MAXABS: return launch_maxabs(op.mx, s);
    case OP_TASKS:
        return launch_small_tasks(op.d_tasks, op.d_unit_task, (int)op.unit_task.size(), op.d_ctr,
                                  (int)op.tasks.size(), s);
    }
    return cudaErrorInvalidValue;
}

// reads and clears the error words of the bounded device waits (tensor-core
// pipeline, task dependencies); synchronises the stream
bool device_wait_error(cudaStream_t s) {
    const int a = tc_read_error(s);
    const int b = small_task_read_error(s);
    return a != 0 || b != 0;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(TN_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

}  // namespace tn

namespace tn {
namespace {

inline float l2f(double x) { return (float)(std::log2(x + 1.0) / 32.0); }

// time per dependency level of a task launch (wait, stage S, compute, release)
constexpr double kTaskLevelMs = 3.0e-3;

// Roofline time of one step in ms: the larger of its algorithmic bytes over
// HBM bandwidth and its arithmetic over the peak of the unit that runs it,
// plus a launch floor.  Nominal GB300 figures: 7 TB/s HBM3e, 80 TFLOP/s FP32
// FMA (152 SMs x 128 lanes x 2 x 2.07 GHz), 2.25 PFLOP/s dense f16/bf16 and
// half of that for tf32 on the tensor cores.  A tensor-core complex MAC
// issues 24 flops in the hi/lo forms (4 real products x 3 piece products) and
// 8 in FP16S.  The cost model learns log2(measured / this), which varies far
// less across sizes than the time itself and so extrapolates to steps larger
// than the ones it was trained on.
double roofline_ms(const Op &op, tn_form form) {
    const double hbm = 7.0e12, fp32 = 80.0e12, floor_ms = 2.0e-3;
    double flops = 0.0, peak = fp32;
    if (op.kind == OP_TASKS) {
        // one launch; the chain of members that feed each other runs one
        // dependency wait (a few microseconds) per link
        const double t = std::max(op.bytes / hbm, 8.0 * op.macs / fp32) * 1e3;
        return t + floor_ms + kTaskLevelMs * (op.task_levels - 1);
    }
    if (op.kind == OP_SMALL && op.small.tc_form) {
        flops = 24.0 * op.macs;
        peak = form == TN_TF32X3 ? 1.125e15 : 2.25e15;
    } else if (op.kind == OP_SMALL || (op.kind == OP_GEMM && op.gemm_variant != 1)) {
        flops = 8.0 * op.macs;
    } else if (op.kind == OP_GEMM) {
        flops = (form == TN_FP16S ? 8.0 : 24.0) * op.macs;
        peak = form == TN_TF32X3 ? 1.125e15 : 2.25e15;
    }
    const double t = std::max(op.bytes / hbm, flops / peak) * 1e3;
    return t + floor_ms;
}

// Expected time of one step in ms, for the order search's time objective:
// the roofline time, but a tensor-core GEMM takes at least its output
// elements over the rate its epilogue writes them.  Measured on GB300 over
// the short-K GEMMs of the 53-qubit 14-cycle step: about 2.2e11 elements/s
// when the epilogue writes the next step's split planes, about 4e11 when it
// writes complex64 (no split).  Short-K GEMMs with large outputs are bound
// by this, not by the tensor cores or HBM.
double expected_ms(const Op &op, tn_form form) {
    double t = roofline_ms(op, form);
    if (op.kind == OP_GEMM && op.gemm_variant == 1) {
        const double out = (double)op.gemm.H * (double)op.gemm.M * (double)op.gemm.N;
        const double rate = op.tc.out.mode != 0 ? 2.2e11 : 4.0e11;
        t = std::max(t, out / rate * 1e3 + 2.0e-3);
    }
    return t;
}

// 16 step features (see tn_plan_op_features in tn.h)
void op_features(const Op &op, tn_form form, float *f) {
    for (int i = 0; i < kCostFeatures; i++) f[i] = 0.f;
    double sh[4] = {0, 0, 0, 0}, units = 1, ksplit = 1;
    int kind = 0;
    switch (op.kind) {
    case OP_TASKS:  // many small steps: the small-step kind, units of all members
        kind = 0;
        sh[0] = (double)op.members.size();
        sh[1] = (double)op.task_levels;
        units = 0;
        for (const Op &m : op.members) units += (double)m.small.rows;
        break;
    case OP_SMALL: {
        kind = 0;
        const double nc = (1 << op.small.nN) <= 32 ? 1.0 : (double)((1 << op.small.nN) / 32);
        sh[0] = std::exp2(op.small.nH); sh[1] = (double)op.small.rows;
        sh[2] = std::exp2(op.small.nN); sh[3] = std::exp2(op.small.nK);
        units = (double)op.small.rows * nc;
        break;
    }
    case OP_PERMUTE:
        kind = 1;
        sh[1] = (double)op.bp.plane_stride;
        units = (double)op.bp.plane_stride;
        break;
    case OP_GEMM:
        kind = op.gemm_variant == 1 ? 3 : 2;
        sh[0] = (double)op.gemm.H; sh[1] = (double)op.gemm.M; sh[2] = (double)op.gemm.N; sh[3] = (double)op.gemm.K;
        if (op.gemm_variant == 1) {
            ksplit = op.tc.ksplit > 0 ? op.tc.ksplit : 1;
            units = std::ceil(sh[1] / 128.0) * std::ceil(sh[2] / 64.0) * sh[0] * ksplit;
        } else {
            units = std::ceil(sh[1] / 64.0) * std::ceil(sh[2] / 64.0) * sh[0];
        }
        break;
    case OP_SPLIT:
        kind = 4;
        sh[1] = (double)op.bp.plane_stride;
        units = (double)op.bp.plane_stride;
        break;
    case OP_MAXABS:  // a read-only bandwidth pass, closest to a permute
        kind = 1;
        sh[1] = (double)op.mx.n;
        units = (double)op.mx.n;
        break;
    }
    f[kind] = 1.f;
    f[5] = l2f(op.macs);
    f[6] = l2f(op.bytes);
    for (int q = 0; q < 4; q++) f[7 + q] = l2f(sh[q]);
    const bool tc = (op.kind == OP_GEMM && op.gemm_variant == 1) || op.kind == OP_SPLIT || op.kind == OP_MAXABS;
    f[11] = (tc && form == TN_TF32X3) ? 1.f : 0.f;
    f[12] = (tc && form == TN_BF16X3) ? 1.f : 0.f;
    f[13] = l2f(units);
    f[14] = (float)(std::log2(roofline_ms(op, form)) / kRoofFeatureScale);
    f[15] = 1.f;
}

}  // namespace

int search_ranked(const std::vector<std::vector<int32_t>> &labels, const std::vector<int32_t> &open,
                  const tn_search_opts &opts, SearchResult &out) {
    if (!opts.cost_model || opts.candidates <= 1) return search_order(labels, open, opts, out);
    std::vector<SearchResult> cands;
    int rc = search_order_top(labels, open, opts, opts.candidates, cands);
    if (rc) return rc;
    std::vector<double> pred;
    int best = 0;
    rc = rank_candidates(labels, open, cands, opts, pred, best);
    if (rc) return rc;
    out = cands[best];
    return TN_OK;
}

int rank_candidates(const std::vector<std::vector<int32_t>> &labels, const std::vector<int32_t> &open,
                    const std::vector<SearchResult> &cands, const tn_search_opts &opts, std::vector<double> &pred_ms,
                    int &best) {
    best = 0;
    pred_ms.assign(cands.size(), 0.0);
    if (!opts.cost_model || cands.empty()) return TN_OK;
    const tn_form form = (opts.rank_form >= TN_FP32 && opts.rank_form <= TN_FP16X3) ? (tn_form)opts.rank_form : TN_FP32;
    std::vector<float> X;
    struct Span { size_t pro0, pro1, bat0, bat1; double blocks; };
    std::vector<Span> spans;
    for (const auto &c : cands) {
        tn_plan P;
        P.form = form;
        P.n_tensors = (int)labels.size();
        P.labels = labels;
        P.open = open;
        P.n_open = (int)open.size();
        P.sliced = c.sliced;
        P.n_sliced = (int)c.sliced.size();
        P.tree = c.tree;
        P.leaf_off.resize(labels.size());
        int64_t off = 0;
        for (size_t i = 0; i < labels.size(); i++) {
            P.leaf_off[i] = off;
            off += (int64_t)1 << labels[i].size();
        }
        int nb = P.n_sliced;
        if (opts.rank_batch_log2 >= 0) nb = std::min(nb, (int)opts.rank_batch_log2);
        if (compile(P, nb) < 0) return TN_ERR_ARG;
        Span sp;
        float f[kCostFeatures];
        sp.pro0 = X.size() / kCostFeatures;
        for (const auto &op : P.prologue) {
            op_features(op, form, f);
            X.insert(X.end(), f, f + kCostFeatures);
        }
        sp.pro1 = sp.bat0 = X.size() / kCostFeatures;
        for (const auto &op : P.batch) {
            op_features(op, form, f);
            X.insert(X.end(), f, f + kCostFeatures);
        }
        sp.bat1 = X.size() / kCostFeatures;
        sp.blocks = std::exp2((double)(P.n_sliced - nb));
        spans.push_back(sp);
    }
    std::vector<float> Y;
    int rc = cost_predict_host(opts.cost_model, X, Y);
    if (rc) return rc;
    for (size_t i = 0; i < cands.size(); i++) {
        double t = 0;
        // the model's output is log2(time / roofline time); feature 14 holds
        // log2(roofline time) / kRoofFeatureScale
        auto step_ms = [&](size_t r) {
            return std::exp2((double)Y[r] + kRoofFeatureScale * (double)X[r * kCostFeatures + 14]);
        };
        for (size_t r = spans[i].pro0; r < spans[i].pro1; r++) t += step_ms(r);
        double tb = 0;
        for (size_t r = spans[i].bat0; r < spans[i].bat1; r++) tb += step_ms(r);
        pred_ms[i] = t + spans[i].blocks * tb;
        if (pred_ms[i] < pred_ms[best]) best = (int)i;
    }
    return TN_OK;
}

}  // namespace tn

using namespace tn;

namespace tn {

// Roofline time of a compiled plan, for all 2^n_sliced slices: every op at
// roofline_ms (bytes over HBM bandwidth or flops over its unit's peak, plus
// a launch floor), the slice-invariant prologue once and the per-block body
// once per block.  The batch width is batch_log2 when >= 0 (capped at
// n_sliced), else the largest whose arena and leaves fit `budget` bytes, as
// tn_plan_create chooses it (0 when none fits).  Host only.
int plan_roofline(tn_plan &P, int batch_log2, double budget, int64_t leaf_bytes, double &ms, int &nb_out,
                  int64_t &arena_out, double *pro_out = nullptr, double *body_out = nullptr, bool expected = false) {
    int nb = batch_log2 >= 0 ? std::min(batch_log2, P.n_sliced) : P.n_sliced;
    int64_t arena = compile(P, nb);
    if (arena < 0) return TN_ERR_ARG;
    if (batch_log2 < 0 && (double)(arena + leaf_bytes) > budget && nb > 0) {
        // the arena grows with the batch width: bisect for the largest fit
        int lo = 0, hi = nb - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            const int64_t a = compile(P, mid);
            if (a < 0) return TN_ERR_ARG;
            if ((double)(a + leaf_bytes) <= budget) lo = mid; else hi = mid - 1;
        }
        nb = lo;
        arena = compile(P, nb);
        if (arena < 0) return TN_ERR_ARG;
    }
    double pro = 0, body = 0;
    for (const auto &op : P.prologue) pro += expected ? expected_ms(op, P.form) : roofline_ms(op, P.form);
    for (const auto &op : P.batch) body += expected ? expected_ms(op, P.form) : roofline_ms(op, P.form);
    ms = pro + std::exp2((double)(P.n_sliced - nb)) * body;
    nb_out = nb;
    arena_out = arena;
    if (pro_out) *pro_out = pro;
    if (body_out) *body_out = body;
    return TN_OK;
}

double tree_roofline_ms(const std::vector<std::vector<int32_t>> &labels, const std::vector<int32_t> &open,
                        const Tree &tree, const std::vector<int32_t> &sliced, tn_form form, int batch_log2,
                        double budget, bool expected) {
    tn_plan P;
    P.form = form;
    P.n_tensors = (int)labels.size();
    P.labels = labels;
    P.open = open;
    P.n_open = (int)open.size();
    P.sliced = sliced;
    P.n_sliced = (int)sliced.size();
    P.tree = tree;
    P.leaf_off.resize(labels.size());
    int64_t off = 0;
    for (size_t i = 0; i < labels.size(); i++) {
        P.leaf_off[i] = off;
        off += (int64_t)1 << labels[i].size();
    }
    double ms = -1;
    int nb = 0;
    int64_t arena = 0;
    if (plan_roofline(P, batch_log2, budget, off * 8, ms, nb, arena, nullptr, nullptr, expected)) return -1.0;
    return ms;
}

}  // namespace tn

namespace tn {

// The host half of plan creation (no CUDA call): checks the network, the
// open and sliced labels and the tree, and copies them into P; *total_elems
// receives the leaves' element count.
int plan_host_setup(tn_plan &P, int n_tensors, const int32_t *ranks, const int32_t *labels, int n_labels,
                    const int32_t *bond_dims, int n_open, const int32_t *open_labels, int n_sliced,
                    const int32_t *sliced_labels, int n_steps, const int32_t *tree, int64_t *total_elems) {
    if (n_tensors <= 0 || !ranks) return fail(TN_ERR_ARG, "need at least one tensor");
    if (n_open < 0 || n_open > kMaxRank || (n_open > 0 && !open_labels)) return fail(TN_ERR_ARG, "bad open labels");
    if (n_sliced < 0 || n_sliced > 62 || (n_sliced > 0 && !sliced_labels)) return fail(TN_ERR_ARG, "bad sliced labels");
    if (n_steps != n_tensors - 1 || (n_steps > 0 && !tree)) return fail(TN_ERR_ARG, "tree must have n_tensors - 1 steps");
    P.n_tensors = n_tensors;
    P.n_open = n_open;
    P.n_sliced = n_sliced;
    P.open.assign(open_labels, open_labels + n_open);
    P.sliced.assign(sliced_labels, sliced_labels + n_sliced);
    // labels: validity
    std::unordered_map<int32_t, int> count;
    size_t off = 0;
    int64_t total = 0;
    P.labels.resize(n_tensors);
    P.leaf_off.resize(n_tensors);
    for (int i = 0; i < n_tensors; i++) {
        if (ranks[i] < 0 || ranks[i] > 30) return fail(TN_ERR_ARG, "tensor rank out of range [0, 30]");
        P.labels[i].assign(labels + off, labels + off + ranks[i]);
        off += ranks[i];
        std::unordered_set<int32_t> seen;
        for (int32_t x : P.labels[i]) {
            if (x < 0) return fail(TN_ERR_ARG, "negative label");
            if (n_labels > 0 && x >= n_labels) return fail(TN_ERR_ARG, "label >= n_labels");
            if (bond_dims && bond_dims[x] != 2) return fail(TN_ERR_ARG, "only bond dimension 2 is supported");
            if (!seen.insert(x).second) return fail(TN_ERR_ARG, "label repeated within a tensor");
            count[x]++;
        }
        P.leaf_off[i] = total;
        total += (int64_t)1 << ranks[i];
    }
    std::unordered_set<int32_t> open_set(P.open.begin(), P.open.end());
    if ((int)open_set.size() != n_open) return fail(TN_ERR_ARG, "open label repeated");
    for (auto &kv : count) {
        if (kv.second > 2) return fail(TN_ERR_ARG, "label held by more than two tensors");
        if (kv.second == 1 && !open_set.count(kv.first)) return fail(TN_ERR_ARG, "label held by one tensor must be open");
        if (kv.second == 2 && open_set.count(kv.first)) return fail(TN_ERR_ARG, "open label held by two tensors");
    }
    for (int32_t x : P.open)
        if (!count.count(x)) return fail(TN_ERR_ARG, "open label held by no tensor");
    std::unordered_set<int32_t> sl;
    for (int32_t x : P.sliced) {
        if (open_set.count(x)) return fail(TN_ERR_ARG, "a sliced label cannot be open");
        if (!count.count(x)) return fail(TN_ERR_ARG, "sliced label held by no tensor");
        if (!sl.insert(x).second) return fail(TN_ERR_ARG, "sliced label repeated");
    }
    P.tree.resize(n_steps);
    std::vector<char> used(2 * n_tensors, 0);
    for (int t = 0; t < n_steps; t++) {
        int a = tree[2 * t], b = tree[2 * t + 1];
        if (a < 0 || b < 0 || a >= n_tensors + t || b >= n_tensors + t || a == b || used[a] || used[b])
            return fail(TN_ERR_ARG, "tree: bad or reused node id");
        used[a] = used[b] = 1;
        P.tree[t] = {a, b};
    }
    *total_elems = total;
    return TN_OK;
}

}  // namespace tn

extern "C" int tn_plan_create(tn_plan_t *out, int n_tensors, const int32_t *ranks, const int32_t *labels,
                              const float *data, int n_labels, const int32_t *bond_dims, int n_open,
                              const int32_t *open_labels, int n_sliced, const int32_t *sliced_labels,
                              int n_steps, const int32_t *tree, tn_form form, const tn_plan_opts *opts) {
    if (!out) return fail(TN_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (form < TN_FP32 || form > TN_FP16X3) return fail(TN_ERR_ARG, "unknown form");
    if (form != TN_FP32 && !tc_form_available(form))
        return fail(TN_ERR_ARG, "this arithmetic form is not compiled into this library");
    if (opts && opts->tc_products != 0 && opts->tc_products != 4 && opts->tc_products != 3)
        return fail(TN_ERR_ARG, "tc_products must be 0, 3 or 4");
    std::unique_ptr<tn_plan> P(new tn_plan());
    P->form = form;
    if (opts) P->opts = *opts;
    else {
        std::memset(&P->opts, 0, sizeof P->opts);
        P->opts.batch_log2 = -1;
    }
    int64_t total = 0;
    int rc0 = plan_host_setup(*P, n_tensors, ranks, labels, n_labels, bond_dims, n_open, open_labels, n_sliced,
                              sliced_labels, n_steps, tree, &total);
    if (rc0) return rc0;
    // device
    if (cudaGetDevice(&P->device) != cudaSuccess) return fail(TN_ERR_CUDA, "no CUDA device");
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemGetInfo");
    const int64_t budget = P->opts.mem_budget > 0 ? P->opts.mem_budget : (int64_t)(0.6 * (double)free_b);
    const int64_t leaf_bytes = total * 8;
    int nb_max = n_sliced;
    if (P->opts.batch_log2 >= 0) nb_max = std::min(nb_max, (int)P->opts.batch_log2);
    int64_t arena = -1;
    int nb = nb_max;
    for (; nb >= 0; nb--) {
        arena = compile(*P, nb);
        if (arena < 0) return TN_ERR_ARG;
        if (arena + leaf_bytes <= budget) break;
    }
    if (nb < 0) return fail(TN_ERR_OOM, "the plan does not fit the memory budget even without batching");
    P->arena_bytes = arena;
    P->leaf_bytes = leaf_bytes;
    e = cudaMalloc(&P->d_leaves, std::max<int64_t>(leaf_bytes, 16));
    if (e != cudaSuccess) return fail(TN_ERR_OOM, "cudaMalloc leaves");
    e = data ? cudaMemcpy(P->d_leaves, data, leaf_bytes, cudaMemcpyHostToDevice)
             : cudaMemset(P->d_leaves, 0, std::max<int64_t>(leaf_bytes, 16));  // leaves set later
    if (e != cudaSuccess) return cuda_fail(e, "copy leaves");
    e = cudaMalloc(&P->d_arena, std::max<int64_t>(arena, 256));
    if (e != cudaSuccess) return fail(TN_ERR_OOM, "cudaMalloc arena");
    resolve_all(*P);
    for (auto *ops : {&P->prologue, &P->batch})
        for (auto &op : *ops)
            if (op.kind == OP_GEMM && op.gemm_variant == 1 && !tc_prepare(op.tc))
                return fail(TN_ERR_CUDA, "TMA descriptor encoding failed");
    // task tables: tasks, unit -> task map and counters in one allocation
    for (auto *ops : {&P->prologue, &P->batch})
        for (auto &op : *ops) {
            if (op.kind != OP_TASKS) continue;
            const size_t tb = sizeof(SmallTask) * op.tasks.size();
            const size_t ub = sizeof(int) * op.unit_task.size();
            const size_t cb = sizeof(int) * (op.tasks.size() + 1);
            char *mem = nullptr;
            e = cudaMalloc(&mem, tb + ub + cb);
            if (e != cudaSuccess) return fail(TN_ERR_OOM, "cudaMalloc task table");
            P->task_mem.push_back(mem);
            op.d_tasks = reinterpret_cast<SmallTask *>(mem);
            op.d_unit_task = reinterpret_cast<int *>(mem + tb);
            op.d_ctr = reinterpret_cast<int *>(mem + tb + ub);
            e = cudaMemcpy(op.d_tasks, op.tasks.data(), tb, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(op.d_unit_task, op.unit_task.data(), ub, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cuda_fail(e, "copy task table");
        }
    if (!P->extract.empty()) {
        e = cudaMalloc(&P->d_extract, sizeof(ExtractEntry) * P->extract.size());
        if (e != cudaSuccess) return fail(TN_ERR_OOM, "cudaMalloc extract table");
        e = cudaMemcpy(P->d_extract, P->extract.data(), sizeof(ExtractEntry) * P->extract.size(),
                       cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "copy extract table");
    }
    *out = P.release();
    return TN_OK;
}

namespace tn {
namespace {

// rows: prologue ops, extract, batch ops, accumulate
tn_plan::ProfRow prof_row(int phase, int idx, const Op &op) {
    tn_plan::ProfRow r{phase, idx, (int)op.kind, op.step, 0.0, 0, op.macs, op.bytes, {0, 0, 0, 0}};
    if (op.kind == OP_GEMM) {
        r.shape[0] = (double)op.gemm.H; r.shape[1] = (double)op.gemm.M;
        r.shape[2] = (double)op.gemm.N; r.shape[3] = (double)op.gemm.K;
    } else if (op.kind == OP_SPLIT) {
        r.shape[1] = (double)op.bp.plane_stride;
    } else if (op.kind == OP_SMALL) {
        r.shape[0] = (double)op.small.nH; r.shape[1] = (double)op.small.rows;
        r.shape[2] = (double)(1 << op.small.nN); r.shape[3] = (double)(1 << op.small.nK);
    } else if (op.kind == OP_PERMUTE) {
        r.shape[1] = (double)op.bp.plane_stride;
    } else if (op.kind == OP_MAXABS) {
        r.shape[1] = (double)op.mx.n;
    } else if (op.kind == OP_TASKS) {
        r.shape[0] = (double)op.members.size();
        r.shape[1] = (double)op.unit_task.size();
        r.shape[2] = (double)op.task_levels;
    }
    return r;
}

void prof_init(tn_plan &P) {
    if (!P.prof.empty()) return;
    int idx = 0;
    for (auto &op : P.prologue) P.prof.push_back(prof_row(0, idx++, op));
    P.prof.push_back({1, 0, 3, -1, 0.0, 0, 0.0, 0.0, {0, 0, 0, 0}});
    idx = 0;
    for (auto &op : P.batch) P.prof.push_back(prof_row(1, idx++, op));
    P.prof.push_back({1, 0, 4, -1, 0.0, 0, 0.0, 0.0, {0, 0, 0, 0}});
    P.prof_ev.resize(2 * P.prof.size());
    for (auto &ev : P.prof_ev) cudaEventCreate(&ev);
}

// Capture ops into an instantiated graph on a private stream (the ops' own
// launch-time setup already ran in an eager call).
// Capture an op list as a graph whose edges are the ops' real dependencies:
// op i follows op j < i when j writes arena bytes that i reads or writes, or
// reads bytes that i writes (buffers share arena space once their lives end).
// Independent ops, such as the small steps of separate subtrees, land on
// different streams of the capture and overlap when the graph runs.
cudaError_t capture_ops(const tn_plan &P, const std::vector<Op> &ops, cudaGraphExec_t *out) {
    *out = nullptr;
    if (ops.empty()) return cudaSuccess;
    const int n = (int)ops.size();
    struct Rg { int64_t lo, hi; };
    auto range = [&](const Operand &w) -> Rg {
        if (w.buf < 0) return {0, 0};
        const Buf &b = P.bufs[w.buf];
        return {b.off, b.off + b.elems * 8};
    };
    auto hit = [](const Rg &a, const Rg &b) { return a.lo < a.hi && b.lo < b.hi && a.lo < b.hi && b.lo < a.hi; };
    std::vector<std::vector<Rg>> rd(n), wr(n);
    for (int i = 0; i < n; i++)
        for_each_operand(ops[i], [&](const Operand &w, bool written) {
            const Rg r = range(w);
            if (r.lo < r.hi) (written ? wr[i] : rd[i]).push_back(r);
        });
    std::vector<std::vector<int>> deps(n);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < i; j++) {
            bool d = false;
            for (const Rg &w : wr[j]) {
                for (const Rg &r : rd[i]) d = d || hit(w, r);
                for (const Rg &w2 : wr[i]) d = d || hit(w, w2);
            }
            for (const Rg &r : rd[j])
                for (const Rg &w2 : wr[i]) d = d || hit(r, w2);
            if (d) deps[i].push_back(j);
        }
    constexpr int kMaxBranches = 16;
    const int kBranches = P.opts.graph_branches > 0 ? std::min(P.opts.graph_branches, kMaxBranches) : 4;
    cudaStream_t cs, br[kMaxBranches];
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    int made = 0;
    for (; made < kBranches && e == cudaSuccess; made++) e = cudaStreamCreateWithFlags(&br[made], cudaStreamNonBlocking);
    if (e != cudaSuccess) made--;
    std::vector<cudaEvent_t> ev(n + 1, nullptr);
    for (int i = 0; i <= n && e == cudaSuccess; i++) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    cudaGraph_t g = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = cudaEventRecord(ev[n], cs);  // fork point
        std::vector<int> tail(kBranches, -1);          // last op on each branch
        std::vector<char> forked(kBranches, 0);
        int rr = 0;
        for (int i = 0; i < n && le == cudaSuccess; i++) {
            // continue the branch whose tail is the latest dependency, else the next branch
            int b = -1, latest = deps[i].empty() ? -1 : deps[i].back();
            for (int q = 0; q < kBranches; q++)
                if (latest >= 0 && tail[q] == latest) b = q;
            if (b < 0) b = (rr++) % kBranches;
            if (!forked[b]) {
                le = cudaStreamWaitEvent(br[b], ev[n], 0);
                forked[b] = 1;
            }
            for (int j : deps[i])
                if (le == cudaSuccess && j != tail[b]) le = cudaStreamWaitEvent(br[b], ev[j], 0);
            if (le == cudaSuccess) le = run_op(P, ops[i], br[b]);
            if (le == cudaSuccess) le = cudaEventRecord(ev[i], br[b]);
            tail[b] = i;
        }
        for (int q = 0; q < kBranches && le == cudaSuccess; q++)  // join
            if (tail[q] >= 0) le = cudaStreamWaitEvent(cs, ev[tail[q]], 0);
        e = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    for (auto x : ev)
        if (x) cudaEventDestroy(x);
    for (int q = 0; q < made; q++) cudaStreamDestroy(br[q]);
    cudaStreamDestroy(cs);
    return e;
}

cudaError_t build_graphs(tn_plan &P) {
    cudaError_t e = capture_ops(P, P.prologue, &P.g_pro);
    if (e == cudaSuccess) e = capture_ops(P, P.batch, &P.g_body);
    if (e == cudaSuccess) P.graphs_ready = true;
    return e;
}

cudaError_t prof_collect(tn_plan &P, size_t r0, size_t r1, cudaStream_t s) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    for (size_t r = r0; r < r1; r++) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, P.prof_ev[2 * r], P.prof_ev[2 * r + 1]) == cudaSuccess) {
            P.prof[r].ms += ms;
            P.prof[r].calls += 1;
        }
    }
    return cudaSuccess;
}

}  // namespace
}  // namespace tn

extern "C" int tn_contract_slices(tn_plan_t P, int64_t begin, int64_t end, double *d_amp, tn_stream_t stream) {
    if (!P) return fail(TN_ERR_ARG, "plan is NULL");
    if (P->failed) return fail(TN_ERR_STATE, "plan is in a failed state");
    const int64_t S = (int64_t)1 << P->n_sliced;
    if (begin < 0 || end > S || begin > end) return fail(TN_ERR_ARG, "slice range outside [0, 2^n_sliced)");
    if (!d_amp) return fail(TN_ERR_ARG, "d_amp is NULL");
    if (begin == end) return TN_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool prof = P->opts.profile != 0;
    if (prof) prof_init(*P);
    cudaError_t e = cudaSuccess;
    if (P->opts.use_graph && !prof && P->graphs_ready) {
        // replay: prologue graph, then per block extract + body graph + FP64 sum
        if (P->g_pro && (e = cudaGraphLaunch(P->g_pro, s)) != cudaSuccess) {
            P->failed = true;
            return cuda_fail(e, "prologue graph launch");
        }
        const int64_t B = (int64_t)1 << P->nb;
        AccumArgs acc = P->accum;
        acc.amp = reinterpret_cast<double2 *>(d_amp);
        for (int64_t base = (begin / B) * B; base < end; base += B) {
            e = launch_extract(P->d_extract, (int)P->extract.size(), P->extract_max_out, (uint64_t)base, s);
            if (e == cudaSuccess && P->g_body) e = cudaGraphLaunch(P->g_body, s);
            acc.b_lo = std::max(begin, base) - base;
            acc.b_hi = std::min(end, base + B) - base;
            if (e == cudaSuccess) e = launch_accum(acc, s);
            if (e != cudaSuccess) {
                P->failed = true;
                return cuda_fail(e, "graph replay");
            }
        }
        P->graph_calls++;
        return TN_OK;
    }
    size_t row = 0;
    auto timed = [&](auto &&launch) -> cudaError_t {
        if (prof) cudaEventRecord(P->prof_ev[2 * row], s);
        cudaError_t r = launch();
        if (prof) cudaEventRecord(P->prof_ev[2 * row + 1], s);
        row++;
        return r;
    };
    for (auto &op : P->prologue)
        if ((e = timed([&] { return run_op(*P, op, s); })) != cudaSuccess) {
            P->failed = true;
            return cuda_fail(e, "prologue launch");
        }
    if (prof && (e = prof_collect(*P, 0, row, s)) != cudaSuccess) { P->failed = true; return cuda_fail(e, "profile"); }
    const size_t row_block = row;
    const int64_t B = (int64_t)1 << P->nb;
    AccumArgs acc = P->accum;
    acc.amp = reinterpret_cast<double2 *>(d_amp);
    for (int64_t base = (begin / B) * B; base < end; base += B) {
        row = row_block;
        if ((e = timed([&] {
                 return launch_extract(P->d_extract, (int)P->extract.size(), P->extract_max_out, (uint64_t)base, s);
             })) != cudaSuccess) { P->failed = true; return cuda_fail(e, "extract launch"); }
        for (auto &op : P->batch)
            if ((e = timed([&] { return run_op(*P, op, s); })) != cudaSuccess) {
                P->failed = true;
                return cuda_fail(e, "step launch");
            }
        acc.b_lo = std::max(begin, base) - base;
        acc.b_hi = std::min(end, base + B) - base;
        if ((e = timed([&] { return launch_accum(acc, s); })) != cudaSuccess) {
            P->failed = true;
            return cuda_fail(e, "accumulate launch");
        }
        if (prof && (e = prof_collect(*P, row_block, row, s)) != cudaSuccess) {
            P->failed = true;
            return cuda_fail(e, "profile");
        }
    }
    if (prof && device_wait_error(s)) {
        P->failed = true;
        return fail(TN_ERR_TIMEOUT, "a bounded device wait expired (tensor-core pipeline or task dependency)");
    }
    if (P->opts.use_graph && !prof && !P->graphs_ready && (e = build_graphs(*P)) != cudaSuccess) {
        P->failed = true;
        return cuda_fail(e, "graph capture");
    }
    return TN_OK;
}

extern "C" int tn_plan_profile(tn_plan_t P, int max_rows, double *rows, int reset) {
    if (!P || (max_rows > 0 && !rows)) return fail(TN_ERR_ARG, "NULL argument");
    int n = 0;
    for (auto &r : P->prof) {
        if (n >= max_rows) break;
        double *o = rows + 12 * n;
        o[0] = r.phase; o[1] = r.idx; o[2] = r.kind; o[3] = r.step;
        o[4] = r.ms; o[5] = (double)r.calls; o[6] = r.macs; o[7] = r.bytes;
        for (int q = 0; q < 4; q++) o[8 + q] = r.shape[q];
        n++;
    }
    if (reset)
        for (auto &r : P->prof) { r.ms = 0; r.calls = 0; }
    return n;
}

namespace tn {
namespace {

// (form, H, M, N, K) -> tuned (chunk bytes, read-out bytes), process-wide
std::map<std::tuple<int, int64_t, int64_t, int64_t, int64_t>, std::pair<int, int>> g_tuned;
std::mutex g_tuned_mu;

}  // namespace
}  // namespace tn

extern "C" int tn_plan_autotune(tn_plan_t P, int reps, tn_stream_t stream) {
    if (!P) return fail(TN_ERR_ARG, "plan is NULL");
    if (P->failed) return fail(TN_ERR_STATE, "plan is in a failed state");
    if (reps < 1) reps = 3;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // (chunk bytes, read-out bytes); read-outs never sparser than the form's
    // default, which bounds the accumulation error
    const int D = tc_default_flush_bytes(P->form);
    const int kCand[][2] = {{128, D}, {128, D / 2 < 128 ? 128 : D / 2}, {64, D}, {64, D / 2}};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(TN_ERR_CUDA, "cudaEventCreate");
    int rc = TN_OK;
    for (auto *ops : {&P->prologue, &P->batch})
        for (auto &op : *ops) {
            if (op.kind != OP_GEMM || op.gemm_variant != 1) continue;
            const auto key = std::make_tuple((int)P->form, op.tc.a.H, op.tc.a.M, op.tc.a.N, op.tc.a.K);
            {
                std::lock_guard<std::mutex> lk(g_tuned_mu);
                auto it = g_tuned.find(key);
                if (it != g_tuned.end()) {
                    op.tc.chunk_bytes = it->second.first;
                    op.tc.flush_bytes = it->second.second;
                    if (!tc_prepare(op.tc)) rc = fail(TN_ERR_CUDA, "TMA descriptor encoding failed");
                    continue;
                }
            }
            // time each candidate on the current buffers (values do not matter)
            float best_ms = 1e30f;
            int best = 0;
            for (int ci = 0; ci < (int)(sizeof kCand / sizeof kCand[0]); ci++) {
                TcGemm g = op.tc;
                g.chunk_bytes = kCand[ci][0];
                g.flush_bytes = kCand[ci][1];
                if (!tc_prepare(g)) continue;
                cudaError_t e = launch_gemm_tc(g, s);  // warm-up
                cudaEventRecord(e0, s);
                for (int r = 0; r < reps && e == cudaSuccess; r++) e = launch_gemm_tc(g, s);
                cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) {
                    rc = cuda_fail(e, "autotune");
                    break;
                }
                if (ms < best_ms) {
                    best_ms = ms;
                    best = ci;
                }
            }
            if (rc) break;
            op.tc.chunk_bytes = kCand[best][0];
            op.tc.flush_bytes = kCand[best][1];
            if (!tc_prepare(op.tc)) { rc = fail(TN_ERR_CUDA, "TMA descriptor encoding failed"); break; }
            std::lock_guard<std::mutex> lk(g_tuned_mu);
            g_tuned[key] = {kCand[best][0], kCand[best][1]};
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == TN_OK && device_wait_error(s))
        rc = fail(TN_ERR_TIMEOUT, "a bounded device wait expired (tensor-core pipeline or task dependency)");
    if (rc) P->failed = true;
    // graphs captured earlier hold the old configuration
    if (P->graphs_ready) {
        if (P->g_pro) cudaGraphExecDestroy(P->g_pro);
        if (P->g_body) cudaGraphExecDestroy(P->g_body);
        P->g_pro = P->g_body = nullptr;
        P->graphs_ready = false;
    }
    return rc;
}

struct tn_batch {
    std::vector<tn_plan_t> plans;
    std::vector<double *> amps;
    int n_streams = 4;
    std::vector<int> stream_of;  // plan -> worker stream (longest job first)
    cudaGraphExec_t exec = nullptr;
    int64_t runs = 0;
};

namespace tn {
namespace {

// every op of one plan for all its slices, overwriting its amplitude tensor
cudaError_t enqueue_plan_all(const tn_plan &P, double *amp, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(amp, 0, sizeof(double) * 2 * ((size_t)1 << P.n_open), s);
    for (const auto &op : P.prologue)
        if (e == cudaSuccess) e = run_op(P, op, s);
    const int64_t B = (int64_t)1 << P.nb, S = (int64_t)1 << P.n_sliced;
    AccumArgs acc = P.accum;
    acc.amp = reinterpret_cast<double2 *>(amp);
    for (int64_t base = 0; base < S && e == cudaSuccess; base += B) {
        e = launch_extract(P.d_extract, (int)P.extract.size(), P.extract_max_out, (uint64_t)base, s);
        for (const auto &op : P.batch)
            if (e == cudaSuccess) e = run_op(P, op, s);
        acc.b_lo = 0;
        acc.b_hi = B;
        if (e == cudaSuccess) e = launch_accum(acc, s);
    }
    return e;
}

cudaError_t capture_batch(tn_batch &b) {
    cudaStream_t s0;
    cudaError_t e = cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    std::vector<cudaStream_t> ws(b.n_streams, nullptr);
    std::vector<cudaEvent_t> done(b.n_streams, nullptr);
    cudaEvent_t fork = nullptr;
    for (int i = 0; i < b.n_streams && e == cudaSuccess; i++) {
        e = cudaStreamCreateWithFlags(&ws[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    cudaGraph_t g = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = cudaEventRecord(fork, s0);
        for (int i = 0; i < b.n_streams && le == cudaSuccess; i++) le = cudaStreamWaitEvent(ws[i], fork, 0);
        for (size_t p = 0; p < b.plans.size() && le == cudaSuccess; p++)
            le = enqueue_plan_all(*b.plans[p], b.amps[p], ws[b.stream_of[p]]);
        for (int i = 0; i < b.n_streams && le == cudaSuccess; i++) {
            le = cudaEventRecord(done[i], ws[i]);
            if (le == cudaSuccess) le = cudaStreamWaitEvent(s0, done[i], 0);
        }
        e = cudaStreamEndCapture(s0, &g);
        if (e == cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b.exec, g, 0);
    if (g) cudaGraphDestroy(g);
    for (int i = 0; i < b.n_streams; i++) {
        if (ws[i]) cudaStreamDestroy(ws[i]);
        if (done[i]) cudaEventDestroy(done[i]);
    }
    if (fork) cudaEventDestroy(fork);
    cudaStreamDestroy(s0);
    return e;
}

}  // namespace
}  // namespace tn

extern "C" int tn_batch_create(tn_batch_t *out, int n_plans, const tn_plan_t *plans, double *const *d_amps,
                               int n_streams) {
    if (!out) return fail(TN_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_plans <= 0 || !plans || !d_amps) return fail(TN_ERR_ARG, "tn_batch_create: need plans and amplitudes");
    std::unique_ptr<tn_batch> b(new tn_batch());
    b->n_streams = n_streams > 0 ? std::min(n_streams, 32) : 4;
    std::vector<double> work(n_plans);
    for (int i = 0; i < n_plans; i++) {
        if (!plans[i] || !d_amps[i]) return fail(TN_ERR_ARG, "tn_batch_create: NULL plan or amplitude buffer");
        if (plans[i]->failed) return fail(TN_ERR_STATE, "tn_batch_create: a plan is in a failed state");
        b->plans.push_back(plans[i]);
        b->amps.push_back(d_amps[i]);
        const tn_plan &P = *plans[i];
        work[i] = P.macs_prologue + P.macs_batch * std::exp2((double)(P.n_sliced - P.nb)) + 1.0;
    }
    // longest job first onto the least-loaded stream
    std::vector<int> order(n_plans);
    for (int i = 0; i < n_plans; i++) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
    std::vector<double> load(b->n_streams, 0.0);
    b->stream_of.assign(n_plans, 0);
    for (int i : order) {
        int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        b->stream_of[i] = k;
        load[k] += work[i];
    }
    *out = b.release();
    return TN_OK;
}

extern "C" int tn_batch_run(tn_batch_t b, tn_stream_t stream) {
    if (!b) return fail(TN_ERR_ARG, "batch is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (!b->exec) {
        // first run: eager on the caller's stream (sets up every kernel), then capture
        for (size_t p = 0; p < b->plans.size() && e == cudaSuccess; p++)
            e = enqueue_plan_all(*b->plans[p], b->amps[p], s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = capture_batch(*b);
    } else {
        e = cudaGraphLaunch(b->exec, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "tn_batch_run");
    b->runs++;
    return TN_OK;
}

extern "C" void tn_batch_destroy(tn_batch_t b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    delete b;
}

extern "C" int tn_plan_op_features(tn_plan_t P, float *out, int max_ops) {
    if (!P || (max_ops > 0 && !out)) return fail(TN_ERR_ARG, "NULL argument");
    int n = 0;
    for (auto *ops : {&P->prologue, &P->batch})
        for (const auto &op : *ops) {
            if (n >= max_ops) return n;
            op_features(op, P->form, out + (size_t)n * kCostFeatures);
            n++;
        }
    return n;
}

extern "C" int tn_contract_slices_host(tn_plan_t P, int64_t begin, int64_t end, const float *h_data, int n_qubits,
                                       double *h_amp, double *h_stats, tn_stream_t stream) {
    if (!P) return fail(TN_ERR_ARG, "plan is NULL");
    if (h_stats && n_qubits < P->n_open) return fail(TN_ERR_ARG, "n_qubits < n_open");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n_amp = (int64_t)1 << P->n_open;
    if (!P->d_host_amp) {
        cudaError_t e = cudaMalloc(&P->d_host_amp, sizeof(double) * (2 * n_amp + 3));
        if (e != cudaSuccess) {
            P->d_host_amp = nullptr;
            cudaGetLastError();
            return fail(TN_ERR_OOM, "tn_contract_slices_host: device amplitude tensor");
        }
    }
    int rc = TN_OK;
    if (h_data) rc = tn_plan_update_data(P, h_data, stream);
    if (rc) return rc;
    cudaError_t e = launch_zero_f64(P->d_host_amp, 2 * n_amp, s);
    if (e != cudaSuccess) return cuda_fail(e, "tn_contract_slices_host");
    rc = tn_contract_slices(P, begin, end, P->d_host_amp, stream);
    if (rc) return rc;
    double *d_stats = P->d_host_amp + 2 * n_amp;
    if (h_stats) {
        e = launch_prob_xeb(reinterpret_cast<const double2 *>(P->d_host_amp), n_amp, nullptr, d_stats,
                            n_qubits - P->n_open, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_stats, d_stats, 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "tn_contract_slices_host: probabilities");
    }
    if (h_amp) {
        e = cudaMemcpyAsync(h_amp, P->d_host_amp, sizeof(double) * 2 * n_amp, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "tn_contract_slices_host: copy out");
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "tn_contract_slices_host");
    return TN_OK;
}

extern "C" int tn_plan_update_data(tn_plan_t P, const float *data, tn_stream_t stream) {
    if (!P || !data) return fail(TN_ERR_ARG, "NULL argument");
    cudaError_t e = cudaMemcpyAsync(P->d_leaves, data, P->leaf_bytes, cudaMemcpyHostToDevice,
                                    reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "tn_plan_update_data");
    return TN_OK;
}

extern "C" void tn_plan_destroy(tn_plan_t P) {
    if (!P) return;
    if (P->d_leaves) cudaFree(P->d_leaves);
    if (P->d_arena) cudaFree(P->d_arena);
    if (P->d_host_amp) cudaFree(P->d_host_amp);
    if (P->d_extract) cudaFree(P->d_extract);
    for (void *m : P->task_mem) cudaFree(m);
    for (auto &ev : P->prof_ev) cudaEventDestroy(ev);
    if (P->g_pro) cudaGraphExecDestroy(P->g_pro);
    if (P->g_body) cudaGraphExecDestroy(P->g_body);
    delete P;
}

namespace tn {
// replace leaf `leaf`'s values by host complex64 data (interleaved, 2^rank
// values), stream-ordered
int plan_load_leaf_host(tn_plan_t P, int leaf, const float *src, cudaStream_t s) {
    if (!P || !src || leaf < 0 || leaf >= P->n_tensors) return fail(TN_ERR_ARG, "plan_load_leaf_host: bad arguments");
    const int64_t n = (int64_t)1 << P->labels[leaf].size();
    cudaError_t e = cudaMemcpyAsync(P->d_leaves + P->leaf_off[leaf], src, sizeof(float2) * n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(TN_ERR_CUDA, std::string("plan_load_leaf_host: ") + cudaGetErrorString(e));
    return TN_OK;
}

// replace leaf `leaf`'s values by complex128 device data (rounded to
// complex64), stream-ordered; the leaf keeps its rank and labels
int plan_load_leaf_c128(tn_plan_t P, int leaf, const double *d_src, cudaStream_t s) {
    if (!P || !d_src || leaf < 0 || leaf >= P->n_tensors) return fail(TN_ERR_ARG, "plan_load_leaf_c128: bad arguments");
    const int64_t n = (int64_t)1 << P->labels[leaf].size();
    cudaError_t e = launch_c128_to_c64(reinterpret_cast<const double2 *>(d_src), P->d_leaves + P->leaf_off[leaf], n, s);
    if (e != cudaSuccess) return fail(TN_ERR_CUDA, std::string("plan_load_leaf_c128: ") + cudaGetErrorString(e));
    return TN_OK;
}
}  // namespace tn

namespace tn {

// One line per compiled op (kind, shape, kernel variant, plan-time notes);
// with with_roofline, each line also gives the op's roofline time.
std::string describe_ops(const tn_plan &P, bool with_roofline) {
    std::string txt;
    char line[512];
    auto put = [&](const char *phase, const Op &op) {
        switch (op.kind) {
        case OP_TASKS: {
            int64_t rows = 0;
            for (const Op &m : op.members) rows += m.small.rows;
            std::snprintf(line, sizeof line, "%s step %d tasks n=%d levels=%d rows=%lld (steps", phase, op.step,
                          (int)op.members.size(), op.task_levels, (long long)rows);
            std::string l(line);
            for (size_t i = 0; i < op.members.size() && i < 8; i++) l += " " + std::to_string(op.members[i].step);
            l += op.members.size() > 8 ? " ...)" : ")";
            std::snprintf(line, sizeof line, "%s", l.c_str());
            break;
        }
        case OP_SMALL: {
            const SmallArgs &a = op.small;
            const char *kern = a.tc_form ? "tensor cores, split in shared memory"
                               : a.tiled == 1 ? "tiled, staged C" : a.tiled == 2 ? "tiled, direct C"
                               : a.tiled == 3 ? "tiled, planar" : "row";
            // bit positions of k in T and of n in C
            std::string kp, np;
            for (int j = 0; j < a.nK; j++) kp += (j ? "," : "") + std::to_string(a.kposT[j]);
            for (int j = 0; j < a.nN; j++) np += (j ? "," : "") + std::to_string(a.nposC[j]);
            std::snprintf(line, sizeof line, "%s step %d small rows=%lld K=%d N=%d H=%d kernel=%s kposT=%s nposC=%s",
                          phase, op.step, (long long)a.rows, 1 << a.nK, 1 << a.nN, 1 << a.nH, kern, kp.c_str(),
                          np.c_str());
            break;
        }
        case OP_GEMM:
            if (op.gemm_variant == 1)
            {
                // planar output: how many of the destination's lowest bits
                // come from the epilogue's half tile in order (its store runs
                // are 2^run elements per plane), and whether lanes store four
                // neighbouring elements
                int run = 0;
                while (run < op.tc.out.ntb && op.tc.out.tpos[run] == run) run++;
                // the tile's six column bits are the destination's six lowest
                bool cols_low = op.tc.out.ntb >= 6;
                for (int k = 0; k < 6 && cols_low; k++) cols_low = op.tc.out.tb[k] == k && op.tc.out.tpos[k] == k;
                char pl[320] = "";
                if (op.tc.out.mode) {
                    // the half tile's bits in destination order (c: column of
                    // the tile, r: row) with their destination positions
                    std::string tbits;
                    for (int k = 0; k < op.tc.out.ntb; k++)
                        tbits += (k ? "," : "") + std::string(op.tc.out.tb[k] < 6 ? "c" : "r") +
                                 std::to_string(op.tc.out.tb[k] < 6 ? op.tc.out.tb[k] : op.tc.out.tb[k] - 6) + "@" +
                                 std::to_string(op.tc.out.tpos[k]);
                    const int direct = tc_planar_direct_run(op.tc.out);
                    // TMA store: the box's extent per dimension (destination bits start@log2 box)
                    TcTmaOut tm;
                    std::string tma = " staged";
                    // (eight-warp kernel only: tiles with more than one accumulator read-out)
                    const int es = tc_plane_bytes(P.form);
                    const int chunk = P.opts.tc_chunk_bytes == 64 ? 64 : 128;
                    int flush = P.opts.tc_flush_bytes > 0 ? P.opts.tc_flush_bytes : tc_default_flush_bytes(P.form);
                    if (flush < chunk) flush = chunk;
                    const bool one_readout = (op.gemm.K * es + chunk - 1) / chunk <= flush / chunk;
                    if (!direct && !one_readout && op.tc.tma_out_ok && op.tc.products != 3 &&
                        tc_planar_tma_fits(op.tc.out, &tm)) {
                        tma = " tma box=";
                        for (int i = 0; i < tm.nd; i++)
                            tma += (i ? "," : "") + std::to_string(tm.start[i]) + "@" + std::to_string(tm.box[i]);
                    }
                    std::snprintf(pl, sizeof pl, " run_bits=%d%s%s%s tile_bits=%s", run,
                                  (op.tc.out.ntb >= 7 && op.tc.out.tpos[0] == 0 && op.tc.out.tpos[1] == 1) ? " quad"
                                                                                                            : "",
                                  cols_low ? " cols_low" : "",
                                  direct ? (" direct=" + std::to_string(1 << direct)).c_str() : tma.c_str(),
                                  tbits.c_str());
                }
                std::snprintf(line, sizeof line,
                              "%s step %d gemm H=%lld M=%lld N=%lld K=%lld tensor-core%s ksplit=%d out=%s%s", phase,
                              op.step, (long long)op.gemm.H, (long long)op.gemm.M, (long long)op.gemm.N,
                              (long long)op.gemm.K, op.tc.products == 3 ? " 3M" : "", op.tc.ksplit,
                              op.tc.out.mode ? "planes" : "complex64", pl);
            }
            else
                std::snprintf(line, sizeof line, "%s step %d gemm H=%lld M=%lld N=%lld K=%lld fp32", phase, op.step,
                              (long long)op.gemm.H, (long long)op.gemm.M, (long long)op.gemm.N, (long long)op.gemm.K);
            break;
        case OP_PERMUTE:
        case OP_SPLIT:
            std::snprintf(line, sizeof line, "%s step %d %s rank=%d mode=%d", phase, op.step,
                          op.kind == OP_SPLIT ? "split" : "permute", op.bp.rank, op.bp.mode);
            break;
        case OP_MAXABS:
            std::snprintf(line, sizeof line, "%s step %d maxabs n=%lld", phase, op.step, (long long)op.mx.n);
            break;
        }
        txt += line;
        if (with_roofline) {
            std::snprintf(line, sizeof line, " roofline_ms=%.6g", roofline_ms(op, P.form));
            txt += line;
        }
        if (!op.note.empty()) txt += " (" + op.note + ")";
        txt += "\n";
    };
    for (const auto &op : P.prologue) put("prologue", op);
    for (const auto &op : P.batch) put("batch", op);
    return txt;
}

int copy_text(const std::string &txt, char *out, int cap) {
    if (cap > 0) {
        const size_t n = std::min(txt.size(), (size_t)cap - 1);
        std::memcpy(out, txt.data(), n);
        out[n] = 0;
    }
    return (int)txt.size();
}

}  // namespace tn

extern "C" int tn_plan_describe(tn_plan_t P, char *out, int cap) {
    if (!P || cap < 0 || (cap > 0 && !out)) return fail(TN_ERR_ARG, "bad arguments");
    return copy_text(describe_ops(*P, false), out, cap);
}

extern "C" int tn_plan_stats(tn_plan_t P, double *out) {
    if (!P || !out) return fail(TN_ERR_ARG, "NULL argument");
    out[0] = P->macs_batch;
    out[1] = (double)((int64_t)1 << P->nb);
    out[2] = (double)P->arena_bytes;
    out[3] = (double)P->tree.size();
    out[4] = (double)P->launches_batch;
    out[5] = P->bytes_batch;
    out[6] = P->macs_prologue;
    out[7] = P->bytes_prologue;
    out[8] = (double)P->launches_prologue;
    out[9] = (double)P->nb;
    out[10] = (double)P->graph_calls;
    return TN_OK;
}

extern "C" int tn_probabilities_xeb(const double *d_amp, int n_open, int n_qubits, double *d_prob, double *d_out,
                                    double *out, tn_stream_t stream) {
    if (!d_amp || !d_out || n_open < 0 || n_open > 40 || n_qubits < n_open) return fail(TN_ERR_ARG, "bad arguments");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = launch_prob_xeb(reinterpret_cast<const double2 *>(d_amp), (int64_t)1 << n_open, d_prob, d_out,
                                    n_qubits - n_open, s);
    if (e != cudaSuccess) return cuda_fail(e, "probabilities");
    if (out) {
        e = cudaMemcpyAsync(out, d_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "probabilities");
    }
    return TN_OK;
}

extern "C" int tn_amplitudes(const tn_circuit *circuit, const uint8_t *fixed_bits, int n_open,
                             const int32_t *open_qubits, tn_form form, const tn_search_opts *search,
                             const tn_plan_opts *opts, double *d_amp, tn_stream_t stream) {
    if (!d_amp) return fail(TN_ERR_ARG, "d_amp is NULL");
    Network net;
    int rc = build_circuit_network(circuit, fixed_bits, n_open, open_qubits, net);
    if (rc) return rc;
    std::vector<std::vector<int32_t>> labs;
    for (auto &t : net.tensors) labs.push_back(t.labels);
    tn_search_opts so = search ? *search : default_search_opts();
    SearchResult r;
    rc = search_ranked(labs, net.open, so, r);
    if (rc) return rc;
    std::vector<int32_t> ranks, flat, tree;
    std::vector<float> data;
    for (auto &t : net.tensors) {
        ranks.push_back(t.rank());
        flat.insert(flat.end(), t.labels.begin(), t.labels.end());
        for (auto &v : t.data) {
            data.push_back((float)v.real());
            data.push_back((float)v.imag());
        }
    }
    for (auto &pr : r.tree) {
        tree.push_back(pr.first);
        tree.push_back(pr.second);
    }
    tn_plan_t plan = nullptr;
    rc = tn_plan_create(&plan, (int)net.tensors.size(), ranks.data(), flat.data(), data.data(), 0, nullptr,
                        n_open, net.open.data(), (int)r.sliced.size(), r.sliced.data(), (int)r.tree.size(),
                        tree.data(), form, opts);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(d_amp, 0, sizeof(double) * 2 * ((size_t)1 << n_open), s);
    if (e != cudaSuccess) { tn_plan_destroy(plan); return cuda_fail(e, "zero amplitudes"); }
    rc = tn_contract_slices(plan, 0, (int64_t)1 << r.sliced.size(), d_amp, stream);
    if (rc == TN_OK) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "contract");
        else if (device_wait_error(s))
            rc = fail(TN_ERR_TIMEOUT, "a bounded device wait expired (tensor-core pipeline or task dependency)");
    }
    tn_plan_destroy(plan);
    return rc;
}

extern "C" int tn_estimate_tree_ms(int n_tensors, const int32_t *ranks, const int32_t *labels, int n_open,
                                   const int32_t *open_labels, int n_sliced, const int32_t *sliced_labels,
                                   int n_steps, const int32_t *tree, tn_form form, const tn_plan_opts *opts,
                                   int batch_log2, int64_t arena_budget, double *out_ms, int *out_batch_log2,
                                   int64_t *out_arena, double *out_prologue_ms, double *out_block_ms) {
    if (form < TN_FP32 || form > TN_FP16X3) return fail(TN_ERR_ARG, "unknown form");
    if (!out_ms) return fail(TN_ERR_ARG, "out_ms is NULL");
    tn_plan P;
    P.form = form;
    if (opts) P.opts = *opts;
    P.opts.batch_log2 = -1;
    int64_t total = 0;
    int rc = plan_host_setup(P, n_tensors, ranks, labels, 0, nullptr, n_open, open_labels, n_sliced, sliced_labels,
                             n_steps, tree, &total);
    if (rc) return rc;
    const double budget = arena_budget > 0 ? (double)arena_budget : kNominalArenaBytes;
    double ms = 0;
    int nb = 0;
    int64_t arena = 0;
    rc = plan_roofline(P, batch_log2, budget, total * 8, ms, nb, arena, out_prologue_ms, out_block_ms);
    if (rc) return rc;
    *out_ms = ms;
    if (out_batch_log2) *out_batch_log2 = nb;
    if (out_arena) *out_arena = arena;
    return TN_OK;
}

extern "C" int tn_describe_tree(int n_tensors, const int32_t *ranks, const int32_t *labels, int n_open,
                                const int32_t *open_labels, int n_sliced, const int32_t *sliced_labels, int n_steps,
                                const int32_t *tree, tn_form form, const tn_plan_opts *opts, int batch_log2,
                                int64_t arena_budget, char *out, int cap) {
    if (form < TN_FP32 || form > TN_FP16X3) return fail(TN_ERR_ARG, "unknown form");
    if (cap < 0 || (cap > 0 && !out)) return fail(TN_ERR_ARG, "bad output buffer");
    tn_plan P;
    P.form = form;
    if (opts) P.opts = *opts;
    P.opts.batch_log2 = -1;
    int64_t total = 0;
    int rc = plan_host_setup(P, n_tensors, ranks, labels, 0, nullptr, n_open, open_labels, n_sliced, sliced_labels,
                             n_steps, tree, &total);
    if (rc) return rc;
    const double budget = arena_budget > 0 ? (double)arena_budget : kNominalArenaBytes;
    double ms = 0;
    int nb = 0;
    int64_t arena = 0;
    rc = plan_roofline(P, batch_log2, budget, total * 8, ms, nb, arena);
    if (rc) return rc;
    return copy_text(describe_ops(P, true), out, cap);
}
