// Circuit -> tensor network with single-qubit gates absorbed into two-qubit
// gates (the simplification of the Sycamore section: single-qubit gates are
// absorbed so that 53 qubits x 20 cycles leaves 381 nodes).  The initial |0>
// vectors and the closed output bits are absorbed too, so every leaf is one
// two-qubit gate of rank <= 4 (plus rank <= 1 leaves for qubits no two-qubit
// gate touches).
//
// Bond labels follow the wire-segment convention: on qubit q the segment after
// the t-th gate is label offset_q + t, offset_q = sum_{q'<q} (g_{q'} + 1).  A
// two-qubit gate's output leg is the segment right after it; the open leg of
// qubit q is its final segment offset_q + g_q.
#include <cstring>
#include <string>

#include "tn_internal.h"

namespace tn {

namespace {

struct M2 {
    cd a[4];  // row-major 2x2
};

M2 identity2() { return M2{{1.0, 0.0, 0.0, 1.0}}; }

M2 mul2(const M2 &x, const M2 &y) {  // x * y
    M2 r;
    r.a[0] = x.a[0] * y.a[0] + x.a[1] * y.a[2];
    r.a[1] = x.a[0] * y.a[1] + x.a[1] * y.a[3];
    r.a[2] = x.a[2] * y.a[0] + x.a[3] * y.a[2];
    r.a[3] = x.a[2] * y.a[1] + x.a[3] * y.a[3];
    return r;
}

// T'[.., i, ..] = sum_j m[i][j] T[.., j, ..] on axis `ax`.  With transpose,
// T'[.., i, ..] = sum_j m[j][i] T[.., j, ..].
void apply_axis(Tensor &t, int ax, const M2 &m, bool transpose) {
    int r = t.rank();
    size_t stride = (size_t)1 << (r - 1 - ax);
    size_t n = t.data.size();
    for (size_t base = 0; base < n; base++) {
        if (base & stride) continue;
        cd x0 = t.data[base], x1 = t.data[base | stride];
        cd m00 = m.a[0], m01 = transpose ? m.a[2] : m.a[1];
        cd m10 = transpose ? m.a[1] : m.a[2], m11 = m.a[3];
        t.data[base] = m00 * x0 + m01 * x1;
        t.data[base | stride] = m10 * x0 + m11 * x1;
    }
}

// contract axis `ax` with vector v: T'[..] = sum_j v[j] T[.., j, ..]
void contract_axis(Tensor &t, int ax, cd v0, cd v1) {
    int r = t.rank();
    size_t stride = (size_t)1 << (r - 1 - ax);
    size_t n = t.data.size();
    std::vector<cd> out;
    out.reserve(n / 2);
    for (size_t base = 0; base < n; base++) {
        if (base & stride) continue;
        out.push_back(v0 * t.data[base] + v1 * t.data[base | stride]);
    }
    t.data.swap(out);
    t.labels.erase(t.labels.begin() + ax);
}

int axis_of(const Tensor &t, int32_t label) {
    for (int i = 0; i < t.rank(); i++)
        if (t.labels[i] == label) return i;
    return -1;
}

}  // namespace

int build_circuit_network(const tn_circuit *c, const uint8_t *fixed_bits, int n_open,
                          const int32_t *open_qubits, Network &out) {
    if (!c || c->n_qubits <= 0 || c->n_gates < 0 || (c->n_gates > 0 && (!c->gate_nq || !c->gate_q || !c->gate_m)))
        return fail(TN_ERR_ARG, "tn_circuit: bad sizes or NULL arrays");
    const int n = c->n_qubits;
    if (n_open < 0 || n_open > n || (n_open > 0 && !open_qubits))
        return fail(TN_ERR_ARG, "bad open qubit list");
    if (!fixed_bits && n_open < n) return fail(TN_ERR_ARG, "fixed_bits is NULL");
    std::vector<int> is_open(n, 0);
    for (int j = 0; j < n_open; j++) {
        int q = open_qubits[j];
        if (q < 0 || q >= n || is_open[q]) return fail(TN_ERR_ARG, "open qubit out of range or repeated");
        is_open[q] = 1;
    }
    // gates per qubit -> offsets
    std::vector<int> count(n, 0);
    for (int g = 0; g < c->n_gates; g++) {
        int k = c->gate_nq[g];
        if (k != 1 && k != 2) return fail(TN_ERR_ARG, "gate_nq must be 1 or 2");
        for (int j = 0; j < k; j++) {
            int q = c->gate_q[2 * g + j];
            if (q < 0 || q >= n) return fail(TN_ERR_ARG, "gate qubit out of range");
            count[q]++;
        }
        if (k == 2 && c->gate_q[2 * g] == c->gate_q[2 * g + 1]) return fail(TN_ERR_ARG, "two-qubit gate on one qubit");
    }
    std::vector<int32_t> offset(n, 0);
    int64_t acc = 0;
    for (int q = 0; q < n; q++) {
        offset[q] = (int32_t)acc;
        acc += count[q] + 1;
    }
    if (acc > INT32_MAX) return fail(TN_ERR_ARG, "too many wire segments");

    // bond[q]: label of the wire segment at q's frontier, i.e. the segment
    // right after the last two-qubit gate on q (segment 0 before any).
    // Pending single-qubit gates sit on that segment and are absorbed into the
    // next two-qubit gate's input (or the last one's output at the end).
    std::vector<M2> pend(n, identity2());
    std::vector<int> seg(n, 0), started(n, 0), last_t(n, -1);
    std::vector<int32_t> bond(n);
    for (int q = 0; q < n; q++) bond[q] = offset[q];
    std::vector<Tensor> ts;
    for (int g = 0; g < c->n_gates; g++) {
        const double *m = c->gate_m + 32 * (size_t)g;
        if (c->gate_nq[g] == 1) {
            int q = c->gate_q[2 * g];
            M2 u;
            for (int e = 0; e < 4; e++) u.a[e] = cd(m[2 * e], m[2 * e + 1]);
            pend[q] = mul2(u, pend[q]);
            seg[q]++;
            continue;
        }
        const int qa = c->gate_q[2 * g], qb = c->gate_q[2 * g + 1];
        Tensor t;
        t.data.resize(16);  // gate matrix reshaped to axes (out_a, out_b, in_a, in_b)
        for (int e = 0; e < 16; e++) t.data[e] = cd(m[2 * e], m[2 * e + 1]);
        seg[qa]++;
        seg[qb]++;
        t.labels = {offset[qa] + seg[qa], offset[qb] + seg[qb], bond[qa], bond[qb]};
        // G' = G (Pa (x) Pb): pending single-qubit gates enter on the inputs
        apply_axis(t, 2, pend[qa], true);
        apply_axis(t, 3, pend[qb], true);
        pend[qa] = identity2();
        pend[qb] = identity2();
        // initial |0>: keep input value 0 where no earlier gate feeds the qubit
        if (!started[qb]) contract_axis(t, 3, 1.0, 0.0);
        if (!started[qa]) contract_axis(t, 2, 1.0, 0.0);
        ts.push_back(std::move(t));
        const int ti = (int)ts.size() - 1;
        started[qa] = started[qb] = 1;
        last_t[qa] = last_t[qb] = ti;
        bond[qa] = offset[qa] + seg[qa];
        bond[qb] = offset[qb] + seg[qb];
    }
    std::vector<int32_t> open_labels(n_open);
    for (int q = 0; q < n; q++) {
        const int32_t final_lab = offset[q] + count[q];
        if (started[q]) {
            Tensor &t = ts[last_t[q]];
            int ax = axis_of(t, bond[q]);
            // trailing single-qubit gates act on the last gate's output leg
            apply_axis(t, ax, pend[q], false);
            if (is_open[q]) {
                t.labels[ax] = final_lab;
            } else {
                const int b = fixed_bits[q] ? 1 : 0;
                contract_axis(t, ax, b == 0 ? 1.0 : 0.0, b == 1 ? 1.0 : 0.0);
            }
        } else {
            // qubit untouched by two-qubit gates: its state is P|0>
            Tensor t;
            const cd v0 = pend[q].a[0], v1 = pend[q].a[2];
            if (is_open[q]) {
                t.labels = {final_lab};
                t.data = {v0, v1};
            } else {
                t.data = {fixed_bits[q] ? v1 : v0};
            }
            ts.push_back(std::move(t));
        }
    }
    for (int j = 0; j < n_open; j++) open_labels[j] = offset[open_qubits[j]] + count[open_qubits[j]];
    out.tensors.swap(ts);
    out.open = open_labels;
    return TN_OK;
}

}  // namespace tn
