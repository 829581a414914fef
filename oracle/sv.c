/*
 * Schroedinger state-vector simulation in complex128, plain C with OpenMP
 * (oracle, test infrastructure only).
 *
 * Computes the amplitudes <s1; s2|U|0...0> of the "Big-head simulation"
 * section by definition: every gate of the circuit is applied, in circuit
 * order, to the full 2^n state vector.  Qubit 0 is the most significant bit
 * of a state index.  Gate g acts on qubits q[g][0..k-1] (k = 1 or 2) with the
 * row-major 2^k x 2^k complex matrix m[g] (row = output basis state, basis
 * index of a pair = 2*bit(q0) + bit(q1)).
 *
 * Shares no code with the CUDA path.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <complex.h>

typedef double complex cplx;

static inline uint64_t insert_zero(uint64_t x, int pos) {
    uint64_t lo = x & ((1ull << pos) - 1);
    return ((x >> pos) << (pos + 1)) | lo;
}

static void apply1(cplx *psi, int n, int q, const double *m) {
    int p = n - 1 - q;
    uint64_t half = 1ull << (n - 1), bit = 1ull << p;
    cplx g00 = m[0] + I * m[1], g01 = m[2] + I * m[3];
    cplx g10 = m[4] + I * m[5], g11 = m[6] + I * m[7];
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < (int64_t)half; j++) {
        uint64_t i0 = insert_zero((uint64_t)j, p), i1 = i0 | bit;
        cplx a0 = psi[i0], a1 = psi[i1];
        psi[i0] = g00 * a0 + g01 * a1;
        psi[i1] = g10 * a0 + g11 * a1;
    }
}

static void apply2(cplx *psi, int n, int q0, int q1, const double *m) {
    int p0 = n - 1 - q0, p1 = n - 1 - q1;
    int lo = p0 < p1 ? p0 : p1, hi = p0 < p1 ? p1 : p0;
    uint64_t quarter = 1ull << (n - 2), b0 = 1ull << p0, b1 = 1ull << p1;
    cplx g[16];
    for (int e = 0; e < 16; e++) g[e] = m[2 * e] + I * m[2 * e + 1];
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < (int64_t)quarter; j++) {
        uint64_t base = insert_zero(insert_zero((uint64_t)j, lo), hi);
        uint64_t idx[4] = {base, base | b1, base | b0, base | b0 | b1};
        cplx a[4], o[4];
        for (int r = 0; r < 4; r++) a[r] = psi[idx[r]];
        for (int r = 0; r < 4; r++) {
            cplx s = 0;
            for (int c = 0; c < 4; c++) s += g[4 * r + c] * a[c];
            o[r] = s;
        }
        for (int r = 0; r < 4; r++) psi[idx[r]] = o[r];
    }
}

/*
 * n_qubits <= 34; gate_nq[g] in {1,2}; gate_q[2g], gate_q[2g+1] the qubits;
 * gate_m[32g ...] the interleaved (re, im) matrix (4 or 16 entries used).
 * fixed_bits[n_qubits] (ignored at open positions), open_qubits[n_open] in
 * output order (first = most significant).  out_amp: 2 * 2^n_open doubles.
 * Returns 0 on success, -1 on bad arguments, -2 if the vector cannot be
 * allocated.
 */
int oracle_sv_amplitudes(int n_qubits, int n_gates, const int *gate_nq, const int *gate_q,
                         const double *gate_m, const int *fixed_bits, int n_open,
                         const int *open_qubits, double *out_amp) {
    if (n_qubits < 1 || n_qubits > 34 || n_open < 0 || n_open > n_qubits) return -1;
    uint64_t dim = 1ull << n_qubits;
    cplx *psi = (cplx *)malloc(dim * sizeof(cplx));
    if (!psi) return -2;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)dim; i++) psi[i] = 0;
    psi[0] = 1;
    for (int g = 0; g < n_gates; g++) {
        if (gate_nq[g] == 1) apply1(psi, n_qubits, gate_q[2 * g], gate_m + 32 * g);
        else apply2(psi, n_qubits, gate_q[2 * g], gate_q[2 * g + 1], gate_m + 32 * g);
    }
    uint64_t base = 0;
    char is_open[64];
    memset(is_open, 0, sizeof is_open);
    for (int j = 0; j < n_open; j++) is_open[open_qubits[j]] = 1;
    for (int q = 0; q < n_qubits; q++)
        if (!is_open[q] && fixed_bits[q]) base |= 1ull << (n_qubits - 1 - q);
    for (uint64_t a = 0; a < (1ull << n_open); a++) {
        uint64_t idx = base;
        for (int j = 0; j < n_open; j++)
            if ((a >> (n_open - 1 - j)) & 1) idx |= 1ull << (n_qubits - 1 - open_qubits[j]);
        out_amp[2 * a] = creal(psi[idx]);
        out_amp[2 * a + 1] = cimag(psi[idx]);
    }
    free(psi);
    return 0;
}
