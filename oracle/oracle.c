/*
 * oracle.c -- plain complex128 CPU state-vector simulator.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline / reference legs may load this file's library.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * What it computes (parity pinned by tests/test_oracle_pins.py):
 *   - state vector of Eq. 1: 2^n complex amplitudes, qubit j = bit j of the
 *     index (Section 2.2, U_j = I^{n-j-1} (x) U (x) I^{j});
 *   - gates applied one at a time to the whole vector, the gate-by-gate scheme
 *     of Algorithm 1: for a k-qubit gate on qubits q[0..k-1], for every base
 *     index b whose bits q[i] are all zero, gather the 2^k amplitudes
 *     b | sum_i c_i 2^{q[i]} (local bit i <-> q[i], the index order of
 *     Eqs. 2-3 with the higher qubit as the more significant local bit when
 *     q = [low, high]), multiply by the 2^k x 2^k matrix, scatter back.
 *
 * Gate matrices (the paper names its gates but gives no matrices; these are
 * the usual textbook / OpenQASM-3 definitions):
 *   H = [[1,1],[1,-1]]/sqrt2, X, Y = [[0,-i],[i,0]], Z = diag(1,-1),
 *   S = diag(1,i), T = diag(1,e^{i pi/4}),
 *   RX(t) = [[c,-is],[-is,c]], RY(t) = [[c,-s],[s,c]]  (c = cos t/2, s = sin t/2),
 *   RZ(t) = diag(e^{-it/2}, e^{it/2}), P(t) = diag(1, e^{it}),
 *   CX (q[0] control), CZ = diag(1,1,1,-1), CP(t) = diag(1,1,1,e^{it}),
 *   RZZ(t) = diag(e^{-it/2}, e^{it/2}, e^{it/2}, e^{-it/2}), SWAP,
 *   U1Q / UNITARY: caller's row-major matrix; DIAG: caller's 2^k diagonal.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

/* oracle-local gate codes (the Python wrapper maps gate names onto these) */
enum {
    O_H = 0, O_X, O_Y, O_Z, O_S, O_T, O_RX, O_RY, O_RZ, O_P,
    O_CX, O_CZ, O_CP, O_RZZ, O_SWAP, O_U1Q, O_UNITARY, O_DIAG
};

#define ORC_MAXK 6

/* Fill m (dim x dim, row-major) with the gate's matrix; returns dim or -1. */
static int gate_matrix(int kind, int k, const double *par, const double *ext, cplx *m)
{
    int dim = 1 << k;
    memset(m, 0, sizeof(cplx) * dim * dim);
    double t = par[0];
    double c = cos(t / 2), s = sin(t / 2);
    switch (kind) {
    case O_H: { double r = 1.0 / sqrt(2.0); m[0] = r; m[1] = r; m[2] = r; m[3] = -r; break; }
    case O_X: m[1] = 1; m[2] = 1; break;
    case O_Y: m[1] = -I; m[2] = I; break;
    case O_Z: m[0] = 1; m[3] = -1; break;
    case O_S: m[0] = 1; m[3] = I; break;
    case O_T: m[0] = 1; m[3] = cexp(I * M_PI / 4); break;
    case O_RX: m[0] = c; m[1] = -I * s; m[2] = -I * s; m[3] = c; break;
    case O_RY: m[0] = c; m[1] = -s; m[2] = s; m[3] = c; break;
    case O_RZ: m[0] = cexp(-I * t / 2); m[3] = cexp(I * t / 2); break;
    case O_P: m[0] = 1; m[3] = cexp(I * t); break;
    case O_CX:
        /* local index = b0 + 2 b1 with b0 the control: swap |01>=1 and |11>=3 */
        m[0 * 4 + 0] = 1; m[2 * 4 + 2] = 1; m[1 * 4 + 3] = 1; m[3 * 4 + 1] = 1; break;
    case O_CZ: m[0] = 1; m[5] = 1; m[10] = 1; m[15] = -1; break;
    case O_CP: m[0] = 1; m[5] = 1; m[10] = 1; m[15] = cexp(I * t); break;
    case O_RZZ:
        m[0] = cexp(-I * t / 2); m[5] = cexp(I * t / 2);
        m[10] = cexp(I * t / 2); m[15] = cexp(-I * t / 2); break;
    case O_SWAP: m[0] = 1; m[1 * 4 + 2] = 1; m[2 * 4 + 1] = 1; m[15] = 1; break;
    case O_U1Q:
    case O_UNITARY:
        for (int i = 0; i < dim * dim; i++) m[i] = ext[2 * i] + I * ext[2 * i + 1];
        break;
    case O_DIAG:
        for (int i = 0; i < dim; i++) m[i * dim + i] = ext[2 * i] + I * ext[2 * i + 1];
        break;
    default: return -1;
    }
    return dim;
}

static int gate_arity(int kind, int nq)
{
    switch (kind) {
    case O_CX: case O_CZ: case O_CP: case O_RZZ: case O_SWAP: return 2;
    case O_UNITARY: case O_DIAG: return nq;
    default: return 1;
    }
}

/* Apply one k-qubit matrix to the whole state (Algorithm 1, one gate). */
static void apply_matrix(int n, cplx *a, int k, const int *q, const cplx *m)
{
    int dim = 1 << k;
    int sq[ORC_MAXK];
    for (int i = 0; i < k; i++) sq[i] = q[i];
    for (int i = 1; i < k; i++)               /* insertion sort, ascending */
        for (int j = i; j > 0 && sq[j - 1] > sq[j]; j--) { int t = sq[j]; sq[j] = sq[j - 1]; sq[j - 1] = t; }
    int64_t nbase = (int64_t)1 << (n - k);
    int64_t off[1 << ORC_MAXK];
    for (int c = 0; c < dim; c++) {
        int64_t o = 0;
        for (int i = 0; i < k; i++) if ((c >> i) & 1) o |= (int64_t)1 << q[i];
        off[c] = o;
    }
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nbase; b++) {
        /* spread b over the non-target bits: insert a 0 at each target position */
        int64_t base = b;
        for (int i = 0; i < k; i++) {
            int64_t low = base & (((int64_t)1 << sq[i]) - 1);
            base = ((base >> sq[i]) << (sq[i] + 1)) | low;
        }
        cplx v[1 << ORC_MAXK], w[1 << ORC_MAXK];
        for (int c = 0; c < dim; c++) v[c] = a[base | off[c]];
        for (int r = 0; r < dim; r++) {
            cplx acc = 0;
            for (int c = 0; c < dim; c++) acc += m[r * dim + c] * v[c];
            w[r] = acc;
        }
        for (int c = 0; c < dim; c++) a[base | off[c]] = w[c];
    }
}

/* Validate a gate list; returns index of the first bad gate or -1. */
static int64_t check_gates(int n, int64_t n_gates, const int *kind, const int *nq, const int *qubits)
{
    for (int64_t g = 0; g < n_gates; g++) {
        if (kind[g] < O_H || kind[g] > O_DIAG) return g;
        int k = gate_arity(kind[g], nq[g]);
        if (k < 1 || k > ORC_MAXK || k > n || k > 6) return g;
        for (int i = 0; i < k; i++) {
            int qi = qubits[g * 6 + i];
            if (qi < 0 || qi >= n) return g;
            for (int j = 0; j < i; j++) if (qubits[g * 6 + j] == qi) return g;
        }
    }
    return -1;
}

/*
 * orc_run: apply n_gates gates to the interleaved (re,im) state in place.
 *   kind[g], nq[g], qubits[6g..6g+5], params[3g..3g+2]; ext_off[g] is the
 *   offset (in doubles) of the gate's matrix/diagonal in ext, or -1.
 * Returns -1 on success, else the index of the first invalid gate.
 */
int64_t orc_run(int n, double *state, int64_t n_gates, const int *kind, const int *nq,
                const int *qubits, const double *params, const double *ext,
                const int64_t *ext_off, int n_threads)
{
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    int64_t bad = check_gates(n, n_gates, kind, nq, qubits);
    if (bad >= 0) return bad;
    cplx *a = (cplx *)state;
    cplx m[64 * 64];
    for (int64_t g = 0; g < n_gates; g++) {
        int k = gate_arity(kind[g], nq[g]);
        const double *e = ext_off[g] >= 0 ? ext + ext_off[g] : NULL;
        gate_matrix(kind[g], k, params + 3 * g, e, m);
        apply_matrix(n, a, k, qubits + 6 * g, m);
    }
    return -1;
}

/* orc_gate_matrix: expose the gate table (for the pins that test it). */
int orc_gate_matrix(int kind, int nq, const double *params, const double *ext, double *out)
{
    if (kind < O_H || kind > O_DIAG) return -1;
    int k = gate_arity(kind, nq);
    if (k < 1 || k > 6) return -1;
    cplx m[64 * 64];
    int dim = gate_matrix(kind, k, params, ext, m);
    memcpy(out, m, sizeof(cplx) * dim * dim);
    return dim;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
