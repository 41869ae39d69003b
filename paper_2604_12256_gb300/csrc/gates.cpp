// gates.cpp -- gate table of the optimizer: dense matrices for the
// non-diagonal gates and phase polynomials for the diagonal ones.
//
// Section 2.2 (Eqs. 2-3) fixes the amplitude-index convention (qubit j = bit
// j, local matrix bit i <-> q[i]); the matrices are the textbook gates.
// Diagonal gates (Section 4.5: Z, S, T, RZ, P, CZ, CP, RZZ and any matrix
// whose off-diagonal entries are zero with unit-modulus diagonal) become
// phase polynomials so that any number of them fuse exactly.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace svs {

static const double kTwoPi = 6.283185307179586476925286766559;

uint64_t turns_of(double radians)
{
    double f = radians / kTwoPi;
    f -= std::floor(f);
    double s = std::ldexp(f, 64);
    if (!(s < 18446744073709551616.0)) return 0;   // rounds up to a full turn
    return (uint64_t)s;
}

cd phase_of(uint64_t w)
{
    // angle in [-pi, pi) from the signed fixed-point value
    double a = std::ldexp((double)(int64_t)w, -64) * kTwoPi;
    return cd(std::cos(a), std::sin(a));
}

void normalize_terms(std::vector<Term> &t)
{
    std::sort(t.begin(), t.end(), [](const Term &a, const Term &b) { return a.mask < b.mask; });
    std::vector<Term> out;
    for (const Term &x : t) {
        if (!out.empty() && out.back().mask == x.mask) out.back().w += x.w;
        else out.push_back(x);
    }
    out.erase(std::remove_if(out.begin(), out.end(), [](const Term &x) { return x.w == 0; }), out.end());
    t.swap(out);
}

std::vector<cd> diag_matrix(const PGate &g)
{
    int dim = 1 << g.k;
    std::vector<cd> m((size_t)dim * dim, cd(0, 0));
    for (int c = 0; c < dim; c++) {
        uint64_t x = 0;
        for (int i = 0; i < g.k; i++) if ((c >> i) & 1) x |= 1ull << g.q[i];
        uint64_t w = 0;
        for (const Term &t : g.terms) if ((x & t.mask) == t.mask) w += t.w;
        m[(size_t)c * dim + c] = phase_of(w);
    }
    return m;
}

static int fixed_arity(uint32_t kind)
{
    switch (kind) {
    case G_CX: case G_CZ: case G_CP: case G_RZZ: case G_SWAP: return 2;
    case G_UNITARY: case G_DIAG: return -1;
    default: return 1;
    }
}

// Phase polynomial of a diagonal with unit-modulus entries d[c] on qubits q:
// the Moebius transform of the entry phases over subsets of the local bits.
static bool phases_to_terms(int k, const int *q, const std::vector<cd> &d, std::vector<Term> &out)
{
    int dim = 1 << k;
    std::vector<uint64_t> ph(dim);
    for (int c = 0; c < dim; c++) {
        if (std::fabs(std::abs(d[c]) - 1.0) > 1e-12) return false;
        ph[c] = turns_of(std::arg(d[c]));
    }
    for (int i = 0; i < k; i++)
        for (int c = 0; c < dim; c++)
            if ((c >> i) & 1) ph[c] -= ph[c ^ (1 << i)];
    out.clear();
    for (int c = 0; c < dim; c++) {
        if (ph[c] == 0) continue;
        uint64_t m = 0;
        for (int i = 0; i < k; i++) if ((c >> i) & 1) m |= 1ull << q[i];
        out.push_back({m, ph[c]});
    }
    normalize_terms(out);
    return true;
}

bool make_gate(const sim_gate &g, int n, PGate &o, std::string &err)
{
    if (g.kind > G_DIAG) { err = "unknown gate kind " + std::to_string(g.kind); return false; }
    int k = fixed_arity(g.kind);
    if (k < 0) {
        k = (int)g.nq;
        if (k < 1 || k > kMaxGateQubits) { err = "unitary/diag gate needs 1..6 qubits"; return false; }
        if (!g.matrix) { err = "unitary/diag gate without matrix"; return false; }
    } else if (g.nq != 0 && (int)g.nq != k) {
        err = "gate kind " + std::to_string(g.kind) + " takes " + std::to_string(k) + " qubits";
        return false;
    }
    if (g.kind == G_U1Q && !g.matrix) { err = "u1q gate without matrix"; return false; }
    if (k > n) { err = "gate wider than the register"; return false; }
    o = PGate();
    o.kind = (int)g.kind;
    o.k = k;
    for (int i = 0; i < k; i++) {
        if (g.q[i] >= (uint32_t)n) { err = "qubit index out of range"; return false; }
        for (int j = 0; j < i; j++)
            if (g.q[j] == g.q[i]) { err = "repeated qubit in a gate"; return false; }
        o.q[i] = (int)g.q[i];
        o.qmask |= 1ull << g.q[i];
    }
    const double t = g.param[0];
    const int a = o.q[0], b = k > 1 ? o.q[1] : 0;
    const uint64_t A = 1ull << a, B = k > 1 ? (1ull << b) : 0;
    auto dense = [&](std::initializer_list<cd> v) { o.M.assign(v.begin(), v.end()); };
    const double r2 = 0.70710678118654752440084436210485;
    const double c = std::cos(t / 2), s = std::sin(t / 2);
    const cd I(0, 1);
    switch (g.kind) {
    case G_H: dense({r2, r2, r2, -r2}); break;
    case G_X: dense({0, 1, 1, 0}); break;
    case G_Y: dense({0, -I, I, 0}); break;
    case G_RX: dense({c, -I * s, -I * s, c}); break;
    case G_RY: dense({c, -s, s, c}); break;
    case G_CX:   // local index b0 + 2 b1, b0 = control: swaps |01> and |11>
        dense({1, 0, 0, 0, 0, 0, 0, 1, 0, 0, 1, 0, 0, 1, 0, 0}); break;
    case G_SWAP:
        o.swap = true;
        dense({1, 0, 0, 0, 0, 0, 1, 0, 0, 1, 0, 0, 0, 0, 0, 1}); break;
    case G_Z: o.diag = true; o.terms = {{A, 1ull << 63}}; break;
    case G_S: o.diag = true; o.terms = {{A, 1ull << 62}}; break;
    case G_T: o.diag = true; o.terms = {{A, 1ull << 61}}; break;
    case G_RZ: o.diag = true; o.terms = {{0, turns_of(-t / 2)}, {A, turns_of(t)}}; break;
    case G_P: o.diag = true; o.terms = {{A, turns_of(t)}}; break;
    case G_CZ: o.diag = true; o.terms = {{A | B, 1ull << 63}}; break;
    case G_CP: o.diag = true; o.terms = {{A | B, turns_of(t)}}; break;
    case G_RZZ:   // -t/2 + t (x_a XOR x_b) = -t/2 + t x_a + t x_b - 2t x_a x_b
        o.diag = true;
        o.terms = {{0, turns_of(-t / 2)}, {A, turns_of(t)}, {B, turns_of(t)}, {A | B, turns_of(-2 * t)}};
        break;
    case G_U1Q:
    case G_UNITARY: {
        int dim = 1 << k;
        o.M.resize((size_t)dim * dim);
        for (int i = 0; i < dim * dim; i++) o.M[i] = cd(g.matrix[2 * i], g.matrix[2 * i + 1]);
        bool isdiag = true;
        for (int r = 0; r < dim && isdiag; r++)
            for (int cc = 0; cc < dim; cc++)
                if (r != cc && o.M[(size_t)r * dim + cc] != cd(0, 0)) { isdiag = false; break; }
        if (isdiag) {
            std::vector<cd> d(dim);
            for (int r = 0; r < dim; r++) d[r] = o.M[(size_t)r * dim + r];
            if (phases_to_terms(k, o.q, d, o.terms)) { o.diag = true; o.M.clear(); }
        }
        break;
    }
    case G_DIAG: {
        int dim = 1 << k;
        std::vector<cd> d(dim);
        for (int i = 0; i < dim; i++) d[i] = cd(g.matrix[2 * i], g.matrix[2 * i + 1]);
        if (phases_to_terms(k, o.q, d, o.terms)) {
            o.diag = true;
        } else {   // not a phase: keep it as a dense (diagonal) matrix
            o.M.assign((size_t)dim * dim, cd(0, 0));
            for (int i = 0; i < dim; i++) o.M[(size_t)i * dim + i] = d[i];
        }
        break;
    }
    default: err = "unhandled gate kind"; return false;
    }
    if (o.diag) normalize_terms(o.terms);
    return true;
}

}  // namespace svs
