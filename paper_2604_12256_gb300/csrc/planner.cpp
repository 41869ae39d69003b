// planner.cpp -- the host optimizer (swarm optimization, Algorithm 4):
//
//   1. ingest + validate the gate list (Section 4.1's `circuit`);
//   2. diagonal detector (Algorithm 8) with the readings listed below;
//   3. merge booster (Algorithms 6-7) for product initial states;
//   4. gate-block search (GBSA mode 0, Algorithm 2's cache blocking) fused
//      with register-stage scheduling, lazy placement of diagonal phases and
//      cost-based gate fusion (GBSA mode 1);
//   5. encoding of each block as a device program (program.h), and of runs
//      of dense 5-qubit blocks as cache-blocked tensor-core sweeps
//      (dense_prog.h).
//
// Readings of the diagonal detector (Algorithm 8), restated from the
// commutation rule it rests on (see diagonal_detector):
//   (i)   a group of one diagonal gate is emitted unchanged;
//   (ii)  no gate passes a gate it does not commute with;
//   (iii) the D bound of Section 4.1 caps a group's qubit set (D = 0:
//         unbounded, the phase-polynomial form needs no table);
//   (iv)  a diagonal gate joins the oldest group it can reach.
// GBSA itself is unspecified (Section 4.2 builds on prior simulators); ours is
// a greedy scan in dependency order (Scheduler, and group_dense_chunks for
// dense blocks).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <sstream>
#include <unordered_map>

#include "dense_prog.h"
#include "internal.h"
#include "program.h"

namespace svs {

static inline int popc(uint64_t x) { return __builtin_popcountll(x); }

void fill_default_options(sim_options &o)
{
    std::memset(&o, 0, sizeof(o));
    o.max_fuse_qubits = 2;
    o.max_diag_qubits = 0;
    o.chunk_qubits = 0;
    o.booster_div = 0;
    o.flags = SIM_F_DIAG | SIM_F_BOOST | SIM_F_BLOCK | SIM_F_FUSE;
    o.dense_precision = SIM_DENSE_SPLIT_TF32;
    o.max_stages = 4;
}

// Instantiated chunk kernels: (C, RB) = (12,5) / (10,5) / (12,4) for
// complex64 and (11,4) / (9,4) for complex128.
static bool chunk_shape(int n, sim_dtype dt, int want_c, int want_rb, int &C, int &RB)
{
    if (dt == SIM_C64) {
        if (want_rb != 5 && n >= 12 && (want_c <= 0 || want_c >= 12)) {
            C = 12;
            RB = 4;
            return true;
        }
        RB = 5;
        // 2^13-amplitude chunks (256 threads) only when asked for
        int cands[3] = {13, 12, 10};
        for (int c : cands)
            if (c <= n && (c == 13 ? want_c == 13 : (want_c <= 0 || c <= want_c))) { C = c; return true; }
    } else {
        RB = 4;
        int cands[2] = {11, 9};
        for (int c : cands)
            if (c <= n && (want_c <= 0 || c <= want_c)) { C = c; return true; }
    }
    return false;
}

void resolve_options(sim_options &o, int n, sim_dtype dt)
{
    if (o.max_fuse_qubits < 1) o.max_fuse_qubits = 1;
    if (o.max_fuse_qubits > 3) o.max_fuse_qubits = 3;
    if (o.max_stages < 1) o.max_stages = 1;
    if (o.max_stages > prog::kMaxStages) o.max_stages = prog::kMaxStages;
    if (o.max_diag_qubits < 0) o.max_diag_qubits = 0;
    // dense-block mode: fused diagonals must fit a 5-qubit block
    if ((o.flags & SIM_F_TC) && (o.max_diag_qubits == 0 || o.max_diag_qubits > 5)) o.max_diag_qubits = 5;
    (void)n;
    (void)dt;
}

// ------------------------------------------------------------ helpers
static std::vector<cd> matmul(const std::vector<cd> &A, const std::vector<cd> &B, int dim)
{
    std::vector<cd> C((size_t)dim * dim, cd(0, 0));
    for (int r = 0; r < dim; r++)
        for (int k = 0; k < dim; k++) {
            cd a = A[(size_t)r * dim + k];
            if (a == cd(0, 0)) continue;
            for (int c = 0; c < dim; c++) C[(size_t)r * dim + c] += a * B[(size_t)k * dim + c];
        }
    return C;
}

// Expand a matrix on positions `pos` (local bit i <-> pos[i]) to the
// positions `upos` (a superset), identity on the extra ones.
static std::vector<cd> expand(const std::vector<cd> &M, int k, const int *pos, int ku, const int *upos)
{
    int du = 1 << ku, d = 1 << k;
    int where[kMaxGateQubits];
    for (int i = 0; i < k; i++)
        for (int j = 0; j < ku; j++) if (upos[j] == pos[i]) where[i] = j;
    uint32_t inmask = 0;
    for (int i = 0; i < k; i++) inmask |= 1u << where[i];
    std::vector<cd> E((size_t)du * du, cd(0, 0));
    for (int r = 0; r < du; r++)
        for (int c = 0; c < du; c++) {
            if ((r & ~inmask) != (c & ~inmask)) continue;
            int lr = 0, lc = 0;
            for (int i = 0; i < k; i++) {
                lr |= ((r >> where[i]) & 1) << i;
                lc |= ((c >> where[i]) & 1) << i;
            }
            E[(size_t)r * du + c] = M[(size_t)lr * d + lc];
        }
    return E;
}

// ------------------------------------------------------------ diagonal detector
// Section 4.5 (Algorithm 8), restated from the rule it rests on: a diagonal
// gate commutes with every other diagonal gate and with every gate on other
// qubits.  A diagonal gate may therefore move back past any run of gates
// that holds no non-diagonal gate on one of its qubits, and merge with a
// diagonal group there; the fused group is one gate whose phase polynomial
// is the sum of its members' polynomials (diagonals multiply).
//
// One pass builds the output.  Each diagonal group in it records its
// "walls": the qubits of the non-diagonal gates emitted after it.  Walls only
// grow, and an older group's walls contain a newer one's, so the groups a
// gate can reach are the newest ones.  A diagonal gate joins the oldest group
// whose walls miss its qubits and whose qubit set stays within D (D = 0: no
// bound, reading (iii)); otherwise it starts a group.  A group of one gate is
// emitted as that gate (reading (i)).  Non-diagonal gates keep their order,
// and no gate passes a gate it does not commute with (reading (ii)).
namespace {
struct DiagGroup {
    size_t slot;            // its place in the output
    uint64_t qubits = 0;    // qubits of its members
    uint64_t walls = 0;     // qubits of non-diagonal gates emitted after it
    std::vector<size_t> members;
};
}  // namespace

static std::vector<PGate> diagonal_detector(const std::vector<PGate> &G, int D, uint64_t &absorbed)
{
    // output slots: a gate of G (>= 0) or a group (-1 - group index)
    std::vector<long> slots;
    std::vector<DiagGroup> groups;
    size_t live = 0;   // groups before this index can no longer be reached
    slots.reserve(G.size());
    uint64_t all = 0;   // every qubit the circuit touches
    for (const PGate &x : G) all |= x.qmask;
    for (size_t t = 0; t < G.size(); t++) {
        const PGate &g = G[t];
        if (!g.diag) {
            slots.push_back((long)t);
            for (size_t k = live; k < groups.size(); k++) groups[k].walls |= g.qmask;
            // the oldest live groups whose walls already hold every qubit of
            // the circuit can take nothing more
            while (live < groups.size() && (groups[live].walls & all) == all) live++;
            continue;
        }
        bool joined = false;
        for (size_t k = live; k < groups.size() && !joined; k++) {
            DiagGroup &grp = groups[k];
            if (grp.walls & g.qmask) continue;
            if (D > 0 && popc(grp.qubits | g.qmask) > D) continue;
            grp.qubits |= g.qmask;
            grp.members.push_back(t);
            joined = true;
        }
        if (!joined) {
            DiagGroup grp;
            grp.slot = slots.size();
            grp.qubits = g.qmask;
            grp.members.push_back(t);
            slots.push_back(-1 - (long)groups.size());
            groups.push_back(std::move(grp));
        }
    }
    std::vector<PGate> res;
    res.reserve(slots.size());
    absorbed = 0;
    for (long sl : slots) {
        if (sl >= 0) {
            res.push_back(G[(size_t)sl]);
            continue;
        }
        const DiagGroup &grp = groups[(size_t)(-1 - sl)];
        if (grp.members.size() == 1) {
            res.push_back(G[grp.members[0]]);
            continue;
        }
        PGate f;
        f.kind = kFusedDiag;
        f.diag = true;
        f.qmask = grp.qubits;
        f.k = popc(grp.qubits);
        f.n_src = 0;
        for (size_t m : grp.members) {
            f.terms.insert(f.terms.end(), G[m].terms.begin(), G[m].terms.end());
            f.n_src += G[m].n_src;
        }
        normalize_terms(f.terms);
        absorbed += grp.members.size() - 1;
        res.push_back(std::move(f));
    }
    return res;
}

// ------------------------------------------------------------ merge booster
// Divider of Algorithm 6: split N into halves (ceil on the second half)
// until every part is <= divSize; parts are queued low qubits first.
static void divider(int N, int divSize, std::vector<int> &que)
{
    if (N <= divSize) { que.push_back(N); return; }
    divider(N >> 1, divSize, que);
    int M = (N & 1) ? N + 1 : N;
    divider(M >> 1, divSize, que);
}

// Gates of `pend` that lie inside [lo, lo+w) and are not preceded by a left-out
// gate on one of their qubits (a dependency-closed prefix: reading of
// genGateBlock).  Taken gates are removed from `pend`.
static std::vector<PGate> take_group(std::vector<PGate> &pend, int lo, int w)
{
    uint64_t grp = (w >= 64 ? ~0ull : ((1ull << w) - 1)) << lo;
    uint64_t blocked = 0;
    std::vector<PGate> taken, keep;
    for (PGate &g : pend) {
        if ((g.qmask & ~grp) == 0 && (g.qmask & blocked) == 0) taken.push_back(std::move(g));
        else { blocked |= g.qmask; keep.push_back(std::move(g)); }
    }
    pend.swap(keep);
    return taken;
}

static PGate shift_gate(const PGate &g, int lo)
{
    PGate s = g;
    s.qmask = g.qmask >> lo;
    for (int i = 0; i < g.k && i < kMaxGateQubits; i++) s.q[i] = g.q[i] - lo;
    for (Term &t : s.terms) t.mask >>= lo;
    return s;
}

// ------------------------------------------------------------ encoding
struct ProgWriter {
    std::vector<uint32_t> w;
    void put(uint32_t v) { w.push_back(v); }
    void put64(uint64_t v) { w.push_back((uint32_t)v); w.push_back((uint32_t)(v >> 32)); }
    void align2() { if (w.size() & 1) w.push_back(0); }
    void align4() { while (w.size() & 3) w.push_back(0); }
    // pad the op that starts at `start` to a multiple of 4 words and record
    // its length (ops start 2 words before a 16-byte boundary)
    void end_op(size_t start)
    {
        while ((w.size() - start) & 3) w.push_back(0);
        w[start + prog::O_WORDS] = (uint32_t)(w.size() - start);
    }
};

static inline uint64_t qweight(uint64_t w, bool f64)
{
    if (f64) return w;
    return (uint64_t)(uint32_t)((w + (1ull << 31)) >> 32);
}

// A stage as scheduled: register positions and ops, in the physical frame
// of the block's load.
struct SOp {
    int type = 0;              // 1 dense, 2 phase
    int k = 0;
    int pos[kMaxGateQubits] = {0};
    uint64_t pmask = 0;
    std::vector<cd> M;
    std::vector<Term> terms;
    int n_src = 0;
};
struct SStage {
    uint64_t R = 0;            // physical positions used as register bits
    std::vector<SOp> ops;
};

// Choose lane bits (first 5 thread bits) with distinct residues modulo the
// swizzle width so that shared-memory accesses are bank-conflict free.
static void stage_layout(int C, int RB, int swz, const std::vector<int> &need_reg, int *reg, int *thr)
{
    std::vector<char> used(C, 0);
    int nr = 0;
    for (int b : need_reg) { reg[nr++] = b; used[b] = 1; }
    int T = C - RB;
    std::vector<int> lanes;
    int nl = std::min(5, T);
    for (int r = 0; r < swz && (int)lanes.size() < nl; r++)
        for (int b = 0; b < C; b++)
            if (!used[b] && b % swz == r) { lanes.push_back(b); used[b] = 1; break; }
    for (int b = 0; b < C && (int)lanes.size() < nl; b++)
        if (!used[b]) { lanes.push_back(b); used[b] = 1; }
    // pad registers with the highest free bits, keep low bits for warps
    for (int b = C - 1; b >= 0 && nr < RB; b--)
        if (!used[b]) { reg[nr++] = b; used[b] = 1; }
    int nt = 0;
    for (int b : lanes) thr[nt++] = b;
    for (int b = 0; b < C; b++)
        if (!used[b]) { thr[nt++] = b; used[b] = 1; }
}

// A direct layout (program.h) for a stage that needs register bits
// `need_reg`, if there is one.  Paired (a 16-byte access per two
// amplitudes) when qubit 0 is needed or a register bit is left for it:
// register bit 0 = chunk bit 0, lanes 0..2 = chunk bits 1..3, lane 3 a bit
// of the remaining swizzle residue (no shared-memory bank conflicts).
// Otherwise unpaired (8-byte accesses): lanes 0..3 = chunk bits 0..3.  The
// other register bits are the needed ones, then the highest free bits; the
// other thread bits the free ones in ascending order.
static bool direct_layout(int C, int RB, int swz, const std::vector<int> &need_reg, int *reg, int *thr)
{
    if (C - RB < 5 || RB < 2) return false;
    int nhigh = 0;
    bool has0 = false;
    for (int b : need_reg) {
        if (b >= 1 && b <= 3) return false;   // qubits 1..3 are lanes
        if (b == 0) has0 = true;
        else nhigh++;
    }
    // paired needs a free bit of residue 0 for lane 3 (bits 1..3 have
    // residues 1..3); without one the unpaired form is conflict-free
    bool free0 = false;
    for (int b = swz; b < C; b += swz) {
        bool taken = false;
        for (int x : need_reg) taken = taken || x == b;
        free0 = free0 || !taken;
    }
    const bool paired = has0 || (nhigh <= RB - 1 && free0);
    if (has0 && nhigh > RB - 1) return false;
    std::vector<char> used(C, 0);
    int nr = 0;
    if (paired) {
        reg[nr++] = 0;
        used[0] = 1;
    }
    for (int b : need_reg)
        if (b != 0) {
            reg[nr++] = b;
            used[b] = 1;
        }
    std::vector<int> lanes;
    for (int b = paired ? 1 : 0; b <= 3; b++) {
        lanes.push_back(b);
        used[b] = 1;
    }
    for (int b = 4; b < C && lanes.size() < 4; b++)
        if (!used[b] && b % swz == 0) { lanes.push_back(b); used[b] = 1; }
    for (int b = C - 1; b >= 4 && nr < RB; b--)
        if (!used[b]) { reg[nr++] = b; used[b] = 1; }
    if (nr < RB) return false;
    const int nl = std::min(5, C - RB);
    for (int b = 0; b < C && (int)lanes.size() < nl; b++)
        if (!used[b]) { lanes.push_back(b); used[b] = 1; }
    int nt = 0;
    for (int b : lanes) thr[nt++] = b;
    for (int b = 0; b < C; b++)
        if (!used[b]) { thr[nt++] = b; used[b] = 1; }
    return nt == C - RB;
}

// Context of one phase segment: where the register and thread bits sit in
// this stage, the segment's number and the launch-wide term tables.
struct DsegCtx {
    int RB = 0, TB = 0;
    bool f64 = false;
    const uint64_t *regphys = nullptr;   // physical bit of register bit j
    const int *gthr = nullptr;           // physical qubit of thread bit i
    uint64_t freem = 0;                  // chunk-selecting qubits
    int d = 0;                           // segment number
    bool hoist = false;                  // thread-only terms go to the thread table
    std::vector<uint32_t> *cta = nullptr, *thr = nullptr;
};

// A real as a double-float pair (hi = nearest float, lo = nearest float of
// the rest): complex128 constants of chunk programs, as the kernels use them.
static void put_df(ProgWriter &pw, long double v)
{
    const float h = (float)v;
    const float l = (float)(v - (long double)h);
    uint32_t a, b;
    std::memcpy(&a, &h, 4);
    std::memcpy(&b, &l, 4);
    pw.put(a);
    pw.put(b);
}

// Split a segment's terms: slot terms (no register bit: slot 0; one register
// bit j: slot 1 + j) go to the CTA table when they only test chunk-selecting
// qubits, to the thread table when they only test thread bits (and the
// segment is hoisted), else stay in the body; a slot-0 term on
// chunk-selecting qubits and one thread bit i goes to the CTA table as a
// coefficient of bit i (slot 1 + RB + i); a term on one register bit alone
// is a constant CTA-table entry of its slot; terms on several register bits
// only fold into the 2^RB table; other terms with several register bits stay
// in the body.
static void encode_dseg(ProgWriter &pw, const std::vector<Term> &terms, const DsegCtx &cx)
{
    const int RB = cx.RB;
    const bool f64 = cx.f64;
    uint64_t regall = 0, thrall = 0;
    for (int j = 0; j < RB; j++) regall |= cx.regphys[j];
    for (int i = 0; i < cx.TB; i++) thrall |= 1ull << cx.gthr[i];
    std::vector<Term> base;
    std::vector<std::vector<Term>> lin(RB);
    std::vector<std::pair<Term, uint32_t>> multi;
    std::vector<uint64_t> tab(1u << RB, 0);
    uint32_t tabmask = 0;   // entries of tab that register-only terms reach
    const uint32_t S = 1 + RB, SCP = prog::cta_stride(RB, cx.TB, f64 ? 8 : 4);
    auto to_tables = [&](uint32_t slot, uint64_t nonreg, uint64_t w) {
        uint64_t mt = nonreg & thrall;
        const uint64_t mc = nonreg & ~thrall;
        if (slot == 0 && mt != 0 && mc != 0 && popc(mt) == 1) {
            int i = 0;
            while (i < cx.TB && (1ull << cx.gthr[i]) != mt) i++;
            if (i < cx.TB) {
                slot = 1 + RB + i;
                mt = 0;
            }
        }
        if (mt == 0) {
            cx.cta->push_back(cx.d * SCP + slot);
            cx.cta->push_back(0);
            cx.cta->push_back((uint32_t)mc);
            cx.cta->push_back((uint32_t)(mc >> 32));
            uint64_t q = qweight(w, f64);
            cx.cta->push_back((uint32_t)q);
            cx.cta->push_back((uint32_t)(q >> 32));
            return true;
        }
        if (mc == 0 && cx.hoist) {
            uint32_t tm = 0;
            for (int i = 0; i < cx.TB; i++) if ((mt >> cx.gthr[i]) & 1) tm |= 1u << i;
            cx.thr->push_back(cx.d * S + slot);
            cx.thr->push_back(tm);
            uint64_t q = qweight(w, f64);
            cx.thr->push_back((uint32_t)q);
            cx.thr->push_back((uint32_t)(q >> 32));
            return true;
        }
        return false;
    };
    uint32_t common = (1u << RB) - 1;
    for (const Term &t : terms) {
        uint32_t rm = 0;
        for (int j = 0; j < RB; j++) if (t.mask & cx.regphys[j]) rm |= 1u << j;
        common &= rm;
        uint64_t nonreg = t.mask & ~regall;
        if (rm == 0) {
            if (!to_tables(0, nonreg, t.w)) base.push_back({nonreg, t.w});
        } else if (nonreg == 0 && popc(rm) == 1) {
            // a phase on one register bit alone: a constant part of lin[j]
            // (a CTA-table entry whose mask is always met)
            to_tables(1 + __builtin_ctz(rm), 0, t.w);
        } else if (nonreg == 0) {
            for (uint32_t m = 0; m < (1u << RB); m++)
                if ((m & rm) == rm) {
                    tab[m] += t.w;
                    if (RB <= 5) tabmask |= 1u << m;
                }
        } else if (popc(rm) == 1) {
            int j = __builtin_ctz(rm);
            if (!to_tables(1 + j, nonreg, t.w)) lin[j].push_back({nonreg, t.w});
        } else {
            multi.push_back({{nonreg, t.w}, rm});
        }
    }
    // a register bit shared by every term: amplitudes without it keep phase 0
    const int pivot = terms.empty() || common == 0 ? -1 : __builtin_ctz(common);
    bool tabnz = false;
    for (uint64_t x : tab) if (qweight(x, f64) != 0) tabnz = true;
    size_t start = pw.w.size();
    pw.put(prog::OP_DSEG);
    pw.put(0);   // words, patched below
    pw.put((uint32_t)cx.d);
    pw.put(tabnz ? 1u : 0u);
    pw.put((uint32_t)base.size());
    pw.put((uint32_t)multi.size());
    for (int j = 0; j < prog::kMaxRB; j++) pw.put(j < RB ? (uint32_t)lin[j].size() : 0);
    pw.put((uint32_t)pivot);
    pw.put(RB <= 5 ? tabmask : 0xffffffffu);
    pw.put(0);
    pw.put(0);
    auto put_term = [&](const Term &t) {
        pw.put64(t.mask);
        pw.put64(qweight(t.w, f64));
    };
    for (const Term &t : base) put_term(t);
    for (int j = 0; j < RB; j++)
        for (const Term &t : lin[j]) put_term(t);
    for (uint32_t m = 0; m < (1u << RB); m++) pw.put64(qweight(tab[m], f64));
    // the same phases as complex factors (the kernels multiply by them instead
    // of evaluating a sin/cos per amplitude)
    for (uint32_t m = 0; m < (1u << RB); m++) {
        const uint64_t q = qweight(tab[m], f64);
        if (q == 0) {   // cis(0) = (1, +0) exactly: no long-double sin/cos
            if (f64) {
                put_df(pw, 1.0L);
                put_df(pw, 0.0L);
            } else {
                pw.put(0x3f800000u);   // 1.0f
                pw.put(0u);            // +0.0f
            }
            continue;
        }
        const long double th = 6.283185307179586476925286766559L *
                               (f64 ? (long double)q * 0x1p-64L : (long double)(uint32_t)q * 0x1p-32L);
        if (f64) {
            put_df(pw, cosl(th));
            put_df(pw, sinl(th));
        } else {
            const float c = (float)cosl(th), sn = (float)sinl(th);
            uint32_t a, b;
            std::memcpy(&a, &c, 4);
            std::memcpy(&b, &sn, 4);
            pw.put(a);
            pw.put(b);
        }
    }
    for (auto &mt : multi) {
        pw.put64(mt.first.mask);
        pw.put(mt.second);
        pw.put(0);
        pw.put64(qweight(mt.first.w, f64));
    }
    pw.end_op(start);
}

static void encode_dense(ProgWriter &pw, const SOp &op, const int *reg, const int *qin, int RB, bool f64)
{
    // register index of each of the op's positions
    int ri[kMaxGateQubits];
    for (int i = 0; i < op.k; i++) {
        ri[i] = -1;
        for (int j = 0; j < RB; j++) if (qin[reg[j]] == op.pos[i]) ri[i] = j;
    }
    // ascending register order; local bit i' of the new matrix <-> sorted[i']
    int order[kMaxGateQubits];
    for (int i = 0; i < op.k; i++) order[i] = i;
    std::sort(order, order + op.k, [&](int a, int b) { return ri[a] < ri[b]; });
    int dim = 1 << op.k;
    std::vector<cd> M2((size_t)dim * dim);
    auto remap = [&](int l) {
        int o = 0;
        for (int i2 = 0; i2 < op.k; i2++) o |= ((l >> order[i2]) & 1) << i2;
        return o;
    };
    for (int r = 0; r < dim; r++)
        for (int c = 0; c < dim; c++) M2[(size_t)remap(r) * dim + remap(c)] = op.M[(size_t)r * dim + c];
    uint32_t code = 0;
    for (int i2 = 0; i2 < op.k; i2++) code |= (uint32_t)ri[order[i2]] << (3 * i2);
    // 2x2 structure after rounding to the state precision: all-real entries
    // (H, RY) or real diagonal with imaginary off-diagonal (RX) need half the
    // arithmetic of a general complex matrix
    uint32_t sub = prog::DS_GENERAL;
    if (op.k == 1) {
        auto rz = [&](double v) { return f64 ? v == 0.0 : (float)v == 0.0f; };
        bool real = true, rx = true;
        for (int i = 0; i < 4; i++) {
            if (!rz(M2[i].imag())) real = false;
            bool diag = (i == 0 || i == 3);
            if (diag ? !rz(M2[i].imag()) : !rz(M2[i].real())) rx = false;
        }
        sub = real ? prog::DS_REAL : rx ? prog::DS_RX : prog::DS_GENERAL;
    }
    size_t start = pw.w.size();
    pw.put(prog::OP_DENSE | (uint32_t)op.k << 8 | sub << 12 | code << 16);
    pw.put(0);
    for (const cd &z : M2) {
        if (f64) {
            put_df(pw, z.real());   // the chunk kernel computes complex128 in double-float
            put_df(pw, z.imag());
        } else {
            float re = (float)z.real(), im = (float)z.imag();
            uint32_t a, b;
            std::memcpy(&a, &re, 4);
            std::memcpy(&b, &im, 4);
            pw.put(a);
            pw.put(b);
        }
    }
    pw.end_op(start);
}

// shared-memory budget of the per-thread term table of one launch
constexpr size_t kThreadTableBytes = 24 * 1024;

// Encode one cache-blocked pass.  Q: physical chunk positions (popcount C);
// lam_end[p]: logical qubit held by position p at the end of the block
// (identity off the chunk); forced_layout: the K3 diagonal sweep's layout.
static std::vector<uint32_t> encode_program(int n, int C, int RB, bool f64, uint64_t Q,
                                            const std::vector<SStage> &stages, const int *lam_end,
                                            bool forced_layout)
{
    int qin[prog::kMaxC];
    int nc = 0;
    for (int p = 0; p < n; p++) if ((Q >> p) & 1) qin[nc++] = p;
    ProgWriter pw;
    pw.w.assign(prog::H_SIZE, 0);
    pw.w[prog::H_MAGIC] = prog::kMagic;
    pw.w[prog::H_C] = (uint32_t)C;
    pw.w[prog::H_RB] = (uint32_t)RB;
    pw.w[prog::H_NSTAGE] = (uint32_t)stages.size();
    pw.w[prog::H_N] = (uint32_t)n;
    pw.w[prog::H_WBYTES] = f64 ? 8 : 4;
    uint64_t nmask = n >= 64 ? ~0ull : ((1ull << n) - 1);
    uint64_t freem = nmask & ~Q;
    pw.w[prog::H_FREE_LO] = (uint32_t)freem;
    pw.w[prog::H_FREE_HI] = (uint32_t)(freem >> 32);
    for (int i = 0; i < C; i++) pw.w[prog::H_QIN + i] = (uint32_t)qin[i];
    for (int i2 = 0; i2 < C; i2++) {
        int src = i2;
        for (int i = 0; i < C; i++) if (lam_end[qin[i]] == qin[i2]) src = i;
        pw.w[prog::H_SPERM + i2] = (uint32_t)src;
    }
    const int swz = prog::swizzle_bits(f64 ? 8 : 4);
    // direct boundary stages (complex64, the lowest 4 qubits in the chunk)
    bool low4 = !f64 && C >= 4;
    for (int i = 0; i < 4 && low4; i++) low4 = qin[i] == i;
    bool sperm_id = true;
    for (int i = 0; i < C; i++) sperm_id = sperm_id && pw.w[prog::H_SPERM + i] == (uint32_t)i;
    uint32_t direct = 0;
    // phase segments whose thread-only terms are summed once per launch:
    // as many as fit the shared-memory budget of the thread table
    int nseg = 0;
    for (const SStage &st : stages)
        for (const SOp &op : st.ops) nseg += op.type == 2;
    const size_t per_seg = (size_t)(1 + RB) * ((size_t)1 << (C - RB)) * (f64 ? 8 : 4);
    const int nhoist = (int)std::min<size_t>((size_t)nseg, kThreadTableBytes / per_seg);
    int nd = 0;
    std::vector<uint32_t> cta, thr_t;
    for (size_t s = 0; s < stages.size(); s++) {
        const SStage &st = stages[s];
        pw.align4();
        size_t sstart = pw.w.size();
        pw.w[prog::H_STAGE_OFF + s] = (uint32_t)sstart;
        int reg[prog::kMaxRB] = {0}, thr[prog::kMaxC] = {0};
        if (forced_layout) {
            for (int j = 0; j < RB; j++) reg[j] = C - RB + j;
            for (int i = 0; i < C - RB; i++) thr[i] = i;
        } else {
            std::vector<int> need;
            for (int i = 0; i < C; i++) if ((st.R >> qin[i]) & 1) need.push_back(i);
            const bool first = s == 0, last = s + 1 == stages.size() && sperm_id;
            if ((first || last) && low4 && direct_layout(C, RB, swz, need, reg, thr)) {
                if (first) direct |= prog::DIRECT_FIRST;
                if (last) direct |= prog::DIRECT_LAST;
            } else {
                stage_layout(C, RB, swz, need, reg, thr);
            }
        }
        pw.w.resize(sstart + prog::S_SIZE, 0);
        pw.w[sstart + prog::S_NOPS] = (uint32_t)st.ops.size();
        for (int j = 0; j < prog::kMaxRB; j++) pw.w[sstart + prog::S_REG + j] = j < RB ? (uint32_t)reg[j] : 0;
        for (int i = 0; i < prog::kMaxC; i++) pw.w[sstart + prog::S_THR + i] = i < C - RB ? (uint32_t)thr[i] : 0;
        for (int i = 0; i < prog::kMaxC; i++)
            pw.w[sstart + prog::S_GTHR + i] = i < C - RB ? (uint32_t)qin[thr[i]] : 0;
        for (int j = 0; j < prog::kMaxRB; j++)
            pw.w[sstart + prog::S_PV + j] = j < RB ? prog::swizzle(1u << reg[j], C, swz) : 0;
        uint64_t regphys[prog::kMaxRB];
        for (int j = 0; j < RB; j++) regphys[j] = 1ull << qin[reg[j]];
        int gthr[prog::kMaxC];
        for (int i = 0; i < C - RB; i++) gthr[i] = qin[thr[i]];
        for (const SOp &op : st.ops) {
            if (op.type == 1) {
                encode_dense(pw, op, reg, qin, RB, f64);
            } else {
                DsegCtx cx;
                cx.RB = RB;
                cx.TB = C - RB;
                cx.f64 = f64;
                cx.regphys = regphys;
                cx.gthr = gthr;
                cx.freem = freem;
                cx.d = nd;
                cx.hoist = nd < nhoist;
                cx.cta = &cta;
                cx.thr = &thr_t;
                encode_dseg(pw, op.terms, cx);
                nd++;
            }
        }
        pw.align2();
        pw.w[sstart + prog::S_WORDS] = (uint32_t)(pw.w.size() - sstart);
    }
    pw.align2();
    pw.w[prog::H_NDSEG] = (uint32_t)nd;
    pw.w[prog::H_NHOIST] = (uint32_t)nhoist;
    pw.w[prog::H_DIRECT] = direct;
    pw.w[prog::H_CTA_OFF] = (uint32_t)pw.w.size();
    pw.w[prog::H_NCTA] = (uint32_t)(cta.size() / prog::kCtaWords);
    pw.w.insert(pw.w.end(), cta.begin(), cta.end());
    pw.w[prog::H_THR_OFF] = (uint32_t)pw.w.size();
    pw.w[prog::H_NTHR] = (uint32_t)(thr_t.size() / prog::kThrWords);
    pw.w.insert(pw.w.end(), thr_t.begin(), thr_t.end());
    pw.align2();
    pw.w[prog::H_WORDS] = (uint32_t)pw.w.size();
    return pw.w;
}

// ------------------------------------------------------------ scheduling
struct Cfg {
    int C, RB, L, F, Smax;
    bool fuse;
    bool f64;
    bool remap = true;   // qubit reordering through the block stores
};

struct PendingDiag {
    uint64_t mask;             // physical positions
    std::vector<Term> terms;   // physical masks
    int n_src;
};

// dense ops applied inside a chunk pass have at most this many qubits
constexpr int kChunkMaxK = 2;
constexpr int kChunkMaxKEncoded = 2;   // arities the chunk kernel dispatches

static int dense_cost(int k) { return k == 1 ? 8 : k == 2 ? 16 : k == 3 ? 48 : 1 << 12; }

struct Scheduler {
    const std::vector<PGate> &G;
    int n;
    Cfg cfg;
    Plan &plan;
    int buf;
    std::vector<char> done;
    std::vector<PendingDiag> pending;
    // Qubit frame (Section 2.3): laminv[q] = position holding logical qubit q,
    // at[p] = logical qubit held by position p.  It persists across blocks:
    // a block's store may move the qubits the next block needs first into the
    // low positions (choose_frame).  lam[p] = where the block's store writes
    // the data it loaded from position p (identity off the block).
    int lam[64], laminv[64], at[64];
    int last_chunk_op = -1;
    std::vector<SStage> last_stages;
    uint64_t last_Q = 0;
    int last_lam[64], last_at[64];
    int blk_pos[64];   // laminv when the current block began

    Scheduler(const std::vector<PGate> &g, int n_, Cfg c, Plan &p, int b) : G(g), n(n_), cfg(c), plan(p), buf(b)
    {
        done.assign(G.size(), 0);
        for (int i = 0; i < 64; i++) lam[i] = laminv[i] = at[i] = i;
    }

    uint64_t phys(uint64_t lm) const
    {
        uint64_t r = 0;
        while (lm) { int q = __builtin_ctzll(lm); lm &= lm - 1; r |= 1ull << laminv[q]; }
        return r;
    }

    // A ready diagonal gate is split into its monomials: each monomial is a
    // diagonal operator on its own qubits only, so it commutes with every gate
    // that misses them and is flushed just before the first gate that does
    // not (the global-phase monomial floats to the end of the circuit).
    void make_pending(const PGate &g)
    {
        for (const Term &t : g.terms) {
            PendingDiag d;
            d.mask = phys(t.mask);
            d.n_src = 0;
            d.terms.push_back({d.mask, t.w});
            pending.push_back(std::move(d));
        }
    }

    // take the pending diagonals meeting `pm` into one phase op
    bool flush(uint64_t pm, SOp &out)
    {
        out = SOp();
        out.type = 2;
        bool any = false;
        std::vector<PendingDiag> keep;
        for (PendingDiag &d : pending) {
            if (d.mask & pm) {
                out.terms.insert(out.terms.end(), d.terms.begin(), d.terms.end());
                out.pmask |= d.mask;
                out.n_src += d.n_src;
                any = true;
            } else {
                keep.push_back(std::move(d));
            }
        }
        pending.swap(keep);
        normalize_terms(out.terms);
        return any;
    }

    bool pending_meets(uint64_t pm) const
    {
        for (const PendingDiag &d : pending)
            if (d.mask & pm) return true;
        return false;
    }

    static bool meets(const SOp &x, uint64_t pm)
    {
        if (x.type == 1) return (x.pmask & pm) != 0;
        for (const Term &t : x.terms) if (t.mask & pm) return true;
        return false;
    }

    // cost-based fusion (GBSA mode 1): merge `op` into an earlier dense op of
    // the stage that it can be moved next to.
    void push_dense(SStage &st, SOp op)
    {
        if (cfg.fuse) {
            for (int i = (int)st.ops.size() - 1; i >= 0; i--) {
                SOp &x = st.ops[i];
                if (x.type == 1) {
                    uint64_t um = x.pmask | op.pmask;
                    int ku = popc(um);
                    if (ku <= cfg.F && dense_cost(ku) <= dense_cost(x.k) + dense_cost(op.k) &&
                        (x.pmask & op.pmask)) {
                        int upos[kMaxGateQubits];
                        int nu = 0;
                        for (int j = 0; j < x.k; j++) upos[nu++] = x.pos[j];
                        for (int j = 0; j < op.k; j++)
                            if (!((x.pmask >> op.pos[j]) & 1)) upos[nu++] = op.pos[j];
                        std::vector<cd> A = expand(x.M, x.k, x.pos, nu, upos);
                        std::vector<cd> B = expand(op.M, op.k, op.pos, nu, upos);
                        x.M = matmul(B, A, 1 << nu);
                        x.k = nu;
                        for (int j = 0; j < nu; j++) x.pos[j] = upos[j];
                        x.pmask = um;
                        x.n_src += op.n_src;
                        return;
                    }
                }
                if (meets(x, op.pmask)) break;
            }
        }
        st.ops.push_back(std::move(op));
    }

    void emit_diag_op(std::vector<Term> terms)
    {
        normalize_terms(terms);
        Op o;
        o.kind = OPK_DIAG;
        o.buf = buf;
        o.n = n;
        o.terms = std::move(terms);
        plan.ops.push_back(std::move(o));
    }

    // Store of a block (positions Q, register stages) that leaves logical
    // qubit q at position npos[q]; commits that frame.
    void emit_block(uint64_t Q, const std::vector<SStage> &stages, const int *npos)
    {
        for (int p = 0; p < 64; p++) lam[p] = (p < n && ((Q >> p) & 1)) ? npos[at[p]] : p;
        Op o;
        o.kind = OPK_CHUNK;
        o.buf = buf;
        o.n = n;
        finalize_chunk(o, Q, stages);
        last_chunk_op = (int)plan.ops.size();
        last_stages = stages;
        last_Q = Q;
        std::memcpy(last_lam, lam, sizeof(lam));
        std::memcpy(last_at, at, sizeof(at));
        plan.ops.push_back(std::move(o));
        // the pending phases follow their qubits: position p -> lam[p]
        for (PendingDiag &d : pending) {
            d.mask = remap(d.mask);
            for (Term &t : d.terms) t.mask = remap(t.mask);
        }
        for (int q = 0; q < n; q++) laminv[q] = npos[q];
        for (int q = 0; q < n; q++) at[npos[q]] = q;
        for (int p = 0; p < 64; p++) lam[p] = p;
    }

    // The frame after a block (qubit reordering of Section 2.3, applied by
    // the block's own store, so it costs no sweep).  The frame is always a
    // set of swaps between a low position l < L and the home position of the
    // qubit it holds, so at most 2L positions are ever displaced.  The
    // earliest-needed qubits of the dense gates still to come move into the
    // low positions, which every block holds anyway, leaving the block's
    // C - L other positions for further qubits.  Only qubits whose positions
    // are (or can be added to) this block's Q move.  SWAP relabellings inside
    // the block are undone by the same store.
    void choose_frame(size_t first, uint64_t &Q, int *npos)
    {
        const int L = cfg.L;
        // the block-start frame (the SWAP relabellings inside the block are
        // undone by its store)
        int fpos[64], fat[64];
        std::memcpy(fpos, blk_pos, sizeof(int) * n);
        for (int q = 0; q < n; q++) fat[fpos[q]] = q;
        for (int q = 0; q < n; q++) npos[q] = fpos[q];
        if (!cfg.remap || L == 0) return;
        // wanted: the qubits of this block needed soonest by the dense gates
        // still to come (their positions are in Q, so the store can move them;
        // the next block then holds them in its low positions for free)
        int want[8], nw = 0;
        for (size_t i = first; i < G.size() && nw < L; i++) {
            if (done[i] || G[i].diag || G[i].swap) continue;
            for (int j = 0; j < G[i].k && nw < L; j++) {
                const int q = G[i].q[j];
                if (!((Q >> fpos[q]) & 1)) continue;
                bool dup = false;
                for (int k = 0; k < nw; k++) dup |= want[k] == q;
                if (!dup) want[nw++] = q;
            }
        }
        auto wanted = [&](int q) {
            for (int k = 0; k < nw; k++) if (want[k] == q) return true;
            return false;
        };
        auto room = [&](uint64_t add) { return popc(Q | add) <= cfg.C; };
        int used[8] = {0};
        for (int l = 0; l < L; l++) {
            const int r = fat[l];                  // resident of low position l
            if (wanted(r)) continue;
            if (r != l && wanted(l)) {
                // the position's own qubit is wanted: send r home, bring l back
                const uint64_t need = (1ull << r);
                if (room(need)) {
                    Q |= need;
                    npos[r] = r;
                    npos[l] = l;
                }
                continue;
            }
            // a wanted qubit at its high home position w takes position l
            int pick = -1;
            for (int k = 0; k < nw && pick < 0; k++) {
                const int w = want[k];
                if (used[k] || w < L || fpos[w] != w) continue;
                uint64_t need = 1ull << w;
                if (r != l) need |= 1ull << r;
                if (room(need)) pick = k;
            }
            if (pick < 0) continue;
            const int w = want[pick];
            used[pick] = 1;
            Q |= 1ull << w;
            if (r != l) {
                Q |= 1ull << r;
                npos[r] = r;                       // the old resident goes home
            }
            npos[w] = l;
            npos[l] = w;                           // qubit l waits at w's home
        }
        // a valid permutation that moves only positions of Q; else no change
        int seen[64] = {0};
        bool ok = true;
        for (int q = 0; q < n && ok; q++) {
            const int p = npos[q];
            ok = p >= 0 && p < n && !seen[p];
            if (ok) seen[p] = 1;
            if (ok && p != fpos[q]) ok = ((Q >> p) & 1) && ((Q >> fpos[q]) & 1);
        }
        if (!ok)
            for (int q = 0; q < n; q++) npos[q] = fpos[q];
    }

    // After the last block: every qubit back to its own position, folded into
    // the last block's store when it holds all displaced positions, else one
    // permutation-only pass.  The pending phases follow.
    void restore_identity_frame()
    {
        uint64_t D = 0;
        for (int q = 0; q < n; q++) if (laminv[q] != q) D |= (1ull << laminv[q]) | (1ull << q);
        if (!D) return;
        int fat[64];
        for (int p = 0; p < n; p++) fat[p] = at[p];
        if (last_chunk_op >= 0 && last_chunk_op == (int)plan.ops.size() - 1 && (D & ~last_Q) == 0) {
            // re-store the last block straight into the identity frame
            std::memcpy(at, last_at, sizeof(at));
            for (int p = 0; p < 64; p++) lam[p] = (p < n && ((last_Q >> p) & 1)) ? at[p] : p;
            finalize_chunk(plan.ops[last_chunk_op], last_Q, last_stages);
            std::memcpy(last_lam, lam, sizeof(lam));
        } else {
            uint64_t Q = ((1ull << cfg.L) - 1) | D;
            for (int p = 0; p < n && popc(Q) < cfg.C; p++) Q |= 1ull << p;
            for (int p = 0; p < 64; p++) lam[p] = (p < n && ((Q >> p) & 1)) ? fat[p] : p;
            std::vector<SStage> one(1);
            Op o;
            o.kind = OPK_CHUNK;
            o.buf = buf;
            o.n = n;
            finalize_chunk(o, Q, one);
            last_chunk_op = (int)plan.ops.size();
            last_stages = one;
            last_Q = Q;
            std::memcpy(last_lam, lam, sizeof(lam));
            for (int p = 0; p < n; p++) last_at[p] = fat[p];
            plan.ops.push_back(std::move(o));
        }
        // pending phases: position p held logical fat[p], now at its home
        for (PendingDiag &d : pending) {
            uint64_t m = 0, x = d.mask;
            while (x) { int p = __builtin_ctzll(x); x &= x - 1; m |= 1ull << fat[p]; }
            d.mask = m;
            for (Term &t : d.terms) {
                uint64_t tm = 0, y = t.mask;
                while (y) { int p = __builtin_ctzll(y); y &= y - 1; tm |= 1ull << fat[p]; }
                t.mask = tm;
            }
        }
        for (int q = 0; q < n; q++) laminv[q] = at[q] = q;
        for (int p = 0; p < 64; p++) lam[p] = p;
    }

    void run()
    {
        const uint64_t lowL = (1ull << cfg.L) - 1;
        size_t first = 0;
        while (true) {
            while (first < G.size() && done[first]) first++;
            bool dense_left = false;
            for (size_t i = first; i < G.size(); i++)
                if (!done[i] && !G[i].diag) { dense_left = true; break; }
            if (!dense_left) {
                for (size_t i = first; i < G.size(); i++)
                    if (!done[i]) { make_pending(G[i]); done[i] = 1; }
                break;
            }
            std::memcpy(blk_pos, laminv, sizeof(blk_pos));
            std::vector<SStage> stages;
            uint64_t Q = lowL;
            for (int s = 0; s < cfg.Smax; s++) {
                SStage st;
                bool placed = false;
                // Layers: place every gate that needs no pending phase; when a
                // gate does need one, flush ALL pending phases at once (they
                // are all ready) and scan again.  One phase segment per layer.
                while (true) {
                    uint64_t blocked = 0;
                    bool need_flush = false;
                    for (size_t i = first; i < G.size(); i++) {
                        if (done[i]) continue;
                        const PGate &g = G[i];
                        if (g.qmask & blocked) { blocked |= g.qmask; continue; }
                        if (g.diag) { make_pending(g); done[i] = 1; continue; }
                        uint64_t P = phys(g.qmask);
                        if (g.swap) {
                            // a relabelling: pending phases live in the physical
                            // frame, so they commute with it
                            if (popc((Q | P) & ~lowL) <= cfg.C - cfg.L) {
                                Q |= P;
                                const int pa = laminv[g.q[0]], pb = laminv[g.q[1]];
                                std::swap(at[pa], at[pb]);
                                laminv[at[pa]] = pa;
                                laminv[at[pb]] = pb;
                                done[i] = 1;
                                placed = true;
                            } else {
                                blocked |= g.qmask;
                            }
                            continue;
                        }
                        if (g.k > kChunkMaxK || popc(st.R | P) > cfg.RB ||
                            popc((Q | P) & ~lowL) > cfg.C - cfg.L) {
                            blocked |= g.qmask;
                            continue;
                        }
                        if (pending_meets(P)) {
                            need_flush = true;
                            blocked |= g.qmask;
                            continue;
                        }
                        SOp d;
                        d.type = 1;
                        d.k = g.k;
                        for (int j = 0; j < g.k; j++) d.pos[j] = laminv[g.q[j]];
                        d.pmask = P;
                        d.M = g.M;
                        d.n_src = g.n_src;
                        push_dense(st, std::move(d));
                        st.R |= P;
                        Q |= P;
                        done[i] = 1;
                        placed = true;
                    }
                    if (!need_flush) break;
                    SOp ph;
                    flush(~0ull, ph);
                    st.ops.push_back(std::move(ph));
                }
                // a trailing flush with no gate after it goes back to pending
                if (!st.ops.empty() && st.ops.back().type == 2) {
                    for (const Term &t : st.ops.back().terms) {
                        PendingDiag d;
                        d.mask = t.mask;
                        d.n_src = 0;
                        d.terms.push_back(t);
                        pending.push_back(std::move(d));
                    }
                    st.ops.pop_back();
                }
                if (!placed) break;
                stages.push_back(std::move(st));
            }
            if (stages.empty()) {
                // the earliest unplaced gate is wider than the register stage
                size_t i = first;
                while (done[i]) i++;
                const PGate &g = G[i];
                SOp ph;
                if (flush(phys(g.qmask), ph)) emit_diag_op(ph.terms);
                Op o;
                o.kind = OPK_GATE;
                o.buf = buf;
                o.n = n;
                o.gate = g;
                for (int j = 0; j < g.k; j++) o.gate.q[j] = laminv[g.q[j]];
                plan.ops.push_back(std::move(o));
                done[i] = 1;
                continue;
            }
            // the frame after this block, then pad the chunk to exactly C
            // positions with the lowest free qubits
            int npos[64];
            choose_frame(first, Q, npos);
            for (int p = 0; p < n && popc(Q) < cfg.C; p++) Q |= 1ull << p;
            emit_block(Q, stages, npos);
        }
        restore_identity_frame();
        // the diagonals left at the end of the circuit
        if (!pending.empty()) {
            std::vector<Term> all;
            for (PendingDiag &d : pending) all.insert(all.end(), d.terms.begin(), d.terms.end());
            pending.clear();
            normalize_terms(all);
            if (all.empty()) return;
            if (all.size() == 1 && all[0].mask == 0 && last_chunk_op >= 0 &&
                last_chunk_op == (int)plan.ops.size() - 1) {
                // only a global phase is left: scale the last dense matrix by it
                for (int s = (int)last_stages.size() - 1; s >= 0; s--) {
                    for (int k = (int)last_stages[s].ops.size() - 1; k >= 0; k--) {
                        SOp &x = last_stages[s].ops[k];
                        if (x.type != 1) continue;
                        cd f = phase_of(all[0].w);
                        for (cd &z : x.M) z *= f;
                        std::memcpy(lam, last_lam, sizeof(lam));
                        finalize_chunk(plan.ops[last_chunk_op], last_Q, last_stages);
                        for (int i = 0; i < 64; i++) lam[i] = laminv[i] = i;
                        return;
                    }
                }
            }
            if (last_chunk_op >= 0 && last_chunk_op == (int)plan.ops.size() - 1) {
                // fold into the end of the last block, in its load frame
                int inv[64];
                for (int p = 0; p < 64; p++) inv[last_lam[p]] = p;
                SOp ph;
                ph.type = 2;
                for (Term &t : all) {
                    uint64_t m = 0, x = t.mask;
                    while (x) { int p = __builtin_ctzll(x); x &= x - 1; m |= 1ull << inv[p]; }
                    ph.terms.push_back({m, t.w});
                }
                normalize_terms(ph.terms);
                last_stages.back().ops.push_back(std::move(ph));
                std::memcpy(lam, last_lam, sizeof(lam));
                Op &o = plan.ops[last_chunk_op];
                finalize_chunk(o, last_Q, last_stages);
                for (int i = 0; i < 64; i++) lam[i] = laminv[i] = i;
            } else {
                emit_diag_op(std::move(all));
            }
        }
    }

    uint64_t remap(uint64_t m) const
    {
        uint64_t r = 0;
        while (m) { int p = __builtin_ctzll(m); m &= m - 1; r |= 1ull << lam[p]; }
        return r;
    }

    void finalize_chunk(Op &o, uint64_t Q, const std::vector<SStage> &stages)
    {
        ChunkProg &cp = o.prog;
        cp.C = cfg.C;
        cp.RB = cfg.RB;
        int nc = 0;
        for (int p = 0; p < n; p++) if ((Q >> p) & 1) { cp.qin[nc] = p; cp.qout[nc] = lam[p]; nc++; }
        cp.stages.clear();
        for (const SStage &s : stages) {
            Stage ps;
            for (const SOp &x : s.ops) {
                StageOp so;
                so.type = x.type;
                so.k = x.k;
                for (int j = 0; j < x.k; j++) so.reg[j] = x.pos[j];
                so.M = x.M;
                so.terms = x.terms;
                so.n_src = x.n_src;
                ps.ops.push_back(std::move(so));
            }
            cp.stages.push_back(std::move(ps));
        }
        o.words = encode_program(n, cfg.C, cfg.RB, cfg.f64, Q, stages, lam, false);
    }
};

// ------------------------------------------------------------ stats
static void account(Plan &p)
{
    sim_plan_stats &s = p.stats;
    int sz = p.dtype == SIM_C64 ? 8 : 16;
    for (size_t i = 0; i < p.ops.size(); i++) {
        const Op &o = p.ops[i];
        double amps = std::ldexp(1.0, o.n);
        // a sweep fed by a fused tensor product reads no state: write-only
        const bool fed = i > 0 && p.ops[i - 1].fused;
        if (fed) s.bytes -= (uint64_t)(amps * sz);
        if (o.fused) {   // no launch of its own
            s.tensor_ops++;
            s.tensor_fused++;
            s.state_updates += (uint64_t)amps;
            s.flops += amps * 6.0;
            continue;
        }
        s.ops++;
        switch (o.kind) {
        case OPK_INIT_BASIS:
            s.bytes += (uint64_t)(amps * sz);
            break;
        case OPK_GATE:
            s.gate_ops++;
            if (o.buf == 0) s.sweeps++;
            s.bytes += (uint64_t)(2 * amps * sz);
            s.state_updates += (uint64_t)amps;
            s.flops += amps * 8.0 * (1 << o.gate.k);
            break;
        case OPK_GATE_DIAG: {
            s.gate_ops++;
            int nz = 0;
            for (int c = 0; c < (1 << o.gate.k); c++) {
                uint64_t x = 0;
                for (int i = 0; i < o.gate.k; i++) if ((c >> i) & 1) x |= 1ull << o.gate.q[i];
                uint64_t w = 0;
                for (const Term &t : o.gate.terms) if ((x & t.mask) == t.mask) w += t.w;
                if (w != 0) nz++;
            }
            double frac = (double)nz / (1 << o.gate.k);
            s.bytes += (uint64_t)(2 * amps * sz * frac);
            s.state_updates += (uint64_t)(amps * frac);
            s.flops += amps * frac * 6.0;
            break;
        }
        case OPK_DIAG:
        case OPK_PHASE_SMALL:
            s.diag_ops++;
            if (o.buf == 0) s.sweeps++;
            s.bytes += (uint64_t)(2 * amps * sz);
            s.state_updates += (uint64_t)amps;
            s.flops += amps * 6.0;
            break;
        case OPK_CHUNK: {
            s.chunk_ops++;
            if (o.buf == 0) s.sweeps++;
            s.bytes += (uint64_t)(2 * amps * sz);
            s.state_updates += (uint64_t)amps;
            for (const Stage &st : o.prog.stages)
                for (const StageOp &x : st.ops) s.flops += x.type == 1 ? amps * 8.0 * (1 << x.k) : amps * 6.0;
            break;
        }
        case OPK_TENSOR:
            s.tensor_ops++;
            s.bytes += (uint64_t)(amps * sz);
            s.state_updates += (uint64_t)amps;
            s.flops += amps * 6.0;
            break;
        case OPK_DENSE_TC:
            s.dense_ops++;
            if (o.buf == 0) s.sweeps++;
            s.bytes += (uint64_t)(2 * amps * sz);
            s.state_updates += (uint64_t)amps;
            s.flops += amps * 8.0 * 32;
            break;
        case OPK_DENSE_CHUNK:
            s.dense_ops += o.blocks.size();
            if (o.buf == 0) s.sweeps++;
            s.bytes += (uint64_t)(2 * amps * sz);
            s.state_updates += (uint64_t)(amps * o.blocks.size());
            s.flops += amps * 8.0 * 32 * o.blocks.size();
            break;
        }
    }
}

// ------------------------------------------------------------ pipeline
static void emit_unfused(const std::vector<PGate> &G, int n, int buf, Plan &plan)
{
    for (const PGate &g : G) {
        Op o;
        o.buf = buf;
        o.n = n;
        if (g.diag && g.kind == kFusedDiag) {
            o.kind = OPK_DIAG;
            o.terms = g.terms;
        } else if (g.diag) {
            o.kind = OPK_GATE_DIAG;
            o.gate = g;
        } else {
            o.kind = OPK_GATE;
            o.gate = g;
        }
        plan.ops.push_back(std::move(o));
    }
}

// Encode the K3 diagonal sweep program (fixed layout: tile of 2^C
// consecutive amplitudes, register bits on top).
static std::vector<uint32_t> encode_diag_sweep(int n, const std::vector<Term> &terms, bool f64, int &C, int &RB)
{
    RB = 4;   // 16 amplitudes per thread: more resident warps than 32 (measured faster)
    C = 7 + RB;
    SStage st;
    SOp ph;
    ph.type = 2;
    ph.terms = terms;
    st.ops.push_back(ph);
    std::vector<SStage> stages{st};
    int lam[64];
    for (int i = 0; i < 64; i++) lam[i] = i;
    return encode_program(n, C, RB, f64, (1ull << C) - 1, stages, lam, true);
}

// Dense-block mode (tensor-core path): GBSA in fusion mode over the whole
// circuit -- greedy in dependency order, each block collects every gate that
// fits a set of at most 5 qubits, and its 32 x 32 unitary is composed in FP64
// (gates applied in order).  Blocks narrower than 5 qubits are widened with
// idle qubits so that every block is one 5-qubit dense sweep.
static void schedule_dense_blocks(const std::vector<PGate> &G, int n, int precision, int buf, Plan &plan)
{
    const int K = n < 5 ? n : 5;
    std::vector<char> done(G.size(), 0);
    size_t first = 0;
    while (true) {
        while (first < G.size() && done[first]) first++;
        if (first >= G.size()) break;
        uint64_t S = 0, blocked = 0;
        std::vector<size_t> members;
        for (size_t i = first; i < G.size(); i++) {
            if (done[i]) continue;
            const PGate &g = G[i];
            if (g.qmask & blocked) { blocked |= g.qmask; continue; }
            if (popc(S | g.qmask) <= K) {
                S |= g.qmask;
                members.push_back(i);
                done[i] = 1;
            } else {
                blocked |= g.qmask;
            }
        }
        if (members.empty()) {
            // a single gate wider than the block: apply it on its own
            const PGate &g = G[first];
            Op o;
            o.buf = buf;
            o.n = n;
            if (g.diag) { o.kind = OPK_DIAG; o.terms = g.terms; }
            else { o.kind = OPK_GATE; o.gate = g; }
            plan.ops.push_back(std::move(o));
            done[first] = 1;
            continue;
        }
        for (int p = 0; p < n && popc(S) < K; p++) S |= 1ull << p;
        int qs[kMaxGateQubits], kq = 0;
        for (int p = 0; p < n; p++) if ((S >> p) & 1) qs[kq++] = p;
        const int dim = 1 << kq;
        std::vector<cd> U((size_t)dim * dim, cd(0, 0));
        for (int i = 0; i < dim; i++) U[(size_t)i * dim + i] = 1;
        int nsrc = 0;
        for (size_t mi : members) {
            const PGate &g = G[mi];
            nsrc += g.n_src;
            if (g.diag) {
                // scale row r by the phase of the basis state it stands for
                for (int r = 0; r < dim; r++) {
                    uint64_t x = 0;
                    for (int b = 0; b < kq; b++) if ((r >> b) & 1) x |= 1ull << qs[b];
                    uint64_t w = 0;
                    for (const Term &t : g.terms) if ((x & t.mask) == t.mask) w += t.w;
                    cd f = phase_of(w);
                    for (int c = 0; c < dim; c++) U[(size_t)r * dim + c] *= f;
                }
            } else {
                std::vector<cd> E = expand(g.M, g.k, g.q, kq, qs);
                U = matmul(E, U, dim);
            }
        }
        Op o;
        o.kind = kq == 5 ? OPK_DENSE_TC : OPK_GATE;
        o.buf = buf;
        o.n = n;
        o.gate.kind = kFusedDense;
        o.gate.k = kq;
        for (int b = 0; b < kq; b++) o.gate.q[b] = qs[b];
        o.gate.qmask = S;
        o.gate.M = std::move(U);
        o.gate.n_src = nsrc;
        o.precision = precision;
        plan.ops.push_back(std::move(o));
    }
}

// TF32 operand rounding (the conversion the kernels use for their A operand,
// cvt.rna: to nearest, ties away from zero, 10 stored mantissa bits): half a
// unit of the 13 dropped bits added to the magnitude, then cleared.
static uint32_t tf32_bits(float x)
{
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return u;
    return (u + 0x1000u) & 0xffffe000u;
}

static float float_of_bits(uint32_t u)
{
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// Device program of a cache-blocked dense-block sweep (dense_prog.h): chunk
// qubits, per block its target bits, row order and swizzled offsets, and its
// 64 x 64 real embedding split into TF32 hi + lo, stacked as one 128-row MMA
// operand (K-major core matrices of 8 rows x 4 elements, rows fastest).
std::vector<uint32_t> encode_dense_chunk(int n, const int *cq, const std::vector<PGate> &blocks)
{
    using namespace dprog;
    const int nb = (int)blocks.size();
    std::vector<uint32_t> w((size_t)H_SIZE + (size_t)nb * kBlkWords, 0);
    const size_t boff = (w.size() + 31) & ~(size_t)31;
    w.resize(boff + (size_t)nb * kBImgWords, 0);
    w[H_MAGIC] = kMagic;
    w[H_N] = (uint32_t)n;
    w[H_NBLK] = (uint32_t)nb;
    w[H_BOFF] = (uint32_t)boff;
    w[H_WORDS] = (uint32_t)w.size();
    uint64_t cm = 0;
    int cbit[64];
    for (int i = 0; i < 64; i++) cbit[i] = -1;
    for (int i = 0; i < kC; i++) {
        w[H_QIN + i] = (uint32_t)cq[i];
        cm |= 1ull << cq[i];
        cbit[cq[i]] = i;
    }
    const uint64_t fm = (n >= 64 ? ~0ull : (1ull << n) - 1) & ~cm;
    w[H_FREE_LO] = (uint32_t)fm;
    w[H_FREE_HI] = (uint32_t)(fm >> 32);
    for (int b = 0; b < nb; b++) {
        const PGate &g = blocks[(size_t)b];
        uint32_t *r = &w[(size_t)H_SIZE + (size_t)b * kBlkWords];
        int T[5];
        uint32_t tmask = 0;
        for (int i = 0; i < 5; i++) {
            T[i] = cbit[g.q[i]];
            tmask |= 1u << T[i];
        }
        r[B_TMASK] = tmask;
        // row bits: lanes 0..3 of a warp take chunk bits of distinct residues
        // mod 4 where the block leaves them (conflict-free half-warp accesses
        // under the swizzle), then the remaining bits in ascending order
        int rows[7], nr = 0;
        uint32_t taken = 0, resid = 0;
        for (int i = 0; i < kC && nr < 4; i++)
            if (!((tmask >> i) & 1) && !((resid >> (i & 3)) & 1)) {
                rows[nr++] = i;
                taken |= 1u << i;
                resid |= 1u << (i & 3);
            }
        for (int i = 0; i < kC; i++)
            if (!((tmask >> i) & 1) && !((taken >> i) & 1)) rows[nr++] = i;
        for (int i = 0; i < 7; i++) r[B_ROWSLOT + i] = slot(1u << rows[i]);
        for (int j = 0; j < 32; j++) {
            uint32_t x = 0;
            for (int i = 0; i < 5; i++)
                if ((j >> i) & 1) x |= 1u << T[i];
            r[B_TOFF + j] = slot(x);
        }
        // B[nn][kk]: output real nn (re 0..31, im 32..63) from input real kk
        uint32_t *bi = &w[boff + (size_t)b * kBImgWords];
        for (int nn = 0; nn < 64; nn++)
            for (int kk = 0; kk < 64; kk++) {
                const cd u = g.M[(size_t)(nn & 31) * 32 + (kk & 31)];
                const double v = nn < 32 ? (kk < 32 ? u.real() : -u.imag()) : (kk < 32 ? u.imag() : u.real());
                const uint32_t hi = tf32_bits((float)v);
                const uint32_t lo = tf32_bits((float)(v - (double)float_of_bits(hi)));
                // one operand of 128 rows: hi in rows 0..63, lo in rows 64..127
                auto word = [](int row, int k) {
                    return (size_t)(((k >> 2) * 16 + (row >> 3)) * 32 + (row & 7) * 4 + (k & 3));
                };
                bi[word(nn, kk)] = hi;
                bi[word(64 + nn, kk)] = lo;
            }
    }
    return w;
}

// Cache blocking of dense blocks (K6 inside K4): the 5-qubit blocks of a run
// share one sweep while their qubits, with qubits 0..3, fit a 2^12-amplitude
// chunk.  Greedy in dependency order like the block search itself: a block
// joins the open sweep unless it shares a qubit with a block left out before
// it (blocks on disjoint qubits commute).
static void group_dense_chunks(Plan &plan, size_t first, int n)
{
    using dprog::kC;
    std::vector<Op> in;
    for (size_t i = first; i < plan.ops.size(); i++) in.push_back(std::move(plan.ops[i]));
    plan.ops.resize(first);
    size_t i = 0;
    while (i < in.size()) {
        if (in[i].kind != OPK_DENSE_TC) {
            plan.ops.push_back(std::move(in[i]));
            i++;
            continue;
        }
        size_t j = i;
        while (j < in.size() && in[j].kind == OPK_DENSE_TC) j++;
        std::vector<char> done(j - i, 0);
        size_t left = j - i, head = 0;
        while (left) {
            while (done[head]) head++;
            Op o;
            o.kind = OPK_DENSE_CHUNK;
            o.buf = in[i].buf;
            o.n = n;
            o.precision = SIM_DENSE_SPLIT_TF32;
            uint64_t S = 0xF, blocked = 0;
            for (size_t k = head; k < j - i && (int)o.blocks.size() < dprog::kMaxBlocks; k++) {
                if (done[k]) continue;
                const uint64_t m = in[i + k].gate.qmask;
                if (m & blocked) {
                    blocked |= m;
                } else if (popc(S | m) <= kC) {
                    S |= m;
                    o.blocks.push_back(std::move(in[i + k].gate));
                    done[k] = 1;
                    left--;
                } else {
                    blocked |= m;
                }
            }
            for (int p = 0; p < n && popc(S) < kC; p++) S |= 1ull << p;
            int c = 0;
            for (int p = 0; p < n; p++)
                if ((S >> p) & 1) o.cq[c++] = p;
            o.words = encode_dense_chunk(n, o.cq, o.blocks);
            plan.ops.push_back(std::move(o));
        }
        i = j;
    }
}

static void schedule(const std::vector<PGate> &G, int n, const sim_options &opt, sim_dtype dt, int buf, Plan &plan)
{
    if ((opt.flags & SIM_F_TC) && n >= 5) {
        // complex64: split-TF32 or FP32 (FP64 and double-float asks run FP32);
        // complex128: true FP64, or double-float for every other ask
        int prec = opt.dense_precision;
        if (dt == SIM_C64) prec = prec == SIM_DENSE_SPLIT_TF32 ? SIM_DENSE_SPLIT_TF32 : SIM_DENSE_FP32;
        else prec = prec == SIM_DENSE_FP64 ? SIM_DENSE_FP64 : SIM_DENSE_DOUBLE_FLOAT;
        const size_t first = plan.ops.size();
        schedule_dense_blocks(G, n, prec, buf, plan);
        // split-TF32 blocks of a state of >= 2^12 amplitudes: cache-blocked,
        // several blocks per sweep (without SIM_F_BLOCK: one sweep per block)
        if (prec == SIM_DENSE_SPLIT_TF32 && dt == SIM_C64 && (opt.flags & SIM_F_BLOCK) && n >= dprog::kC)
            group_dense_chunks(plan, first, n);
        return;
    }
    int C = 0, RB = 0;
    // kernels specialised per program hold 32 amplitudes per thread (fewer
    // register stages per sweep); the interpreter is faster at 16
    const int want_rb = opt.register_bits ? opt.register_bits : ((opt.flags & SIM_F_JIT) && dt == SIM_C64 ? 5 : 0);
    bool blocked = (opt.flags & SIM_F_BLOCK) && chunk_shape(n, dt, opt.chunk_qubits, want_rb, C, RB);
    if (!blocked) {
        emit_unfused(G, n, buf, plan);
        return;
    }
    Cfg cfg;
    cfg.C = C;
    cfg.RB = RB;
    cfg.L = std::min(dt == SIM_C64 ? 4 : 3, C - RB);
    cfg.F = opt.max_fuse_qubits;
    cfg.Smax = opt.max_stages;
    cfg.fuse = (opt.flags & SIM_F_FUSE) != 0;
    cfg.remap = (opt.flags & SIM_F_REMAP) != 0;
    cfg.f64 = dt == SIM_C128;
    Scheduler s(G, n, cfg, plan, buf);
    s.run();
}

// Merge booster (Algorithm 7 with the Divider of Algorithm 6).  The state is
// the product basis state |basis>; qubits are split into contiguous groups
// (low qubits first).  Each group simulates the dependency-closed prefix of
// gates that stay inside it on its own 2^w sub-state; groups then merge
// pairwise by tensor products (the higher range is the left factor) and the
// merged groups take their next prefixes, until one group spans all n
// qubits.  Returns the gates left for the full state.  Readings: 0-based
// qubit ranges; an odd group is carried up unmerged; divSize = (n+B-1)/B
// when B > 0, else the chunk width (every leaf fits one cached chunk).
static void run_booster(std::vector<PGate> &pend, int n, const sim_options &opt, sim_dtype dt, uint64_t basis,
                        Plan &plan)
{
    int def_div = dt == SIM_C64 ? 12 : 11;
    int divSize = opt.booster_div > 0 ? (n + opt.booster_div - 1) / opt.booster_div : def_div;
    if (divSize < 1) divSize = 1;
    std::vector<int> que;
    divider(n, divSize, que);
    if (que.size() < 2) return;
    plan.booster_queue = que;
    struct Grp {
        int lo, w, buf;
    };
    std::vector<Grp> groups;
    int lo = 0;
    for (int w : que) {
        plan.buf_qubits.push_back(w);
        Grp g{lo, w, (int)plan.buf_qubits.size() - 1};
        Op o;
        o.kind = OPK_INIT_BASIS;
        o.buf = g.buf;
        o.n = w;
        o.basis = (basis >> lo) & ((1ull << w) - 1);
        plan.ops.push_back(std::move(o));
        groups.push_back(g);
        lo += w;
    }
    while (groups.size() > 1) {
        // generation step: every group's entanglement-free prefix
        for (const Grp &g : groups) {
            std::vector<PGate> sub = take_group(pend, g.lo, g.w);
            if (sub.empty()) continue;
            for (PGate &x : sub) {
                plan.stats.boosted_gates += x.n_src;
                x = shift_gate(x, g.lo);
            }
            if (opt.flags & SIM_F_DIAG) {
                uint64_t absorbed = 0;
                sub = diagonal_detector(sub, opt.max_diag_qubits, absorbed);
                plan.stats.diag_fused += absorbed;
            }
            schedule(sub, g.w, opt, dt, g.buf, plan);
        }
        // merge step: pairwise tensor products, the last merge writes the state
        std::vector<Grp> next;
        const bool final_merge = groups.size() == 2;
        for (size_t i = 0; i + 1 < groups.size(); i += 2) {
            const Grp &a = groups[i], &b = groups[i + 1];
            int w = a.w + b.w;
            int nb = 0;
            if (!final_merge) {
                plan.buf_qubits.push_back(w);
                nb = (int)plan.buf_qubits.size() - 1;
            }
            Op o;
            o.kind = OPK_TENSOR;
            o.buf = nb;
            o.n = w;
            o.buf_lo = a.buf;
            o.n_lo = a.w;
            o.buf_hi = b.buf;
            o.n_hi = b.w;
            plan.ops.push_back(std::move(o));
            next.push_back({a.lo, w, nb});
        }
        if (groups.size() & 1) next.push_back(groups.back());
        groups.swap(next);
    }
}

static void finalize_words(Plan &plan)
{
    bool f64 = plan.dtype == SIM_C128;
    for (Op &o : plan.ops) {
        if (o.kind == OPK_DIAG) {
            int C, RB;
            if (o.n >= 11) {
                o.words = encode_diag_sweep(o.n, o.terms, f64, C, RB);
            } else {
                // too small for the diagonal sweep's tile: run it as a one-stage chunk pass
                int Cc = 0, RBc = 0;
                if (!chunk_shape(o.n, plan.dtype, 0, 0, Cc, RBc)) {
                    // below every chunk shape: one thread per amplitude sums the terms
                    o.kind = OPK_PHASE_SMALL;
                    continue;
                }
                o.kind = OPK_CHUNK;
                SStage st;
                SOp ph;
                ph.type = 2;
                ph.terms = o.terms;
                st.ops.push_back(ph);
                std::vector<SStage> stages{st};
                int lam[64];
                for (int i = 0; i < 64; i++) lam[i] = i;
                uint64_t Q = (1ull << Cc) - 1;
                o.prog.C = Cc;
                o.prog.RB = RBc;
                for (int i = 0; i < Cc; i++) o.prog.qin[i] = o.prog.qout[i] = i;
                Stage ps;
                StageOp so;
                so.type = 2;
                so.terms = o.terms;
                ps.ops.push_back(so);
                o.prog.stages.push_back(ps);
                o.words = encode_program(o.n, Cc, RBc, f64, Q, stages, lam, false);
            }
        }
    }
}

// Walk an encoded program the way the kernels do and check every offset,
// count and bit position before it can reach the GPU.
static bool validate_program(const std::vector<uint32_t> &w, int n, bool diag_sweep, std::string &err)
{
    auto bad = [&](const char *m) { err = std::string("internal: invalid device program: ") + m; return false; };
    const size_t W = w.size();
    if (W < (size_t)prog::H_SIZE || w[prog::H_MAGIC] != prog::kMagic) return bad("header");
    if (w[prog::H_WORDS] != W || (W & 1)) return bad("program length");
    const int C = (int)w[prog::H_C], RB = (int)w[prog::H_RB], ns = (int)w[prog::H_NSTAGE];
    if (C < 1 || C > prog::kMaxC || C > n || RB < 1 || RB > prog::kMaxRB || RB >= C) return bad("shape");
    if (ns < 0 || ns > prog::kMaxStages || (diag_sweep && ns != 1)) return bad("stage count");
    if ((int)w[prog::H_N] != n) return bad("n");
    const int wb = (int)w[prog::H_WBYTES];
    if (wb != 4 && wb != 8) return bad("weight size");
    uint64_t freem = (uint64_t)w[prog::H_FREE_LO] | ((uint64_t)w[prog::H_FREE_HI] << 32);
    uint64_t qm = 0;
    for (int i = 0; i < C; i++) {
        uint32_t q = w[prog::H_QIN + i];
        if ((int)q >= n || ((qm >> q) & 1)) return bad("qin");
        qm |= 1ull << q;
    }
    uint64_t nmask = n >= 64 ? ~0ull : ((1ull << n) - 1);
    if ((qm & freem) || ((qm | freem) != nmask)) return bad("free mask");
    if (!diag_sweep && (qm & 1) == 0) return bad("qubit 0 must be a chunk bit");
    uint32_t sp = 0;
    for (int i = 0; i < C; i++) {
        uint32_t b = w[prog::H_SPERM + i];
        if ((int)b >= C || ((sp >> b) & 1)) return bad("store permutation");
        sp |= 1u << b;
    }
    // launch-wide term tables
    const uint32_t ND = w[prog::H_NDSEG], NH = w[prog::H_NHOIST], S = 1 + RB, TB = C - RB,
                   SC = prog::cta_slots(RB, TB), SCP = prog::cta_stride(RB, TB, (uint32_t)wb);
    if (ND > (uint32_t)prog::kMaxDseg || NH > ND) return bad("segment counts");
    if (prog::smem_bytes(w.data(), diag_sweep) > 200 * 1024) return bad("shared memory");
    {
        size_t co = w[prog::H_CTA_OFF], cn = w[prog::H_NCTA], to = w[prog::H_THR_OFF], tn = w[prog::H_NTHR];
        if (co + cn * prog::kCtaWords > W || to + tn * prog::kThrWords > W) return bad("term tables");
        for (size_t i = 0; i < cn; i++)
            if (w[co + i * prog::kCtaWords] >= ND * SCP || w[co + i * prog::kCtaWords] % SCP >= SC)
                return bad("CTA table slot");
        for (size_t i = 0; i < tn; i++) {
            if (w[to + i * prog::kThrWords] >= NH * S) return bad("thread table slot");
            if (w[to + i * prog::kThrWords + 1] >> TB) return bad("thread table mask");
        }
    }
    const uint32_t direct = w[prog::H_DIRECT];
    if (direct & ~3u) return bad("direct flags");
    auto direct_ok = [&](size_t so) {
        const bool paired = w[so + prog::S_REG] == 0;
        bool ok = wb == 4 && C - RB >= 5;
        for (int i = 0; i < (paired ? 3 : 4) && ok; i++)
            ok = w[so + prog::S_THR + i] == (uint32_t)(i + (paired ? 1 : 0));
        for (int i = 0; i < 4 && ok; i++) ok = w[prog::H_QIN + i] == (uint32_t)i;
        return ok;
    };
    if ((direct & prog::DIRECT_FIRST) && (ns < 1 || !direct_ok(w[prog::H_STAGE_OFF]))) return bad("direct first stage");
    if (direct & prog::DIRECT_LAST) {
        bool ok = ns >= 1 && direct_ok(w[prog::H_STAGE_OFF + ns - 1]);
        for (int i = 0; i < C && ok; i++) ok = w[prog::H_SPERM + i] == (uint32_t)i;
        if (!ok) return bad("direct last stage");
    }
    uint32_t nseg_seen = 0;
    for (int s = 0; s < ns; s++) {
        size_t so = w[prog::H_STAGE_OFF + s];
        if ((so & 3) || so + prog::S_SIZE > W) return bad("stage offset");
        uint32_t seen = 0;
        for (int j = 0; j < RB; j++) {
            uint32_t b = w[so + prog::S_REG + j];
            if ((int)b >= C || ((seen >> b) & 1)) return bad("register bits");
            seen |= 1u << b;
        }
        for (int i = 0; i < C - RB; i++) {
            uint32_t b = w[so + prog::S_THR + i];
            if ((int)b >= C || ((seen >> b) & 1)) return bad("thread bits");
            if (w[so + prog::S_GTHR + i] != w[prog::H_QIN + b]) return bad("thread bit positions");
            if (i < RB && w[so + prog::S_PV + i] !=
                              prog::swizzle(1u << w[so + prog::S_REG + i], C, prog::swizzle_bits(w[prog::H_WBYTES])))
                return bad("register offsets");
            seen |= 1u << b;
        }
        const uint32_t nops = w[so + prog::S_NOPS];
        size_t op = so + prog::S_SIZE;
        for (uint32_t k = 0; k < nops; k++) {
            // bodies are 16-byte aligned: ops start at 2 (mod 4) words
            if (op + 2 > W || (op & 3) != 2) return bad("op offset");
            const uint32_t hdr = w[op], len = w[op + prog::O_WORDS];
            if (len < 4 || (len & 3) || op + len > W) return bad("op length");
            const int type = hdr & 0xff;
            if (type == prog::OP_DENSE) {
                if (diag_sweep) return bad("dense op in a diagonal sweep");
                const int kq = (hdr >> 8) & 0xf, code = (int)(hdr >> 16), sub = (hdr >> 12) & 0xf;
                if (kq < 1 || kq > kChunkMaxKEncoded) return bad("dense arity");
                if (sub > prog::DS_RX || (sub != prog::DS_GENERAL && kq != 1)) return bad("dense subtype");
                int prev = -1;
                for (int i = 0; i < kq; i++) {
                    int p = (code >> (3 * i)) & 7;
                    if (p >= RB || p <= prev) return bad("dense positions");
                    prev = p;
                }
                if (code >> (3 * kq)) return bad("dense code");
                size_t need = 2 + (size_t)2 * (1u << (2 * kq)) * (wb == 8 ? 2 : 1);
                if (len < need) return bad("dense body");
            } else if (type == prog::OP_DSEG) {
                if (len < (size_t)prog::O_BODY + prog::D_TERMS) return bad("phase header");
                const uint32_t *b = &w[op + prog::O_BODY];
                if ((int32_t)b[prog::D_PIVOT] < -1 || (int32_t)b[prog::D_PIVOT] >= RB) return bad("phase pivot");
                if (b[prog::D_FLAGS] > 1) return bad("phase flags");
                if (b[prog::D_INDEX] != nseg_seen++) return bad("phase segment number");
                size_t nterm = b[prog::D_NBASE];
                for (int j = 0; j < prog::kMaxRB; j++) {
                    if (j >= RB && b[prog::D_NLIN + j]) return bad("phase lin count");
                    nterm += b[prog::D_NLIN + j];
                }
                size_t need = prog::O_BODY + prog::D_TERMS + nterm * prog::kTermWords + 2 * ((size_t)1 << RB) +
                              prog::ctab_words(RB, wb) + (size_t)b[prog::D_NMULTI] * prog::kMultiWords;
                if (len < need) return bad("phase body");
            } else {
                return bad("op type");
            }
            op += len;
        }
        if (op > so + w[so + prog::S_WORDS] || so + w[so + prog::S_WORDS] > W) return bad("stage length");
    }
    return true;
}

bool make_batch_ops(int n, sim_dtype dt, const sim_gate *gates, size_t ng, std::vector<uint32_t> &words, int &nops,
                    std::string &err, bool &too_wide)
{
    too_wide = false;
    std::vector<PGate> G;
    G.reserve(ng);
    for (size_t i = 0; i < ng; i++) {
        PGate g;
        if (!make_gate(gates[i], n, g, err)) {
            err = "gate " + std::to_string(i) + ": " + err;
            return false;
        }
        if (!g.diag && g.k > 3) {
            too_wide = true;
            err = "dense gate wider than 3 qubits";
            return false;
        }
        G.push_back(std::move(g));
    }
    uint64_t absorbed = 0;
    G = diagonal_detector(G, 0, absorbed);
    const bool f64 = dt == SIM_C128;
    nops = 0;
    for (const PGate &g : G) {
        const size_t start = words.size();
        if (g.diag) {
            if (g.terms.size() > 16000) { err = "phase polynomial too long for the batch path"; too_wide = true; return false; }
            words.push_back(2);   // BOP_PHASE; length patched below
            words.push_back((uint32_t)g.terms.size());
            for (const Term &t : g.terms) {
                words.push_back((uint32_t)t.mask);
                words.push_back((uint32_t)(t.mask >> 32));
                words.push_back((uint32_t)t.w);
                words.push_back((uint32_t)(t.w >> 32));
            }
            words[start] |= (uint32_t)(words.size() - start) << 16;
        } else {
            words.push_back(1u | (uint32_t)g.k << 8);   // BOP_DENSE
            for (int i = 0; i < 3; i++) words.push_back(i < g.k ? (uint32_t)g.q[i] : 0u);
            for (const cd &z : g.M) {
                if (f64) {
                    double re = z.real(), im = z.imag();
                    uint64_t a, b;
                    std::memcpy(&a, &re, 8);
                    std::memcpy(&b, &im, 8);
                    words.push_back((uint32_t)a);
                    words.push_back((uint32_t)(a >> 32));
                    words.push_back((uint32_t)b);
                    words.push_back((uint32_t)(b >> 32));
                } else {
                    float re = (float)z.real(), im = (float)z.imag();
                    uint32_t a, b;
                    std::memcpy(&a, &re, 4);
                    std::memcpy(&b, &im, 4);
                    words.push_back(a);
                    words.push_back(b);
                }
            }
            words[start] |= (uint32_t)(words.size() - start) << 16;
        }
        nops++;
    }
    return true;
}

// ------------------------------------------------------------ Euler split
// A one-qubit unitary U = e^{i phi} V, V = [[p, -conj(q)], [q, conj(p)]] in
// SU(2), is exactly D1 R D2 with R = [[|p|, -|q|], [|q|, |p|]] real,
// D2 = diag(1, e^{-i(a+b)}) and D1 = e^{i phi} diag(e^{ia}, e^{ib}), a =
// arg p, b = arg q.  Where U's neighbours on its qubit are diagonal gates (or
// the circuit's ends), D1 and D2 join those diagonals' phase polynomial and
// the sweep applies only the real R, which costs a third of a complex 2x2.
// D2 commutes back to the previous gate on the qubit (diagonal, or none) and
// is emitted right after it, so that it joins the phases flushed before the
// whole layer of R's rather than forcing one flush per R.  Real and RX-form
// matrices (already cheap) are left alone.
static std::vector<PGate> euler_split(const std::vector<PGate> &G, int n, uint64_t &split)
{
    split = 0;
    // neighbours on the qubit: previous / next gate touching it
    std::vector<int> prev(G.size(), -1), next(G.size(), -1), last(n, -1);
    for (size_t i = 0; i < G.size(); i++)
        for (int j = 0; j < G[i].k; j++) {
            const int q = G[i].q[j];
            if (last[q] >= 0 && G[i].k == 1) prev[i] = last[q];
            if (last[q] >= 0 && G[last[q]].k == 1) next[last[q]] = (int)i;
            last[q] = (int)i;
        }
    std::vector<PGate> front;                  // D2s of gates first on their qubit
    std::vector<std::vector<PGate>> after(G.size());   // D2s emitted after gate i
    std::vector<std::vector<PGate>> at(G.size());      // gate i's replacement (R, D1), if split
    std::vector<char> done(G.size(), 0);
    for (size_t i = 0; i < G.size(); i++) {
        const PGate &g = G[i];
        bool cand = g.k == 1 && !g.diag && !g.swap && g.M.size() == 4 && (prev[i] < 0 || G[prev[i]].diag) &&
                    (next[i] < 0 || G[next[i]].diag);
        if (cand) {
            bool real = true, rx = true;
            for (int e = 0; e < 4; e++) {
                real = real && g.M[e].imag() == 0;
                rx = rx && ((e == 0 || e == 3) ? g.M[e].imag() == 0 : g.M[e].real() == 0);
            }
            cand = !real && !rx;
        }
        cd p, q, det;
        if (cand) {
            det = g.M[0] * g.M[3] - g.M[1] * g.M[2];
            cand = std::abs(std::abs(det) - 1.0) < 1e-12;
        }
        double phi = 0;
        if (cand) {
            phi = 0.5 * std::arg(det);
            const cd e = std::polar(1.0, -phi);
            p = g.M[0] * e;
            q = g.M[2] * e;
            // V must be [[p, -conj q], [q, conj p]] (det V = 1, up to the
            // branch of the square root: then p, q change sign together)
            const cd v01 = g.M[1] * e, v11 = g.M[3] * e;
            cand = std::abs(v01 + std::conj(q)) < 1e-12 && std::abs(v11 - std::conj(p)) < 1e-12;
        }
        if (!cand) continue;
        const double a = std::abs(p) > 0 ? std::arg(p) : 0.0, b = std::abs(q) > 0 ? std::arg(q) : 0.0;
        const int qb = g.q[0];
        auto diag_gate = [&](double th0, double th1) {
            PGate d;
            d.kind = kFusedDiag;
            d.diag = true;
            d.k = 1;
            d.q[0] = qb;
            d.qmask = 1ull << qb;
            d.n_src = 0;
            d.terms = {Term{0, turns_of(th0)}, Term{1ull << qb, turns_of(th1 - th0)}};
            normalize_terms(d.terms);
            return d;
        };
        (prev[i] >= 0 ? after[prev[i]] : front).push_back(diag_gate(0.0, -(a + b)));   // D2
        PGate r;
        r.kind = kFusedDense;
        r.k = 1;
        r.q[0] = qb;
        r.qmask = 1ull << qb;
        r.n_src = g.n_src;
        r.M = {cd(std::abs(p), 0), cd(-std::abs(q), 0), cd(std::abs(q), 0), cd(std::abs(p), 0)};
        at[i].push_back(std::move(r));
        at[i].push_back(diag_gate(phi + a, phi + b));   // D1
        done[i] = 1;
        split++;
    }
    std::vector<PGate> out(front);
    out.reserve(G.size() + 2 * split);
    for (size_t i = 0; i < G.size(); i++) {
        if (done[i]) out.insert(out.end(), at[i].begin(), at[i].end());
        else out.push_back(G[i]);
        out.insert(out.end(), after[i].begin(), after[i].end());
    }
    return out;
}

// ------------------------------------------------------------ chunk shape
// Complex64 plans for the specialised kernels, with no shape asked for,
// choose between chunks of 2^12 amplitudes and of 2^13 (one more qubit per
// sweep, so often fewer sweeps) by planning both.  The choice is kept per
// circuit structure (gate kinds and qubits, options; not the angles), so
// repeated applies of a structure plan once.
// The checks the dense-block sweep kernel relies on: header, chunk qubits
// (qubits 0..3 first, ascending, below n), five distinct target bits per
// block, row bits and offsets that cover the chunk exactly once, B images
// inside the program and 16-byte aligned.
static bool validate_dense_chunk(const std::vector<uint32_t> &w, int n, std::string &err)
{
    using namespace dprog;
    auto bad = [&](const char *m) { err = std::string("internal: invalid dense-block program: ") + m; return false; };
    if (w.size() < (size_t)H_SIZE || w[H_MAGIC] != kMagic || w[H_WORDS] != w.size()) return bad("header");
    if ((int)w[H_N] != n || n < kC || n > 40) return bad("n");
    const size_t nb = w[H_NBLK], boff = w[H_BOFF];
    if (nb < 1 || nb > (size_t)kMaxBlocks) return bad("block count");
    if (boff % 32 != 0 || boff < (size_t)H_SIZE + nb * kBlkWords || boff + nb * kBImgWords != w.size())
        return bad("B images");
    uint64_t cm = 0;
    for (int i = 0; i < kC; i++) {
        const uint32_t q = w[H_QIN + i];
        if ((int)q >= n || (i < 4 && q != (uint32_t)i) || (i > 0 && q <= w[H_QIN + i - 1])) return bad("chunk qubits");
        cm |= 1ull << q;
    }
    const uint64_t fm = (uint64_t)w[H_FREE_LO] | ((uint64_t)w[H_FREE_HI] << 32);
    if (fm != (((1ull << n) - 1) & ~cm)) return bad("free mask");
    std::vector<char> seen(1u << kC);
    for (size_t b = 0; b < nb; b++) {
        const uint32_t *r = &w[H_SIZE + b * kBlkWords];
        if (popc(r[B_TMASK]) != 5 || (r[B_TMASK] >> kC) != 0) return bad("targets");
        std::fill(seen.begin(), seen.end(), 0);
        for (uint32_t t = 0; t < (uint32_t)kCols; t++) {
            uint32_t rb = 0;
            for (int i = 0; i < 7; i++)
                if ((t >> i) & 1) rb ^= r[B_ROWSLOT + i];
            for (int j = 0; j < 32; j++) {
                const uint32_t sl = rb ^ r[B_TOFF + j];
                if (sl >= (1u << kC) || seen[sl]) return bad("chunk cover");
                seen[sl] = 1;
            }
        }
    }
    return true;
}

static bool auto_chunk_shape(int n, sim_dtype dt, const sim_options &o)
{
    return dt == SIM_C64 && n >= 16 && (o.flags & SIM_F_JIT) && (o.flags & SIM_F_BLOCK) && !(o.flags & SIM_F_TC) &&
           o.chunk_qubits == 0 && (o.register_bits == 0 || o.register_bits == 5);
}

static uint64_t shape_key(int n, sim_dtype dt, const sim_options &o, bool product_state, const sim_gate *gates,
                          size_t ng)
{
    uint64_t h = 1469598103934665603ull;   // FNV-1a, 64 bit
    auto mix = [&](uint64_t v) {
        for (int i = 0; i < 8; i++) {
            h ^= (v >> (8 * i)) & 255;
            h *= 1099511628211ull;
        }
    };
    mix((uint64_t)n);
    mix((uint64_t)dt);
    mix(o.flags);
    mix((uint64_t)(uint32_t)o.max_fuse_qubits | (uint64_t)(uint32_t)o.max_diag_qubits << 32);
    mix((uint64_t)(uint32_t)o.max_stages | (uint64_t)(uint32_t)o.booster_div << 32);
    mix(product_state ? 1 : 0);
    mix(ng);
    for (size_t i = 0; i < ng; i++) {
        const sim_gate &g = gates[i];
        mix((uint64_t)g.kind | (uint64_t)g.nq << 32);
        for (uint32_t j = 0; j < g.nq && j < 6; j++) mix(g.q[j]);
    }
    return h;
}

static std::mutex g_shape_mu;
static std::unordered_map<uint64_t, int> g_shapes;

static int cached_shape(uint64_t key)
{
    std::lock_guard<std::mutex> lk(g_shape_mu);
    auto it = g_shapes.find(key);
    return it == g_shapes.end() ? 0 : it->second;
}

static void remember_shape(uint64_t key, int cq)
{
    std::lock_guard<std::mutex> lk(g_shape_mu);
    if (g_shapes.size() >= 4096) g_shapes.clear();
    g_shapes[key] = cq;
}

// passes over the whole state in a plan
static size_t full_sweeps(const Plan &p)
{
    size_t k = 0;
    for (const Op &o : p.ops)
        if (o.buf == 0 && (o.kind == OPK_GATE || o.kind == OPK_GATE_DIAG || o.kind == OPK_DIAG || o.kind == OPK_CHUNK ||
                           o.kind == OPK_DENSE_TC || o.kind == OPK_DENSE_CHUNK))
            k++;
    return k;
}

bool make_plan(int n, sim_dtype dt, uint64_t basis, const sim_gate *gates, size_t ng, const sim_options &opt_in,
               Plan &plan, std::string &err)
{
    auto t0 = std::chrono::steady_clock::now();
    sim_options opt = opt_in;
    resolve_options(opt, n, dt);
    plan = Plan();
    plan.n = n;
    plan.dtype = dt;
    plan.buf_qubits.push_back(n);
    std::vector<PGate> G;
    G.reserve(ng);
    for (size_t i = 0; i < ng; i++) {
        PGate g;
        if (!make_gate(gates[i], n, g, err)) {
            err = "gate " + std::to_string(i) + ": " + err;
            return false;
        }
        G.push_back(std::move(g));
    }
    plan.stats.gates_in = ng;
    // Algorithm 4, machine level: booster, diagonal detector, blocking + fusion
    if ((opt.flags & SIM_F_BOOST) && basis != UINT64_MAX && ng > 0) run_booster(G, n, opt, dt, basis, plan);
    if ((opt.flags & SIM_F_DIAG) && (opt.flags & SIM_F_BLOCK) && !(opt.flags & SIM_F_TC)) {
        uint64_t nsplit = 0;
        G = euler_split(G, n, nsplit);
    }
    // cache-blocked dense blocks: the blocks absorb diagonal gates anyway, and
    // the detector's fused diagonals can split runs of blocks; plan with and
    // without it and keep the cheaper (a sweep costs about as much as 2.5
    // blocks of tensor-core work on this GPU)
    const bool dense_blocked = (opt.flags & SIM_F_TC) && (opt.flags & SIM_F_BLOCK) && dt == SIM_C64 &&
                               opt.dense_precision == SIM_DENSE_SPLIT_TF32 && n >= dprog::kC;
    if ((opt.flags & SIM_F_DIAG) && dense_blocked) {
        uint64_t absorbed = 0;
        std::vector<PGate> Gd = diagonal_detector(G, opt.max_diag_qubits, absorbed);
        Plan pd = plan, pn = plan;
        schedule(Gd, n, opt, dt, 0, pd);
        schedule(G, n, opt, dt, 0, pn);
        auto cost = [](const Plan &p) {
            size_t sw = 0, bl = 0;
            for (const Op &o : p.ops) {
                if (o.buf != 0) continue;
                if (o.kind == OPK_DENSE_CHUNK) { sw++; bl += o.blocks.size(); }
                else if (o.kind != OPK_INIT_BASIS && o.kind != OPK_TENSOR) { sw++; bl++; }
            }
            return 5.0 * (double)sw + 2.0 * (double)bl;
        };
        if (cost(pd) <= cost(pn)) {
            plan = std::move(pd);
            plan.stats.diag_fused += absorbed;
        } else {
            plan = std::move(pn);
        }
    } else {
    if (opt.flags & SIM_F_DIAG) {
        uint64_t absorbed = 0;
        G = diagonal_detector(G, opt.max_diag_qubits, absorbed);
        plan.stats.diag_fused += absorbed;
    }
    if (auto_chunk_shape(n, dt, opt)) {
        // the full state's chunk shape: 2^12 or 2^13 amplitudes, whichever
        // the cost model says is cheaper for this circuit's structure
        const uint64_t key = shape_key(n, dt, opt, basis != UINT64_MAX, gates, ng);
        int cq = cached_shape(key);
        if (cq) {
            sim_options o = opt;
            o.chunk_qubits = cq;
            schedule(G, n, o, dt, 0, plan);
        } else {
            Plan p12 = plan, p13 = plan;
            sim_options o12 = opt, o13 = opt;
            o12.chunk_qubits = 12;
            o13.chunk_qubits = 13;
            schedule(G, n, o12, dt, 0, p12);
            schedule(G, n, o13, dt, 0, p13);
            // a sweep of 2^13-amplitude chunks (one CTA of 256 threads per
            // SM) takes about 1.1 times as long as one of 2^12 (two CTAs of
            // 128): measured 1.06-1.14 on the benchmarked workloads
            cq = full_sweeps(p13) * 11 < full_sweeps(p12) * 10 ? 13 : 12;
            remember_shape(key, cq);
            plan = cq == 13 ? std::move(p13) : std::move(p12);
        }
    } else {
        schedule(G, n, opt, dt, 0, plan);
    }
    }
    finalize_words(plan);
    // a tensor product that only feeds the next sweep of the same buffer is
    // computed by that sweep's loads: one write-only pass instead of a write
    // and a read-write pass
    for (size_t i = 0; i + 1 < plan.ops.size(); i++) {
        Op &t = plan.ops[i];
        const Op &x = plan.ops[i + 1];
        if (t.kind == OPK_TENSOR && x.buf == t.buf && x.n == t.n && (x.kind == OPK_DIAG || x.kind == OPK_CHUNK))
            t.fused = true;
    }
    for (const Op &o : plan.ops) {
        if (o.kind == OPK_CHUNK || o.kind == OPK_DIAG)
            if (!validate_program(o.words, o.n, o.kind == OPK_DIAG, err)) return false;
        if ((o.kind == OPK_GATE || o.kind == OPK_DENSE_TC) &&
            (o.gate.k < 1 || o.gate.k > kMaxGateQubits || o.gate.M.size() != ((size_t)1 << (2 * o.gate.k)))) {
            err = "internal: bad dense gate op";
            return false;
        }
        if (o.kind == OPK_DENSE_CHUNK && !validate_dense_chunk(o.words, o.n, err)) return false;
    }
    account(plan);
    plan.stats.plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return true;
}

// ------------------------------------------------------------ JSON
static void jnum(std::ostringstream &os, double v)
{
    char b[40];
    snprintf(b, sizeof b, "%.17g", v);
    os << b;
}

static void jterms(std::ostringstream &os, const std::vector<Term> &t)
{
    os << "[";
    for (size_t i = 0; i < t.size(); i++) os << (i ? "," : "") << "[\"" << t[i].mask << "\",\"" << t[i].w << "\"]";
    os << "]";
}

static void jmat(std::ostringstream &os, const std::vector<cd> &M)
{
    os << "[";
    for (size_t i = 0; i < M.size(); i++) {
        os << (i ? "," : "") << "[";
        jnum(os, M[i].real());
        os << ",";
        jnum(os, M[i].imag());
        os << "]";
    }
    os << "]";
}

std::string plan_json(const Plan &p)
{
    std::ostringstream os;
    const sim_plan_stats &s = p.stats;
    os << "{\"n\":" << p.n << ",\"dtype\":" << (int)p.dtype << ",\"wbits\":" << (p.dtype == SIM_C64 ? 32 : 64);
    os << ",\"stats\":{\"gates_in\":" << s.gates_in << ",\"ops\":" << s.ops << ",\"sweeps\":" << s.sweeps
       << ",\"chunk_ops\":" << s.chunk_ops << ",\"diag_ops\":" << s.diag_ops << ",\"gate_ops\":" << s.gate_ops
       << ",\"tensor_ops\":" << s.tensor_ops << ",\"tensor_fused\":" << s.tensor_fused << ",\"dense_ops\":" << s.dense_ops << ",\"diag_fused\":" << s.diag_fused
       << ",\"boosted_gates\":" << s.boosted_gates << ",\"state_updates\":" << s.state_updates
       << ",\"bytes\":" << s.bytes << "}";
    os << ",\"buffers\":[";
    for (size_t i = 0; i < p.buf_qubits.size(); i++) os << (i ? "," : "") << p.buf_qubits[i];
    os << "],\"booster_queue\":[";
    for (size_t i = 0; i < p.booster_queue.size(); i++) os << (i ? "," : "") << p.booster_queue[i];
    os << "],\"ops\":[";
    for (size_t oi = 0; oi < p.ops.size(); oi++) {
        const Op &o = p.ops[oi];
        os << (oi ? "," : "") << "{\"buf\":" << o.buf << ",\"n\":" << o.n << ",";
        switch (o.kind) {
        case OPK_INIT_BASIS: os << "\"op\":\"init\",\"basis\":\"" << o.basis << "\""; break;
        case OPK_GATE:
            os << "\"op\":\"gate\",\"qubits\":[";
            for (int i = 0; i < o.gate.k; i++) os << (i ? "," : "") << o.gate.q[i];
            os << "],\"matrix\":";
            jmat(os, o.gate.M);
            break;
        case OPK_GATE_DIAG:
            os << "\"op\":\"phase\",\"terms\":";
            jterms(os, o.gate.terms);
            break;
        case OPK_DIAG:
        case OPK_PHASE_SMALL:
            os << "\"op\":\"phase\",\"terms\":";
            jterms(os, o.terms);
            break;
        case OPK_CHUNK: {
            const ChunkProg &cp = o.prog;
            os << "\"op\":\"chunk\",\"C\":" << cp.C << ",\"qin\":[";
            for (int i = 0; i < cp.C; i++) os << (i ? "," : "") << cp.qin[i];
            os << "],\"qout\":[";
            for (int i = 0; i < cp.C; i++) os << (i ? "," : "") << cp.qout[i];
            os << "],\"words\":" << o.words.size() << ",\"direct\":" << o.words[prog::H_DIRECT] << ",\"layouts\":[";
            // each stage's register and thread bits (chunk bit numbers)
            for (uint32_t si = 0; si < o.words[prog::H_NSTAGE]; si++) {
                const size_t so = o.words[prog::H_STAGE_OFF + si];
                const int RBw = (int)o.words[prog::H_RB], TBw = (int)o.words[prog::H_C] - RBw;
                os << (si ? "," : "") << "{\"reg\":[";
                for (int j = 0; j < RBw; j++) os << (j ? "," : "") << o.words[so + prog::S_REG + j];
                os << "],\"thr\":[";
                for (int i = 0; i < TBw; i++) os << (i ? "," : "") << o.words[so + prog::S_THR + i];
                os << "]}";
            }
            os << "],\"stages\":[";
            for (size_t si = 0; si < cp.stages.size(); si++) {
                os << (si ? "," : "") << "[";
                const Stage &st = cp.stages[si];
                for (size_t k = 0; k < st.ops.size(); k++) {
                    const StageOp &x = st.ops[k];
                    os << (k ? "," : "");
                    if (x.type == 1) {
                        os << "{\"dense\":[";
                        for (int i = 0; i < x.k; i++) os << (i ? "," : "") << x.reg[i];
                        os << "],\"matrix\":";
                        jmat(os, x.M);
                        os << "}";
                    } else {
                        os << "{\"phase\":";
                        jterms(os, x.terms);
                        os << "}";
                    }
                }
                os << "]";
            }
            os << "]";
            break;
        }
        case OPK_TENSOR:
            os << "\"op\":\"tensor\",\"lo\":" << o.buf_lo << ",\"hi\":" << o.buf_hi << ",\"n_lo\":" << o.n_lo
               << ",\"n_hi\":" << o.n_hi << ",\"fused\":" << (o.fused ? "true" : "false");
            break;
        case OPK_DENSE_TC:
            os << "\"op\":\"gate\",\"qubits\":[";
            for (int i = 0; i < o.gate.k; i++) os << (i ? "," : "") << o.gate.q[i];
            os << "],\"matrix\":";
            jmat(os, o.gate.M);
            break;
        case OPK_DENSE_CHUNK:
            os << "\"op\":\"dense_chunk\",\"qin\":[";
            for (int i = 0; i < dprog::kC; i++) os << (i ? "," : "") << o.cq[i];
            os << "],\"words\":" << o.words.size() << ",\"blocks\":[";
            for (size_t b = 0; b < o.blocks.size(); b++) {
                const PGate &g = o.blocks[b];
                os << (b ? "," : "") << "{\"qubits\":[";
                for (int i = 0; i < g.k; i++) os << (i ? "," : "") << g.q[i];
                os << "],\"matrix\":";
                jmat(os, g.M);
                os << "}";
            }
            os << "]";
            break;
        }
        os << "}";
    }
    os << "]}";
    return os.str();
}

}  // namespace svs
