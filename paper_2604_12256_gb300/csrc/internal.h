// internal.h -- host-side types shared by the optimizer, the executor and
// the C ABI of libsvsim.  Nothing here is visible outside the library.
#pragma once

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "svsim.h"

namespace svs {

using cd = std::complex<double>;

constexpr int kMaxQubitsC64 = 34;
constexpr int kMaxQubitsC128 = 33;
constexpr int kMaxGateQubits = 6;

// One monomial of a diagonal phase polynomial: every diagonal unitary on
// qubits S is exp(2 pi i phi(x)) with phi(x) = sum_t w_t * prod_{j in mask_t} x_j
// (mod 1), x_j = bit j of the amplitude index.  Weights are fixed-point turns:
// w / 2^64 of a full turn, so sums of terms are exact modulo one turn.
struct Term {
    uint64_t mask;
    uint64_t w;
};

// Gate as seen by the optimizer (one input gate or a fusion of several).
struct PGate {
    int kind = -1;                 // sim_gate_kind of the input gate, or kFused*
    int k = 0;                     // number of qubits
    int q[kMaxGateQubits] = {0};   // local matrix bit i <-> qubit q[i]
    uint64_t qmask = 0;            // OR of 1 << q[i]
    bool diag = false;             // diagonal unitary: `terms` is authoritative
    bool swap = false;             // SWAP: a relabelling of two qubits
    std::vector<cd> M;             // 2^k x 2^k row-major (dense gates)
    std::vector<Term> terms;       // phase polynomial (diagonal gates)
    int n_src = 1;                 // input gates folded into this one
};

enum { kFusedDiag = 100, kFusedDense = 101 };

// Convert radians to fixed-point turns (mod 1 turn).
uint64_t turns_of(double radians);
// exp(2 pi i w / 2^64)
cd phase_of(uint64_t w);

// Build an optimizer gate from an ABI gate; returns false with a message.
bool make_gate(const sim_gate &g, int n, PGate &out, std::string &err);

// Dense matrix of a diagonal gate over its own qubits (local basis).
std::vector<cd> diag_matrix(const PGate &g);

// Merge terms with equal masks, drop zero weights, sort by mask.
void normalize_terms(std::vector<Term> &t);

// ---------------------------------------------------------------- the plan
enum OpKind {
    OPK_INIT_BASIS = 0,  // buffer <- |basis>
    OPK_GATE = 1,        // one dense gate, whole-vector sweep (Algorithm 1)
    OPK_GATE_DIAG = 2,   // one diagonal gate, touches only amplitudes it changes
    OPK_DIAG = 3,        // fused diagonal phase sweep (Algorithm 5, diagonal branch)
    OPK_CHUNK = 4,       // cache-blocked chunk sweep (Algorithm 5, all-in-one branch)
    OPK_TENSOR = 5,      // tensor product of two sub-states (Algorithm 5, first branch)
    OPK_DENSE_TC = 6,    // dense 5-qubit block as a tensor-core GEMM
    OPK_PHASE_SMALL = 7, // fused diagonal on a register too small for the sweep kernels
    OPK_DENSE_CHUNK = 8, // dense 5-qubit blocks inside a cache-blocked sweep (tensor cores)
};

// A chunk program: one cached chunk of C qubits passes through a sequence of
// register stages; in each stage RB chunk bits live in registers.
struct StageOp {
    int type = 0;                  // 1 dense on register bits, 2 phase segment
    int k = 0;
    int reg[kMaxGateQubits] = {0}; // register-bit positions, ascending
    std::vector<cd> M;             // matrix in that ascending local order
    std::vector<Term> terms;       // phase terms, masks in the load frame
    int n_src = 0;
    // for the JSON plan: the same operation on logical qubits
    int lq[kMaxGateQubits] = {0};
    std::vector<cd> M_logical;
    std::vector<Term> terms_logical;
};

struct Stage {
    int reg[8] = {0};              // chunk bit held by register bit j
    std::vector<StageOp> ops;
};

struct ChunkProg {
    int C = 0, RB = 0;
    int qin[16] = {0};             // physical qubit of chunk bit i when loading
    int qout[16] = {0};            // physical qubit of chunk bit i when storing
    std::vector<Stage> stages;
};

struct Op {
    OpKind kind;
    int buf = 0;                   // 0 = the state; >0 = booster sub-state
    int n = 0;                     // qubits of that buffer
    uint64_t basis = 0;            // INIT_BASIS
    PGate gate;                    // GATE / GATE_DIAG
    std::vector<Term> terms;       // DIAG
    ChunkProg prog;                // CHUNK
    int buf_lo = 0, buf_hi = 0, n_lo = 0, n_hi = 0;   // TENSOR: buf <- hi (x) lo
    bool fused = false;            // TENSOR: computed by the next op's loads, not launched
    std::vector<uint32_t> words;   // CHUNK / DIAG / DENSE_CHUNK: encoded device program
    int precision = 0;             // DENSE_TC: SIM_DENSE_* arithmetic
    std::vector<PGate> blocks;     // DENSE_CHUNK: the 5-qubit blocks, in order
    int cq[16] = {0};              // DENSE_CHUNK: chunk qubits, ascending
};

// Profile slot (sim_profile index) of an op kind: a dense-block sweep counts
// as a dense block, whether it holds one block or several.
inline int profile_kind(int kind) { return kind == OPK_DENSE_CHUNK ? OPK_DENSE_TC : kind; }

struct Plan {
    int n = 0;
    sim_dtype dtype = SIM_C64;
    std::vector<Op> ops;
    std::vector<int> buf_qubits;   // qubit count of each buffer id (0 = state)
    std::vector<int> booster_queue;   // Divider output (Algorithm 6), empty if unused
    sim_plan_stats stats{};
};

// Optimizer entry point (Algorithm 4).  basis = UINT64_MAX: unknown state.
bool make_plan(int n, sim_dtype dt, uint64_t basis, const sim_gate *gates, size_t ng,
               const sim_options &opt, Plan &plan, std::string &err);
std::string plan_json(const Plan &p);
// Device program of a cache-blocked dense-block sweep (dense_prog.h): chunk
// qubits cq[0..11] ascending with qubits 0..3 first, 5-qubit blocks in order.
std::vector<uint32_t> encode_dense_chunk(int n, const int *cq, const std::vector<PGate> &blocks);

// Serving: ops of the one-CTA batch kernel (batch.h) for a small circuit --
// the diagonal detector's fused phases and dense gates of <= 3 qubits.
// Returns false (err set) for invalid gates or wider dense gates.
bool make_batch_ops(int n, sim_dtype dt, const sim_gate *gates, size_t ng, std::vector<uint32_t> &words, int &nops,
                    std::string &err, bool &too_wide);

}  // namespace svs

// Point an existing handle at another state buffer / size (serving workers
// reuse one handle and one buffer); the state becomes |0...0> (lazily).
int svs_rebind(sim_t *s, int n, sim_dtype dt, void *dev_buf, size_t bytes);

namespace svs {
// host-side fault injection (fault.cpp): true when the next allocation /
// launch is to fail; dev_malloc is cudaMalloc behind that check
bool fault_alloc_fails();
bool fault_launch_fails();
cudaError_t dev_malloc(void **p, size_t bytes);
void fill_default_options(sim_options &o);
void resolve_options(sim_options &o, int n, sim_dtype dt);

}  // namespace svs
