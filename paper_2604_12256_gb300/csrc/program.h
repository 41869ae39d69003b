// program.h -- word layout of the device programs run by the cache-blocked
// chunk kernel (K4) and the fused-diagonal sweep (K3).  The host encoder
// (planner.cpp) writes it; the kernels (k_chunk.cu) read it with uniform
// loads.  All offsets are in 32-bit words; every op and stage starts on an
// even word so doubles are 8-byte aligned.
//
// A program describes one pass over the state: the state is cut into chunks
// of 2^C amplitudes (Algorithm 2's chunks).  Chunk bit i is physical qubit
// qin[i]; the remaining n-C qubits select the chunk.  Inside a chunk the
// amplitudes go through `n_stages` register stages: in a stage, thread bit i
// of the thread index is chunk bit thr[i] and register bit j of a thread's
// register index is chunk bit reg[j].  Ops of a stage act on register bits
// only (dense) or on any index bit (phase segment).  On the store, output
// bit i' (physical qubit qin[i']) takes chunk bit sperm[i'], which realises
// the SWAP relabelling of Section 2.3 for free.
#pragma once

#include <cstdint>

namespace svs {
namespace prog {

constexpr uint32_t kMagic = 0x53565031u;   // "SVP1"
constexpr int kMaxC = 16;
constexpr int kMaxRB = 8;
constexpr int kMaxStages = 32;

// header
enum : int {
    H_MAGIC = 0,
    H_C = 1,
    H_RB = 2,
    H_NSTAGE = 3,
    H_N = 4,
    H_WBYTES = 5,        // 4: phase weights are uint32 turns; 8: uint64 turns
    H_FREE_LO = 6,       // mask of physical qubits NOT in the chunk
    H_FREE_HI = 7,
    H_QIN = 8,           // kMaxC words
    H_SPERM = H_QIN + kMaxC,
    H_STAGE_OFF = H_SPERM + kMaxC,   // kMaxStages words
    H_SIZE = H_STAGE_OFF + kMaxStages
};

// stage
enum : int {
    S_NOPS = 0,
    S_WORDS = 1,
    S_REG = 2,                 // kMaxRB words
    S_THR = S_REG + kMaxRB,    // kMaxC words
    S_GTHR = S_THR + kMaxC,    // kMaxC words: physical qubit of thread bit i (= qin[thr[i]])
    S_SIZE = S_GTHR + kMaxC    // even
};

// op header
enum : int { OP_DENSE = 1, OP_DSEG = 2 };
enum : int { O_HDR = 0, O_WORDS = 1, O_BODY = 2 };
// dense: hdr = OP_DENSE | k << 8 | code << 16 with code = p0 + 8 p1 + 64 p2
//        (register positions, ascending); body = 2 * 4^k reals (float or double)
// phase segment (DSEG) body:
enum : int {
    D_NBASE = 0,          // terms on thread/chunk bits only
    D_NMULTI = 1,         // terms with >= 2 register bits and other bits
    D_NLIN = 2,           // kMaxRB counts: terms with register bit j and other bits
    D_TERMS = D_NLIN + kMaxRB   // even
};
// term (4 words): mask_lo, mask_hi, w_lo, w_hi   (mask over physical qubits,
//                 register bits removed; w: uint32 in w_lo or uint64)
// then reg table: 2^RB entries x 2 words (phase of the register-only terms)
// multi term (6 words): mask_lo, mask_hi, regmask, 0, w_lo, w_hi
constexpr int kTermWords = 4;
constexpr int kMultiWords = 6;

}  // namespace prog
}  // namespace svs
