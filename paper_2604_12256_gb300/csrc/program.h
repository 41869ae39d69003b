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

#if defined(__CUDACC_RTC__)
// run-time compilation of specialised sweep kernels: no host headers
typedef int int32_t;
typedef unsigned int uint32_t;
typedef unsigned long long uint64_t;
typedef long long int64_t;
typedef decltype(sizeof(0)) size_t;
#else
#include <cstddef>
#include <cstdint>
#endif

#if defined(__CUDACC__)
#define PROG_HD __host__ __device__
#else
#define PROG_HD
#endif

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
    // Phase segments are numbered 0..ND-1.  Their terms on chunk-selecting
    // (free) qubits only are summed once per chunk (CTA table); terms on
    // thread bits only are summed once per launch per thread (thread table,
    // for segments < NHOIST); the rest stay in the segment body.
    H_NDSEG = H_STAGE_OFF + kMaxStages,
    H_NHOIST,
    H_CTA_OFF,           // CTA table: word offset, count (kCtaWords each)
    H_NCTA,
    H_THR_OFF,           // thread table: word offset, count (kThrWords each)
    H_NTHR,
    H_WORDS,             // total words of the program (it is staged in shared memory)
    H_DIRECT,            // bit 0: stage 0's layout is a direct layout, bit 1: the last
                         // stage's is and the store permutation is the identity
    H_SIZE
};
// CTA-table entry: slot (= d * cta_stride + s: s = 0 base, 1 + j linear in
// register bit j, 1 + RB + i linear in thread bit i), 0, mask_lo, mask_hi,
// w_lo, w_hi
constexpr int kCtaWords = 6;
// thread-table entry: slot, mask over the thread-index bits, w_lo, w_hi
constexpr int kThrWords = 4;
constexpr int kMaxDseg = 64;

// stage.  Stages start on 4-word (16-byte) boundaries; S_SIZE = 2 (mod 4)
// and every op is padded to a multiple of 4 words, so each op starts 2 words
// before a 16-byte boundary and its body (O_BODY = 2) is 16-byte aligned: the
// kernels read stage headers, op bodies and tables with 128-bit loads.
enum : int {
    S_NOPS = 0,
    S_WORDS = 1,
    S_PV = 4,                  // kMaxRB words: swizzled shared-memory offset of register bit j
    S_REG = S_PV + kMaxRB,     // kMaxRB words
    S_THR = S_REG + kMaxRB,    // kMaxC words
    S_GTHR = S_THR + kMaxC,    // kMaxC words: physical qubit of thread bit i (= qin[thr[i]])
    S_SIZE = S_GTHR + kMaxC + 2
};
static_assert(S_PV % 4 == 0 && S_SIZE % 4 == 2, "stage header alignment");

// Direct layout of a stage: paired, register bit 0 is chunk bit 0 (qubit 0,
// so a thread's amplitudes m and m + 1 are adjacent in HBM: one 16-byte
// complex64 access) and thread bits 0..2 are chunk bits 1..3 (qubits 1..3:
// eight lanes cover 128 contiguous bytes); or unpaired, thread bits 0..3 are
// chunk bits 0..3 (16 lanes, 128 bytes).  A stage with such a layout can take its
// amplitudes straight from HBM (the first stage) or write them straight back
// (the last), without a pass through shared memory; kernels specialised to
// the program do so, the interpreter ignores the flags.
enum : uint32_t { DIRECT_FIRST = 1, DIRECT_LAST = 2 };

// Shared-memory swizzle of the chunk (interleaved complex amplitudes):
// element y lives at y ^ fold(y >> sw), folding sw-bit groups into the low
// bits.  Linear over GF(2), so offsets of disjoint bit sets combine by XOR.
// sw = log2 of the amplitudes in one 128-byte bank row: a warp's 8-byte
// (complex64) accesses are served by half-warps and 16-byte (complex128)
// ones by quarter-warps, so lanes whose chunk bits have distinct residues
// mod sw never share a bank.
PROG_HD inline constexpr int swizzle_bits(uint32_t wbytes) { return wbytes == 8 ? 3 : 4; }
inline uint32_t swizzle(uint32_t y, int C, int sw)
{
    uint32_t r = y;
    for (int s = sw; s < C; s += sw) r ^= (y >> s) & ((1u << sw) - 1);
    return r;
}

// op header
enum : int { OP_DENSE = 1, OP_DSEG = 2 };
enum : int { O_HDR = 0, O_WORDS = 1, O_BODY = 2 };
// dense: hdr = OP_DENSE | k << 8 | code << 16 with code = p0 + 8 p1 + 64 p2
//        (register positions, ascending); body = 2 * 4^k reals (float or double)
// phase segment (DSEG) body (16-byte aligned, read as 128-bit words):
enum : int {
    D_INDEX = 0,          // segment number d
    D_FLAGS = 1,          // bit 0: the register-only table is not all zero
    D_NBASE = 2,          // terms on thread/chunk bits only
    D_NMULTI = 3,         // terms with >= 2 register bits and other bits
    D_NLIN = 4,           // kMaxRB counts: terms with register bit j and other bits
    D_PIVOT = D_NLIN + kMaxRB,   // register bit present in every term, or -1:
                                 // then only amplitudes with that bit set change
    D_TABMASK = D_PIVOT + 1,     // bit m (RB <= 5): some register-only term has all
                                 // its register bits in m, so entry m of the
                                 // register-only table has terms (whatever their
                                 // weights sum to); 0xffffffff for RB > 5
    D_TERMS = D_PIVOT + 4        // 16-byte aligned (words D_PIVOT + 2, + 3 are 0)
};
static_assert(D_NLIN % 4 == 0 && D_TERMS % 4 == 0, "segment header alignment");
// dense op subtypes (hdr bits 12..15), for k = 1
enum : int { DS_GENERAL = 0, DS_REAL = 1, DS_RX = 2 };
// term (4 words): mask_lo, mask_hi, w_lo, w_hi   (mask over physical qubits,
//                 register bits removed; w: uint32 in w_lo or uint64)
// then reg table: 2^RB entries x 2 words (phase of the register-only terms),
// then the same table as complex factors cis(2 pi w / 2^wbits): 2^RB entries
// x (re, im) as float (2 words) or double-float (4 words), 16-byte aligned,
// multi term (6 words): mask_lo, mask_hi, regmask, 0, w_lo, w_hi
constexpr int kTermWords = 4;
constexpr int kMultiWords = 6;
// words of the complex register table (wb = bytes per real: 4 or 8)
PROG_HD inline constexpr uint32_t ctab_words(uint32_t RB, uint32_t wb) { return (1u << RB) * (wb == 8 ? 4 : 2); }

// Shared phase sums of one segment.  CTA table (per chunk): slot 0 = the
// segment's phase at register index 0, slot 1 + j = the coefficient of
// register bit j, slot 1 + RB + i = the coefficient of thread bit i (terms on
// chunk-selecting qubits and one thread bit).  Thread table (per launch): the
// first 1 + RB of those slots for terms on thread bits only.
PROG_HD inline constexpr uint32_t cta_slots(uint32_t RB, uint32_t TB) { return 1 + RB + TB; }
// a segment's CTA slots padded to 16 bytes (read with 128-bit loads)
PROG_HD inline constexpr uint32_t cta_stride(uint32_t RB, uint32_t TB, uint32_t wb)
{
    return wb == 8 ? (cta_slots(RB, TB) + 1) & ~1u : (cta_slots(RB, TB) + 3) & ~3u;
}
// The CTA table is triple-buffered: while chunk i reads buffer i mod 3, the
// sums of chunk i + 1 are accumulated into buffer (i + 1) mod 3 and buffer
// (i + 2) mod 3 is cleared, all between barriers the chunk needs anyway.
constexpr int kCtaBuffers = 3;
PROG_HD inline constexpr size_t cta_buffer_bytes(uint32_t nd, uint32_t RB, uint32_t TB, uint32_t wb)
{
    return ((size_t)nd * cta_stride(RB, TB, wb) * wb + 15) & ~(size_t)15;
}

// Dynamic shared memory of a launch of this program: the chunk's amplitudes
// (chunk kernel only), the program, the CTA-table buffers, the per-thread
// sums and the per-thread stage layouts (chunk kernel only).
inline size_t smem_bytes(const uint32_t *w, bool diag_sweep)
{
    const size_t C = w[H_C], RB = w[H_RB], wb = w[H_WBYTES];
    const size_t T = (size_t)1 << (C - RB), S = 1 + RB;
    const size_t planes = diag_sweep ? 0 : 2 * ((size_t)1 << C) * wb;
    const size_t progw = ((size_t)w[H_WORDS] * 4 + 15) & ~(size_t)15;
    // per-thread stage layouts (chunk kernel): thread part of x0 and of the
    // swizzled register-block offset for every stage
    const size_t layouts = diag_sweep ? 0 : (size_t)w[H_NSTAGE] * T * 12;
    return planes + progw + kCtaBuffers * cta_buffer_bytes(w[H_NDSEG], (uint32_t)RB, (uint32_t)(C - RB), (uint32_t)wb) +
           (((size_t)w[H_NHOIST] * S * T * wb + 15) & ~(size_t)15) + layouts;
}

}  // namespace prog
}  // namespace svs
