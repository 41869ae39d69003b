// dense_prog.h -- word layout of the program of a cache-blocked dense-block
// sweep (K6 inside K4): one pass over a complex64 state in chunks of 2^12
// amplitudes, each chunk taking a sequence of fused 5-qubit blocks on the
// tensor cores while it stays in shared memory (the all-in-one branch of
// Algorithm 5 applied to the dense blocks of Algorithm 4's fusion mode).
// The host encoder (planner.cpp) writes it, k_dense_chunk.cu reads it.
//
// Chunk bit i is physical qubit qin[i] (ascending; bits 0..3 are qubits 0..3,
// so a chunk is made of 128-byte segments).  A block acts on five chunk bits
// T; the other seven index its 128 columns.  Column t of a block is the MMA
// row t (and TMEM lane t): its chunk index is the XOR of rowslot[i] over the
// set bits i of t, and target index j adds toff[j] -- both already passed
// through the shared-memory swizzle slot() below, which is linear over GF(2).
#pragma once

#include <cstdint>

#if defined(__CUDACC__)
#define DPROG_HD __host__ __device__
#else
#define DPROG_HD
#endif

namespace svs {
namespace dprog {

constexpr uint32_t kMagic = 0x53564431u;   // "SVD1"
constexpr int kC = 12;                     // chunk qubits
constexpr int kCols = 1 << (kC - 5);       // columns of a block in one chunk (MMA M)
constexpr int kMaxBlocks = 48;             // blocks per sweep (their records sit in shared memory)

enum : int {
    H_MAGIC = 0,
    H_N = 1,
    H_NBLK = 2,
    H_BOFF = 3,          // word offset of the first B image (a multiple of 32)
    H_WORDS = 4,         // total words
    H_FREE_LO = 5,       // mask of the physical qubits not in the chunk
    H_FREE_HI = 6,
    H_QIN = 8,           // kC words
    H_SIZE = 32
};

// block record (kBlkWords words at H_SIZE + b * kBlkWords)
enum : int {
    B_TMASK = 0,         // the five target chunk bits
    B_ROWSLOT = 1,       // 7 words: slot(1 << chunk bit of row bit i)
    B_TOFF = 8,          // 32 words: slot(chunk offset of target index j)
    kBlkWords = 40
};

// B image of block b at H_BOFF + b * kBImgWords: the real embedding
// [[Ur, -Ui], [Ui, Ur]] (N = 64 output reals x K = 64 input reals) as TF32
// hi (rows 0..63) stacked over lo (rows 64..127), one 128-row operand in the
// K-major core-matrix layout
constexpr int kBImgWords = 2 * 64 * 64;

// Shared-memory slot of chunk amplitude x (8-byte complex64 units): the two
// high nibbles fold into the low one, so 16 lanes whose chunk bits have
// distinct residues mod 4 hit distinct bank pairs.
DPROG_HD inline uint32_t slot(uint32_t x)
{
    return x ^ ((x >> 4) & 15u) ^ ((x >> 8) & 15u);
}

}  // namespace dprog
}  // namespace svs
