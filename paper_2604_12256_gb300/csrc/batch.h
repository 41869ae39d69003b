// batch.h -- small-circuit batches of the serving loop: one CTA per request,
// the whole circuit on a shared-memory state (k_batch.cu), and the host side
// that packs requests into one launch (serve.cpp).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace svs {

constexpr int kBatchThreads = 256;
constexpr int kBatchMaxN64 = 13;     // 2^13 x (8 + 8) B = 128 KiB shared memory
constexpr int kBatchMaxN128 = 12;    // 2^12 x (16 + 8) B =  96 KiB
constexpr int kBatchMaxTopK = 128;
constexpr int kBatchMaxGateQubits = 3;

// ops: hdr = type | k << 8 | length_in_words << 16
enum { BOP_DENSE = 1, BOP_PHASE = 2 };
// BOP_DENSE: hdr, q0, q1, q2, then 2 x 4^k reals (float or double), row-major
// BOP_PHASE: hdr, n_terms, then n_terms x {mask_lo, mask_hi, w_lo, w_hi}
//            (w: uint64 fixed-point turns)

struct BatchReq {
    int n;
    int nops;
    uint32_t ops_off;      // word offset of the first op in the blob
    uint32_t masks_off;    // word offset of nmask uint64 Z masks
    int nmask;
    int top_k;
    uint64_t basis;
    uint64_t out_off;      // double offset: nmask <Z>, top_k p, top_k indices
};

size_t batch_smem_bytes(int n, bool f64);
cudaError_t launch_batch(const BatchReq *reqs_dev, int nreq, int max_n, const uint32_t *blob_dev, double *outs_dev,
                         bool f64, cudaStream_t st);

}  // namespace svs
