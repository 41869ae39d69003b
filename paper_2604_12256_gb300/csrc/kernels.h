// kernels.h -- host-side launchers of the CUDA kernels (one translation unit
// per kernel family).  All launchers enqueue on `st` and return the launch
// status; none allocates memory.  `a` is the interleaved complex state of 2^n
// amplitudes (float2 for is_f64 == false, double2 otherwise).
#pragma once

#include <cstdint>
#include <string>
#include <memory>
#include <vector>

#include <cuda_runtime.h>

namespace svs {

constexpr int kNumSMs = 152;   // sizing fallback when the device query fails

// Kernels launched by this library in this process: every launcher adds the
// number of kernels it enqueued when the launch succeeded.
cudaError_t counted(cudaError_t e, int kernels);
uint64_t launches_total();

// |basis> : zero the vector and set one amplitude to 1 (write-only sweep)
cudaError_t launch_init_basis(void *a, int n, bool is_f64, uint64_t basis, cudaStream_t st);

// One k-qubit dense gate over the whole vector (Algorithm 1).  q: the gate's
// qubits (local bit i <-> q[i]); dmat: device matrix, 2^k x 2^k row-major
// complex of the state's precision.
cudaError_t launch_gate_dense(void *a, int n, bool is_f64, int k, const int *q,
                              const void *dmat, cudaStream_t st);

// One diagonal gate: multiply only the amplitudes whose local index c has
// d[c] != 1.  nz: number of such c; cidx: their local indices (host array,
// <= 64); dvals: device array of nz complex factors (state precision).
cudaError_t launch_gate_diag(void *a, int n, bool is_f64, int k, const int *q, int nz,
                             const int *cidx, const void *dvals, cudaStream_t st);

// out[h * 2^n_lo + l] = hi[h] * lo[l]  (the merge of Algorithm 7 / K7)
cudaError_t launch_tensor(void *out, const void *hi, int n_hi, const void *lo, int n_lo,
                          bool is_f64, cudaStream_t st);

// ---- read-out (FP64 accumulation, fixed reduction order) ----
// Partials buffer `part` must hold reduce_partials() (= kReduceBlocks)
// doubles per term.  The reductions' grids are fixed, so every sum's order
// is independent of the device: the norm runs 1024 blocks of 256 threads,
// the <Z> kernel 512 (a power-of-two stride either way; fewer blocks halve
// the <Z> kernel's per-block setup and 16-term block reductions, while the
// light norm kernel needs the blocks to keep enough loads in flight).
constexpr int kReduceBlocks = 1024;
int reduce_partials();
// sum_x |a_x|^2 -> *out_dev (device double)
cudaError_t launch_norm(const void *a, int n, bool is_f64, double *part, double *out_dev,
                        cudaStream_t st);
// <Z_m> for nt <= 16 masks (device array) -> out_dev[nt]
cudaError_t launch_expect_z(const void *a, int n, bool is_f64, const uint64_t *masks_dev, int nt,
                            double *part, double *out_dev, cudaStream_t st);
// p_x for all x -> out_dev[2^n]
cudaError_t launch_probs(const void *a, int n, bool is_f64, double *out_dev, cudaStream_t st);
// top-k (k <= 1024): scratch must hold topk_scratch_bytes(k); results to
// idx_dev[k], p_dev[k] (largest first, ties to the lower index).
// warp_keep = kTopWarpKeep (< k) lets the complex64 kernel's warps keep only
// their best kTopWarpKeep candidates; *warp_slice then receives the
// amplitudes per warp slice (else 0), and the result is exact unless
// topk_warp_suspect() holds for it, when the call must be repeated with
// warp_keep = 0.
constexpr int kTopWarpKeep = 16;
size_t topk_scratch_bytes(int k);
cudaError_t launch_topk(const void *a, int n, bool is_f64, int k, void *scratch,
                        uint64_t *idx_dev, double *p_dev, cudaStream_t st, int warp_keep = 0,
                        int64_t *warp_slice = nullptr);
// true when some warp slice holds >= keep of the k result indices (it may
// have dropped an element of the true top k)
bool topk_warp_suspect(const uint64_t *idx, int k, int64_t slice, int keep);

// ---- optimizer-driven sweeps ----
// Optional input of a sweep: instead of reading the state, amplitude x is
// hi[x >> n_lo] * lo[x & (2^n_lo - 1)], the merge-booster tensor product
// (Algorithm 7) that feeds this sweep and is never written on its own.
// hi == nullptr: the sweep reads the state.  hi, lo: device sub-states of the
// state's precision, 2^(n - n_lo) and 2^n_lo amplitudes.
struct TensorSrc {
    const void *hi = nullptr;
    const void *lo = nullptr;
    int n_lo = 0;
};

// Fused diagonal phase sweep (K3) and cache-blocked chunk sweep (K4): `prog`
// is a device program written by the encoder in program.h.
// `smem` = prog::smem_bytes() of the program (dynamic shared memory).
cudaError_t launch_diag_sweep(void *a, int n, bool is_f64, const uint32_t *prog, size_t smem, TensorSrc src,
                              cudaStream_t st);
cudaError_t launch_chunk(void *a, int n, bool is_f64, int C, int RB, const uint32_t *prog, size_t smem,
                         TensorSrc src, cudaStream_t st);

// Chunk sweeps specialised to one program (jit.cpp; complex64, C = 12,
// RB = 4 or 5): jit_prepare finds (or generates and compiles with NVRTC, in
// parallel) the kernel of each host program and the values of its parameter
// block; launch_chunk_jit runs it on the device copy `prog` of program `w`,
// with the same arguments and results as launch_chunk.  Fused diagonal
// sweeps (K3, complex64, RB = 4) likewise: launch_diag_jit has
// launch_diag_sweep's arguments and results.  Kernels are keyed by their
// generated source, which holds the program's structure only (its numbers
// are parameters), and kept at most jit_set_cache_limit() at a time.
// JIT_CHUNK_FED: a chunk program whose sweep computes its input from a fused
// merge-booster product (it must be launched with that product's factors).
enum { JIT_CHUNK = 0, JIT_DIAG = 1, JIT_CHUNK_FED = 2 };
struct JitProg {
    const std::vector<uint32_t> *w;   // host program words
    int kind;                         // JIT_CHUNK, JIT_DIAG or JIT_CHUNK_FED
};
struct JitKernel;
struct JitHandle {
    std::shared_ptr<JitKernel> k;                        // null: run the interpreter kernel
    std::shared_ptr<const std::vector<uint32_t>> vals;   // the launch's parameter block
};
bool jit_supported(bool is_f64, int C, int RB);
bool jit_supported_diag(bool is_f64, int RB);
bool jit_prepare(const std::vector<JitProg> &progs, std::vector<JitHandle> &out, std::string &err);
cudaError_t launch_chunk_jit(const JitHandle &h, void *a, int n, const std::vector<uint32_t> &w, const uint32_t *prog,
                             size_t smem, TensorSrc src, cudaStream_t st);
cudaError_t launch_diag_jit(const JitHandle &h, void *a, int n, const std::vector<uint32_t> &w, const uint32_t *prog,
                            size_t smem, TensorSrc src, cudaStream_t st);
// kernels cached now; total compiles and their wall time (ms) so far
size_t jit_cache_size(double *compile_ms, uint64_t *compiles);
void jit_set_cache_limit(size_t max_kernels);
// the generated source with its parameter values, and its NVRTC compile (no device needed)
bool jit_source(const std::vector<uint32_t> &w, int kind, std::string &src, std::vector<uint32_t> &vals,
                std::string &err);
bool jit_compile(const std::string &src, std::vector<char> &cubin, std::string &err);

// Phase polynomial on small registers: one thread per amplitude sums the
// nt terms (device array of {mask, w} pairs, uint64 turns).
cudaError_t launch_phase_small(void *a, int n, bool is_f64, const uint64_t *terms_dev, int nt, cudaStream_t st);

// Dense 5-qubit block (K6): q = the 5 qubits (local bit i <-> q[i]), U64 =
// device 32 x 32 row-major complex matrix in FP64.  precision: 0 split-TF32
// on the tensor cores, 1 FP32 CUDA cores (complex64 states); complex128
// states: 2 FP64 on the FP64 pipe, anything else double-float on the FP32
// pipe (about 48 significant bits).  status: device int set to 1 when a bounded wait
// of the tensor-core kernel gave up.
cudaError_t launch_dense5(void *a, int n, bool is_f64, int precision, const int *q, const void *U64, int *status,
                          cudaStream_t st);
// Cache-blocked dense-block sweep (K6 inside K4, complex64, split-TF32 on the
// tensor cores): the blocks of the device program `prog` (dense_prog.h, in
// device memory, 16-byte aligned) applied chunk by chunk in one pass over the
// 2^n state.  status: device int set to 1 when a bounded wait gave up.
cudaError_t launch_dense_chunk(void *a, int n, const uint32_t *prog, int *status, cudaStream_t st);
// Self-test only: the same kernel with its MMA issue suppressed.
cudaError_t launch_dense_chunk_wait_selftest(void *a, int n, const uint32_t *prog, int *status, uint32_t wait_limit,
                                             cudaStream_t st);
// Self-test only: the tensor-core block kernel with its MMA issue suppressed,
// so that its bounded waits (wait_limit polls each) run out; *status -> 1.
cudaError_t launch_dense5_wait_selftest(void *a, int n, const void *U64, int *status, uint32_t wait_limit,
                                        cudaStream_t st);

int device_sm_count();

}  // namespace svs
