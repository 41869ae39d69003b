/*
 * svsim.h -- C ABI of the GB300 (sm_103a) full state-vector simulator.
 *
 * The library simulates a quantum circuit on a 2^n-amplitude complex state
 * vector resident in GPU memory (Eq. 1 of the paper: |phi> = sum_i a_i |i>,
 * qubit j = bit j of the index i).  A circuit is restructured on the host by
 * the optimizer of Section 4.2 (Algorithm 4: diagonal detector, merge booster,
 * gate-block search for cache blocking and fusion) and executed by the
 * adaptive simulator of Section 4.3 (Algorithm 5) as a sequence of CUDA
 * kernels: fused-diagonal phase sweeps, cache-blocked chunk sweeps, tensor
 * products and read-out reductions.
 *
 * Conventions (apply to every function below):
 *  - Every function returns a sim_status; nothing throws across the ABI.  On
 *    failure the handle's message is available from sim_last_error() (or
 *    sim_global_error() when no handle exists yet).
 *  - Host arrays passed in are borrowed: read (or written) only during the
 *    call.  Device memory belongs to the handle, except the buffer given to
 *    sim_create_on(), which stays the caller's.
 *  - Calls on one handle are ordered on the handle's CUDA stream; a handle is
 *    not thread-safe, separate handles are independent.  Functions that
 *    return host results synchronise the handle's stream before returning.
 *  - Amplitudes are interleaved (re, im): float pairs for SIM_C64, double
 *    pairs for SIM_C128.  Indices are 64-bit.
 *  - n is limited to 1..34 for SIM_C64 and 1..33 for SIM_C128
 *    (SIM_EUNSUPPORTED beyond); qubit indices of a gate must be < n and
 *    distinct (SIM_EINVAL otherwise).
 */
#ifndef SVSIM_H
#define SVSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sim_t sim_t;

/* Amplitude type of a state vector.  The paper runs complex128 (Section 5.1).
 * SIM_C64: float (re, im) pairs; sweeps compute in FP32, with FP64 for fused
 * matrix composition and every reduction.  SIM_C128: double (re, im) pairs in
 * memory and at the ABI; the cache-blocked, phase and dense-block kernels
 * compute in double-float -- each real as an unevaluated sum of two floats,
 * about 48 significant bits (this GPU's FP64 rate is 1/64 of its FP32 rate)
 * -- except dense blocks asked for SIM_DENSE_FP64 (true FP64), the
 * gate-by-gate kernels and the reductions, which run FP64. */
typedef enum { SIM_C64 = 0, SIM_C128 = 1 } sim_dtype;

typedef enum {
    SIM_OK = 0,
    SIM_EINVAL = 1,        /* bad argument or gate                         */
    SIM_ENOMEM = 2,        /* device or host allocation failed / no room    */
    SIM_ECUDA = 3,         /* a CUDA call failed (message has the CUDA text) */
    SIM_ETIMEOUT = 4,      /* a bounded wait ran out                        */
    SIM_EBUSY = 5,         /* resource in use                               */
    SIM_EUNSUPPORTED = 6   /* size or feature outside what is built         */
} sim_status;

/* Gate kinds (Section 2.2 names the gates; matrices are the textbook ones:
 * RX(t) = exp(-i t X/2), RY(t) = exp(-i t Y/2), RZ(t) = exp(-i t Z/2),
 * P(t) = diag(1, e^{it}), CP(t) = diag(1,1,1,e^{it}), RZZ(t) = exp(-i t ZZ/2),
 * CX with q[0] the control).  For a gate on q[0..k-1], bit i of the local
 * matrix index belongs to qubit q[i] (Eqs. 2-3). */
typedef enum {
    G_H = 0, G_X, G_Y, G_Z, G_S, G_T, G_RX, G_RY, G_RZ, G_P,
    G_CX, G_CZ, G_CP, G_RZZ, G_SWAP,
    G_U1Q,       /* 2x2 matrix in .matrix                                   */
    G_UNITARY,   /* 2^k x 2^k matrix in .matrix, k = nq (1..6)              */
    G_DIAG       /* 2^k diagonal entries in .matrix, k = nq (1..6)          */
} sim_gate_kind;

/* One gate.  .matrix (U1Q, UNITARY: row-major; DIAG: the diagonal) holds
 * interleaved (re, im) doubles and is borrowed for the call; it is ignored
 * for named gates.  Angles are in radians in .param[0]. */
typedef struct {
    uint32_t kind;
    uint32_t nq;          /* number of qubits (named gates: may be 0 = default) */
    uint32_t q[6];
    double param[3];
    const double *matrix;
} sim_gate;

/* Optimizer switches (Algorithm 4 stages), combinable. */
enum {
    SIM_F_DIAG = 1u << 0,   /* diagonal detector (Algorithm 8)                */
    SIM_F_BOOST = 1u << 1,  /* merge booster (Algorithms 6-7)                 */
    SIM_F_BLOCK = 1u << 2,  /* cache blocking (gate-block search, Algorithm 2) */
    SIM_F_FUSE = 1u << 3,   /* cost-based gate fusion inside blocks           */
    SIM_F_TC = 1u << 4,     /* dense fused blocks on the tensor cores          */
    SIM_F_REMAP = 1u << 5,  /* qubit reordering (Section 2.3) by block stores:
                               the qubits of a block needed soonest by later
                               gates move into the low positions, which the
                               next block holds anyway; no extra sweep (one
                               restoring sweep at most).  Opt-in: fewer sweeps
                               on nearest-neighbour layered circuits, heavier
                               sweeps on random ones                          */
    SIM_F_JIT = 1u << 6,    /* complex64 cache-blocked and fused-diagonal
                               sweeps run kernels specialised to their
                               program: ops decoded once on the host and
                               compiled (NVRTC, needs libnvrtc.so.13) into
                               straight-line code.  A kernel holds the
                               program's structure (op kinds, positions,
                               layouts, table shapes); its numbers (matrix
                               entries, phase weights) are passed per launch,
                               so circuits that differ only in their angles
                               share kernels.  Kernels are cached for the
                               process (sim_jit_cache bounds how many); the
                               first apply of a new structure pays its compile
                               (1-3 s for 25-40-op sweeps, up to tens of
                               seconds for the largest, in parallel over a
                               plan's programs; the environment variable
                               SVSIM_JIT_FAST_COMPILE=min|mid|max trades run
                               time for compile time).  Results equal the
                               interpreter kernels' up to rounding order      */
    SIM_F_ALL = 0x7f
};

/* Arithmetic of dense fused 5-qubit blocks (SIM_F_TC).  complex64 states:
 * SIM_DENSE_SPLIT_TF32 on the tensor cores (three TF32 products, FP32
 * accumulation) or SIM_DENSE_FP32 on the CUDA cores (the other two values run
 * FP32 too).  complex128 states: SIM_DENSE_FP64 runs true FP64 on the FP64
 * pipe; every other value runs double-float on the FP32 pipe (about 48
 * significant bits, several times faster here). */
enum { SIM_DENSE_SPLIT_TF32 = 0, SIM_DENSE_FP32 = 1, SIM_DENSE_FP64 = 2, SIM_DENSE_DOUBLE_FLOAT = 3 };

/* The environment of Section 4.1 (N comes from the handle, R is 0: one GPU). */
typedef struct {
    int max_fuse_qubits;   /* F: largest fused dense block (default 2)            */
    int max_diag_qubits;   /* D: largest fused diagonal, 0 = unbounded (default 0) */
    int chunk_qubits;      /* C: qubits per cached chunk (0 = default: 12 c64, 11 c128) */
    int booster_div;       /* B: Divider uses divSize = (n+B-1)/B; 0 = divSize C   */
    uint32_t flags;        /* SIM_F_* (default SIM_F_DIAG|BOOST|BLOCK|FUSE)       */
    int dense_precision;   /* SIM_DENSE_* for the tensor-core path                 */
    int max_stages;        /* register stages per cached chunk (default 4)         */
    int register_bits;     /* chunk bits held in registers per thread (0 = default) */
    int reserved[4];
} sim_options;

/* Counts of the last executed plan (Section 5's "state vector updates"). */
typedef struct {
    uint64_t gates_in;       /* gates in the circuit                              */
    uint64_t ops;            /* kernel launches on the state                      */
    uint64_t sweeps;         /* full read+write passes over the 2^n state          */
    uint64_t chunk_ops, diag_ops, gate_ops, dense_ops, tensor_ops, permute_ops;
    uint64_t diag_fused;     /* gates absorbed by the diagonal detector           */
    uint64_t boosted_gates;  /* gates run on merge-booster sub-states              */
    uint64_t state_updates;  /* sum over ops of amplitudes touched (Section 3)     */
    uint64_t bytes;          /* algorithmic HBM bytes of the plan                  */
    double flops;            /* algorithmic floating-point operations              */
    double plan_ms;          /* host optimizer time                                */
    uint64_t tensor_fused;   /* tensor products computed by the next sweep's loads
                                (counted in tensor_ops, not launched)              */
} sim_plan_stats;

/* ------------------------------------------------------------ lifecycle */

/* Fill *opt with the defaults listed in sim_options. */
int sim_default_options(sim_options *opt);

/* Allocate a 2^n state of the given dtype on the current CUDA device, set it
 * to |0...0> and create a private stream.  The state is Eq. 1's vector
 * |phi> = sum_{i in [0, 2^N)} a_i |i> (Section 2.1), a_i stored at index i,
 * qubit j = bit j of i.  SIM_ENOMEM if 2^n * bytes/amp
 * exceeds free device memory. */
int sim_create(int n_qubits, sim_dtype dtype, sim_t **out);

/* Like sim_create, but on a caller-owned device buffer of >= 2^n amplitudes
 * (bytes is its size) and a caller-owned stream (cudaStream_t, may be NULL
 * for the legacy default stream).  The buffer is set to |0...0>. */
int sim_create_on(int n_qubits, sim_dtype dtype, void *dev_buf, size_t bytes,
                  void *cuda_stream, sim_t **out);

int sim_destroy(sim_t *s);

/* Set the state to the computational basis state |basis_index>.  The merge
 * booster (Section 4.4) needs a product state and is only used while the
 * state is known to be one (after create / reset). */
int sim_reset(sim_t *s, uint64_t basis_index);

/* Apply n gates (borrowed host array) with the given options (NULL =
 * defaults).  Plans on the host (Algorithm 4) and enqueues the kernels
 * (Algorithm 5) on the handle's stream; returns once enqueued. */
int sim_apply_circuit(sim_t *s, const sim_gate *gates, size_t n,
                      const sim_options *opt);

/* Wait for all work enqueued on the handle. */
int sim_sync(sim_t *s);

/* ------------------------------------------------------------ read-out */

/* p_x = |a_x|^2 for all 2^n x, as doubles, into a host array of 2^n: the
 * final probability distribution that full-state simulation yields (Section
 * 1's motivation for full-state simulation), from Eq. 1's amplitudes. */
int sim_probabilities(sim_t *s, double *out);

/* The k (1..1024) largest probabilities, ties to the lower index, largest
 * first: idx[k], prob[k] host arrays (Section 2.1: p_x = |a_x|^2, in FP64).
 * Exact.  For complex64 and 16 < k <= 128 the state is read once with
 * warps that keep only their best 16 candidates, and a second time only
 * when one warp's slice holds 16 of the result (a top k crowded into one
 * region, e.g. a uniform state's ties).  Synchronises the handle's stream. */
int sim_top_k(sim_t *s, int k, uint64_t *idx, double *prob);

/* <Z-string m> = sum_x |a_x|^2 (-1)^popcount(x & m) for n_terms masks: the
 * expectation of the Pauli-Z product on the qubits set in m, a read-out of
 * the probability distribution above (each qubit j in m contributes the
 * sign of Z on bit j of the basis index, Section 2.1).  Partial sums in a
 * fixed order, FP64 across blocks; masks with bits >= n are rejected. */
int sim_expectation(sim_t *s, const uint64_t *z_masks, size_t n_terms, double *out);

/* Both read-outs above in one call: the k largest probabilities (as
 * sim_top_k) and n_terms <Z-string> values (as sim_expectation, 16 strings
 * per pass; out may be NULL when n_terms = 0).  The top-k and the first 16 strings'
 * sums run concurrently on the handle's stream and a second stream the
 * handle creates on first use, and one synchronisation waits for both; the
 * results equal those of the two separate calls.  Synchronises the handle's
 * stream. */
int sim_top_k_expectation(sim_t *s, int k, uint64_t *idx, double *prob, const uint64_t *z_masks, size_t n_terms,
                          double *out);

/* Squared norm sum_x |a_x|^2, accumulated in FP64 (Section 2.1: the state
 * vector has unit L2 norm; this reads how far rounding moved it). */
int sim_norm(sim_t *s, double *out);

/* <Z-string m> like sim_expectation, for callers that cannot allocate device
 * memory when they need the result -- code running inside an allocator or
 * memory-pool callback, embedded callers whose device memory is owned and
 * budgeted by a host framework, programs that forbid allocation after
 * start-up.  It allocates nothing (no cudaMalloc / cudaFree, no allocating
 * library call): the reduction partials live in a fixed device array of
 * 128 KiB compiled into the library, present on every device that loads it
 * until the process exits.  (The paper has no counterpart; this is an
 * interface convenience.)
 *
 *   dev_state  2^n amplitudes in device memory (interleaved, dtype's precision)
 *   dev_masks  n_terms Z-string masks in device memory (bits < n_qubits)
 *   n_terms    1..16 (the fixed array's capacity; SIM_EINVAL beyond)
 *   dev_out    n_terms doubles in device memory, written when the stream
 *              reaches the kernels (the call only enqueues them)
 *   cuda_stream the cudaStream_t to run on (NULL: legacy default stream)
 *
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  Every
 * call on a device shares the one array: calls whose kernels overlap on the
 * GPU (different streams, no ordering between them) race and must be
 * serialised by the caller.  Each call overwrites every partial it reads, so
 * nothing needs clearing.  Errors: SIM_EINVAL / SIM_EUNSUPPORTED for bad
 * arguments, SIM_ECUDA for a failed CUDA call; the message is available from
 * sim_noalloc_error(). */
int sim_expectation_noalloc(const void *dev_state, int n_qubits, sim_dtype dtype,
                            const uint64_t *dev_masks, size_t n_terms, double *dev_out,
                            void *cuda_stream);
const char *sim_noalloc_error(void);

/* Copy the state out of / into host memory (bytes = 2^n * bytes/amp): Eq. 1's
 * amplitudes a_i in index order, interleaved (re, im).  SIM_EINVAL when bytes
 * is not the state's size.  sim_set_state ends the product-state knowledge
 * (the merge booster of Section 4.4 needs a product state: none after it). */
int sim_get_state(sim_t *s, void *host, size_t bytes);
int sim_set_state(sim_t *s, const void *host, size_t bytes);

/* Device pointer of the state and its CUDA stream (for zero-copy use). */
int sim_state_device(sim_t *s, void **dev_ptr, void **cuda_stream);

int sim_last_plan_stats(const sim_t *s, sim_plan_stats *out);

/* Per-kernel-kind device time, recorded with CUDA events around every launch
 * on the handle's stream while enabled.  Index = kind for launches on the
 * state, 8 + kind for launches on merge-booster sub-states: 0 basis init,
 * 1 gate-by-gate dense gate, 2 gate-by-gate diagonal gate, 3 fused diagonal
 * sweep, 4 cache-blocked chunk sweep, 5 tensor product, 6 dense block,
 * 7 small-register phase.  `bytes` is the algorithmic HBM traffic of those
 * launches (2 x 2^n x bytes/amp per read+write sweep, 2^n x bytes/amp for a
 * write-only tensor product or basis init). */
typedef struct {
    uint64_t launches[16];
    double ms[16];
    double bytes[16];
    uint64_t h2d_bytes;      /* plan constants copied host -> device          */
} sim_profile;

/* on != 0: clear the counters and start recording; 0: stop.  on = 2
 * records only the launches on the handle's own state, not those on the
 * merge booster's sub-states (two events fewer around each of those small
 * launches); their counters stay zero. */
int sim_profile_enable(sim_t *s, int on);
/* Synchronise the handle's stream and return the accumulated counters. */
int sim_profile_read(sim_t *s, sim_profile *out);
/* Kernels this library has launched in this process, over all handles,
 * servers and threads (a launch that failed to enqueue is not counted).  A
 * diagnostic with no counterpart in the paper; never fails. */
uint64_t sim_kernel_launches(void);
/* Self-test of the bounded waits of the two tensor-core kernels (the dense
 * block sweep and the cache-blocked dense-block sweep), on the current
 * device.  It runs each kernel with its MMA issue suppressed, so that every
 * mbarrier wait gives up after a few thousand polls, and checks three things:
 * the kernel sets its status word, leaves the state untouched and frees its
 * tensor memory; and a normal launch afterwards still works.  SIM_OK when all
 * hold; otherwise the failing check is in sim_global_error().  Allocates
 * about 100 KB of device memory.  No counterpart in the paper. */
int sim_selftest_wait_timeout(void);
const char *sim_last_error(const sim_t *s);
const char *sim_global_error(void);

/* Host-side fault injection for tests (no counterpart in the paper).  Lets
 * the next `skip` operations of a kind through and arms the `count` after
 * them to fail as if the device had refused them, without touching the GPU: SIM_FAULT_ALLOC -- the library's device
 * allocations (states, merge-booster sub-states, plan constants, read-out
 * scratch, serving buffers) return SIM_ENOMEM without calling cudaMalloc;
 * SIM_FAULT_LAUNCH -- sim_apply_circuit skips the launch and returns
 * SIM_ECUDA (the state is then undefined, the handle stays usable).
 * count = 0 disarms.  The environment variable SVSIM_FAULT = "alloc:N" or
 * "launch:N" arms N failures (no skip) at load.  SIM_EINVAL for an unknown
 * kind or a negative number. */
enum { SIM_FAULT_ALLOC = 1, SIM_FAULT_LAUNCH = 2 };
int sim_fault_inject(int kind, int skip, int count);

/* ------------------------------------------------------------ planner only */

/* Run the optimizer alone (no GPU needed) for an n-qubit circuit starting
 * from the product state |basis_index> (pass UINT64_MAX for "unknown state":
 * no booster) and write a JSON description of the plan into buf (at most
 * buflen bytes including the terminating NUL).  *needed receives the full
 * length + 1; returns SIM_ENOMEM (and fills nothing) when buflen is too small.
 * Used to check the optimizer's algebra on the CPU. */
int sim_plan_json(int n_qubits, sim_dtype dtype, uint64_t basis_index,
                  const sim_gate *gates, size_t n, const sim_options *opt,
                  char *buf, size_t buflen, size_t *needed);

/* Plan the circuit as sim_plan_json does and generate and compile (NVRTC,
 * no GPU needed) the specialised kernel of every chunk sweep that SIM_F_JIT
 * would run; *n_programs receives their count.  SIM_EINVAL with the
 * compiler's log in sim_global_error() when one does not compile. */
int sim_jit_check(int n_qubits, sim_dtype dtype, uint64_t basis_index, const sim_gate *gates, size_t n,
                  const sim_options *opt, int *n_programs);

/* Specialised kernels cached by this process now, and the wall time all
 * compiles so far took (ms). */
int sim_jit_info(uint64_t *programs, double *compile_ms);

/* The specialised-kernel cache (no counterpart in the paper; a resource
 * control).  max_kernels > 0 sets the most kernels kept loaded (default 256;
 * least recently used first out -- an evicted kernel's module is unloaded
 * once no launch can use it, after synchronising the devices it ran on);
 * 0 leaves it.  *kernels: cached now; *compiles: NVRTC compiles so far. */
int sim_jit_cache(int max_kernels, uint64_t *kernels, uint64_t *compiles);

/* The generated CUDA source of every specialised sweep of the plan (as
 * sim_plan_json plans it; no GPU needed), each after a comment line giving
 * its parameter-block size, into buf (at most buflen bytes including the
 * terminating NUL); *needed receives the full length + 1, SIM_ENOMEM (and
 * nothing written) when buflen is too small.  Two circuits that differ only
 * in their angles have equal sources. */
int sim_jit_sources(int n_qubits, sim_dtype dtype, uint64_t basis_index, const sim_gate *gates, size_t n,
                    const sim_options *opt, char *buf, size_t buflen, size_t *needed);

/* ------------------------------------------------------------ serving */
/* A request loop with continuous batching (not in the paper; the serving
 * pattern around its simulator).  Requests are admitted as they arrive:
 * circuits small enough for one CTA's shared memory (n <= 13 complex64,
 * n <= 12 complex128, gates of <= 3 qubits, top_k <= 128) are packed into
 * one kernel launch, one CTA per circuit, state kept on chip; larger ones run
 * the full optimizer + kernel pipeline on one of n_streams worker streams,
 * admitted only while the sum of their state footprints (2^n x bytes/amp)
 * stays within hbm_budget.  Batches and worker streams overlap on the GPU. */
typedef struct srv_t srv_t;

typedef struct {
    int n_qubits;
    sim_dtype dtype;
    const sim_gate *gates;     /* copied by srv_submit (matrices included) */
    size_t n_gates;
    uint64_t basis;            /* initial basis state */
    int top_k;                 /* 0..1024 largest probabilities to return   */
    const uint64_t *z_masks;   /* copied; <Z-string> values to return       */
    size_t n_masks;            /* 0..64                                     */
} srv_request;

typedef struct {
    int status;                /* SIM_OK or the request's error code        */
    int top_k;
    int n_masks;
    int path;                  /* 0 shared-memory batch, 1 full-state pipeline */
    uint64_t top_idx[1024];    /* ties to the lower index, largest first    */
    double top_p[1024];
    double expect[64];
    double latency_ms;         /* submit -> result ready                   */
    double queue_ms;           /* submit -> start of its GPU work          */
} srv_result;

typedef struct {
    uint64_t submitted, completed, failed;
    uint64_t batched, batches; /* requests run by batch launches, launches  */
    double p50_ms, p99_ms, mean_ms, max_ms;   /* latency of completed requests */
    double elapsed_s;          /* first submit -> last completion           */
    double circuits_per_s;
    size_t hbm_budget, hbm_peak;   /* admitted state bytes: budget and peak */
} srv_stats;

/* Start a server on the current device.  n_streams worker streams (>= 1)
 * for full-state requests plus one batch stream.  The paper has no serving
 * loop; each request is one run of the simulator above (Algorithms 4-5 on
 * its circuit) and its read-outs.  SIM_EINVAL for n_streams outside 1..64 or
 * a zero budget, SIM_ENOMEM when host memory runs out, SIM_ECUDA when a
 * stream cannot be created. */
int srv_create(size_t hbm_budget_bytes, int n_streams, srv_t **out);
/* Queue a request (copied).  SIM_EINVAL for malformed requests, SIM_ENOMEM
 * when its state alone exceeds the budget.  *ticket identifies it. */
int srv_submit(srv_t *s, const srv_request *req, uint64_t *ticket);
/* Wait up to timeout_ms (-1: forever) for a ticket's result; SIM_ETIMEOUT if
 * it is not ready.  A returned result releases the ticket. */
int srv_poll(srv_t *s, uint64_t ticket, srv_result *out, int timeout_ms);
int srv_get_stats(srv_t *s, srv_stats *out);
/* Finish the queued work, stop the threads, free everything. */
int srv_destroy(srv_t *s);

#ifdef __cplusplus
}
#endif
#endif /* SVSIM_H */
