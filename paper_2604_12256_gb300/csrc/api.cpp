// api.cpp -- the C ABI of include/svsim.h and the executor (the adaptive
// simulation of Algorithm 5): runs a plan's ops as kernel launches on the
// handle's stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "internal.h"
#include "kernels.h"
#include "program.h"

using namespace svs;

struct sim_t {
    int n = 0;
    sim_dtype dt = SIM_C64;
    void *state = nullptr;
    bool own_state = false;
    size_t state_bytes = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    bool product = true;        // state is the basis state `basis`
    bool reset_pending = true;  // |basis> not yet written (lazy: a booster plan overwrites it)
    uint64_t basis = 0;
    double *d_part = nullptr;   // reduction partials
    double *d_out = nullptr;    // small device results
    uint64_t *d_masks = nullptr;
    int *d_status = nullptr;    // set by kernels whose bounded waits gave up
    void *d_topk = nullptr;
    size_t topk_bytes = 0;
    unsigned char *d_const = nullptr;   // plan constants
    size_t const_bytes = 0;
    unsigned char *h_pin = nullptr;     // pinned staging of plan constants
    size_t pin_bytes = 0;
    cudaEvent_t pin_ev = nullptr;
    bool pin_pending = false;
    cudaStream_t aux = nullptr;         // second stream of the combined read-out
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::vector<void *> sub;            // booster sub-state buffers
    std::vector<size_t> sub_bytes;
    std::string err;
    sim_plan_stats stats{};
    // profiling: event pairs around launches, resolved at sim_profile_read
    bool prof_on = false;
    bool prof_all = true;       // false: only ops on the handle's state (not the booster's sub-states)
    sim_profile prof{};
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    struct Pend { int kind; size_t e0; double bytes; };
    std::vector<Pend> prof_pend;
};

static cudaEvent_t prof_event(sim_t *s, size_t i)
{
    while (s->ev_pool.size() <= i) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        s->ev_pool.push_back(e);
    }
    return s->ev_pool[i];
}

// record the start of a launch on buffer `buf` (0: the handle's state);
// returns the pair index, or -1 when it is not recorded
static long prof_begin(sim_t *s, int buf = 0)
{
    if (!s->prof_on || (buf != 0 && !s->prof_all)) return -1;
    size_t i = s->ev_used;
    cudaEvent_t a = prof_event(s, i), b = prof_event(s, i + 1);
    if (!a || !b) return -1;
    s->ev_used += 2;
    cudaEventRecord(a, s->stream);
    return (long)i;
}

static void prof_end(sim_t *s, long i, int kind, double bytes)
{
    if (i < 0) return;
    cudaEventRecord(s->ev_pool[i + 1], s->stream);
    s->prof_pend.push_back({kind, (size_t)i, bytes});
}

static thread_local std::string g_err;

static int fail(sim_t *s, int code, const std::string &msg)
{
    if (s) s->err = msg;
    g_err = msg;
    return code;
}

static int cuda_fail(sim_t *s, cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (e == cudaErrorMemoryAllocation) return fail(s, SIM_ENOMEM, m);
    return fail(s, SIM_ECUDA, m);
}

#define CK(s, call)                                     \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(s, e_, #call); \
    } while (0)

static size_t amp_bytes(sim_dtype dt) { return dt == SIM_C64 ? 8 : 16; }

static int check_n(int n, sim_dtype dt)
{
    if (dt != SIM_C64 && dt != SIM_C128) return fail(nullptr, SIM_EINVAL, "dtype must be SIM_C64 or SIM_C128");
    int mx = dt == SIM_C64 ? kMaxQubitsC64 : kMaxQubitsC128;
    if (n < 1) return fail(nullptr, SIM_EINVAL, "n_qubits must be >= 1");
    if (n > mx) return fail(nullptr, SIM_EUNSUPPORTED, "n_qubits above the supported maximum");
    return SIM_OK;
}

static int alloc_aux(sim_t *s)
{
    int np = reduce_partials();
    CK(s, dev_malloc((void **)&s->d_part, sizeof(double) * np * 16));
    CK(s, dev_malloc((void **)&s->d_out, sizeof(double) * 64));
    CK(s, dev_malloc((void **)&s->d_masks, sizeof(uint64_t) * 64));
    CK(s, dev_malloc((void **)&s->d_status, sizeof(int)));
    CK(s, cudaMemset(s->d_status, 0, sizeof(int)));
    CK(s, cudaEventCreateWithFlags(&s->pin_ev, cudaEventDisableTiming));
    return SIM_OK;
}

static void free_all(sim_t *s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->own_state && s->state) cudaFree(s->state);
    if (s->d_part) cudaFree(s->d_part);
    if (s->d_out) cudaFree(s->d_out);
    if (s->d_masks) cudaFree(s->d_masks);
    if (s->d_status) cudaFree(s->d_status);
    if (s->d_topk) cudaFree(s->d_topk);
    if (s->d_const) cudaFree(s->d_const);
    if (s->h_pin) cudaFreeHost(s->h_pin);
    if (s->pin_ev) cudaEventDestroy(s->pin_ev);
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    for (void *p : s->sub) if (p) cudaFree(p);
    if (s->aux) { cudaStreamSynchronize(s->aux); cudaStreamDestroy(s->aux); }
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->ev_join) cudaEventDestroy(s->ev_join);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

// after a synchronisation: report (and clear) a kernel's timed-out wait
static int check_status(sim_t *s)
{
    int st = 0;
    CK(s, cudaMemcpy(&st, s->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0) {
        CK(s, cudaMemset(s->d_status, 0, sizeof(int)));
        return fail(s, SIM_ETIMEOUT, "a kernel's bounded wait for the tensor cores timed out; results are invalid");
    }
    return SIM_OK;
}

// write the pending |basis> (sim_reset is lazy)
static int materialize(sim_t *s)
{
    if (!s->reset_pending) return SIM_OK;
    long pe = prof_begin(s);
    CK(s, launch_init_basis(s->state, s->n, s->dt == SIM_C128, s->basis, s->stream));
    prof_end(s, pe, OPK_INIT_BASIS, (double)s->state_bytes);
    s->reset_pending = false;
    return SIM_OK;
}

extern "C" {

int sim_default_options(sim_options *opt)
{
    if (!opt) return fail(nullptr, SIM_EINVAL, "null options");
    fill_default_options(*opt);
    return SIM_OK;
}

const char *sim_global_error(void) { return g_err.c_str(); }

uint64_t sim_kernel_launches(void) { return launches_total(); }

int sim_selftest_wait_timeout(void)
{
    const int n = 10;
    const size_t N = (size_t)1 << n;
    std::vector<float2> h(N), back(N);
    for (size_t i = 0; i < N; i++) h[i] = make_float2(0.001f * (float)i, -0.0005f * (float)i);
    std::vector<double2> u(32 * 32);
    for (int r = 0; r < 32; r++)
        for (int c = 0; c < 32; c++) u[r * 32 + c] = make_double2(r == (c ^ 1) ? 1.0 : 0.0, 0.0);   // X on qubit 0
    float2 *d_a = nullptr;
    double2 *d_u = nullptr;
    int *d_st = nullptr;
    cudaStream_t st = nullptr;
    std::string msg;
    int rc = SIM_OK, flag = 0;
    auto ck = [&](cudaError_t e, const char *where) {
        if (e != cudaSuccess && rc == SIM_OK) { rc = cuda_fail(nullptr, e, where); }
        return rc == SIM_OK;
    };
    const int q[5] = {0, 1, 2, 3, 4};
    if (ck(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream") &&
        ck(cudaMalloc((void **)&d_a, N * sizeof(float2)), "malloc") &&
        ck(cudaMalloc((void **)&d_u, u.size() * sizeof(double2)), "malloc") &&
        ck(cudaMalloc((void **)&d_st, sizeof(int)), "malloc") &&
        ck(cudaMemcpy(d_a, h.data(), N * sizeof(float2), cudaMemcpyHostToDevice), "copy") &&
        ck(cudaMemcpy(d_u, u.data(), u.size() * sizeof(double2), cudaMemcpyHostToDevice), "copy") &&
        ck(cudaMemset(d_st, 0, sizeof(int)), "memset") &&
        // 1. every wait runs out: the status word is set, the state untouched
        ck(launch_dense5_wait_selftest(d_a, n, d_u, d_st, 1u << 12, st), "self-test launch") &&
        ck(cudaStreamSynchronize(st), "self-test sync") &&
        ck(cudaMemcpy(&flag, d_st, sizeof(int), cudaMemcpyDeviceToHost), "status read") &&
        ck(cudaMemcpy(back.data(), d_a, N * sizeof(float2), cudaMemcpyDeviceToHost), "state read")) {
        if (flag != 1) { rc = SIM_EINVAL; msg = "the timed-out wait did not set the status word"; }
        for (size_t i = 0; rc == SIM_OK && i < N; i++)
            if (back[i].x != h[i].x || back[i].y != h[i].y) { rc = SIM_EINVAL; msg = "the aborted kernel wrote the state"; }
    }
    // 2. the context is still usable: a normal split-TF32 block is exact up to the TF32 split
    if (rc == SIM_OK && ck(cudaMemset(d_st, 0, sizeof(int)), "memset") &&
        ck(launch_dense5(d_a, n, false, SIM_DENSE_SPLIT_TF32, q, d_u, d_st, st), "block launch") &&
        ck(cudaStreamSynchronize(st), "block sync") &&
        ck(cudaMemcpy(&flag, d_st, sizeof(int), cudaMemcpyDeviceToHost), "status read") &&
        ck(cudaMemcpy(back.data(), d_a, N * sizeof(float2), cudaMemcpyDeviceToHost), "state read")) {
        if (flag != 0) { rc = SIM_ETIMEOUT; msg = "a normal block launch timed out after the self-test"; }
        for (size_t i = 0; rc == SIM_OK && i < N; i++) {
            const float2 want = h[i ^ 1];
            if (std::fabs(back[i].x - want.x) > 1e-6f * (1.f + std::fabs(want.x)) ||
                std::fabs(back[i].y - want.y) > 1e-6f * (1.f + std::fabs(want.y))) {
                rc = SIM_EINVAL;
                msg = "the block product after the self-test is wrong";
            }
        }
    }
    // 3-4. the same two checks for the cache-blocked dense-block sweep, on one
    // 2^12-amplitude chunk with one block (X on qubit 0)
    const int n2 = 12;
    const size_t N2 = (size_t)1 << n2;
    std::vector<float2> h2(N2), back2(N2);
    for (size_t i = 0; i < N2; i++) h2[i] = make_float2(0.0002f * (float)i, 0.0001f * (float)(N2 - i));
    float2 *d_a2 = nullptr;
    uint32_t *d_prog = nullptr;
    std::vector<uint32_t> words;
    {
        PGate g;
        g.kind = kFusedDense;
        g.k = 5;
        for (int i = 0; i < 5; i++) g.q[i] = i;
        g.qmask = 31;
        g.M.assign(32 * 32, cd(0, 0));
        for (int r = 0; r < 32; r++) g.M[(size_t)r * 32 + (r ^ 1)] = 1;
        int cq[16];
        for (int i = 0; i < 12; i++) cq[i] = i;
        words = encode_dense_chunk(n2, cq, std::vector<PGate>{g});
    }
    if (rc == SIM_OK && ck(cudaMalloc((void **)&d_a2, N2 * sizeof(float2)), "malloc") &&
        ck(cudaMalloc((void **)&d_prog, words.size() * 4), "malloc") &&
        ck(cudaMemcpy(d_a2, h2.data(), N2 * sizeof(float2), cudaMemcpyHostToDevice), "copy") &&
        ck(cudaMemcpy(d_prog, words.data(), words.size() * 4, cudaMemcpyHostToDevice), "copy") &&
        ck(cudaMemset(d_st, 0, sizeof(int)), "memset") &&
        ck(launch_dense_chunk_wait_selftest(d_a2, n2, d_prog, d_st, 1u << 12, st), "self-test launch") &&
        ck(cudaStreamSynchronize(st), "self-test sync") &&
        ck(cudaMemcpy(&flag, d_st, sizeof(int), cudaMemcpyDeviceToHost), "status read") &&
        ck(cudaMemcpy(back2.data(), d_a2, N2 * sizeof(float2), cudaMemcpyDeviceToHost), "state read")) {
        if (flag != 1) { rc = SIM_EINVAL; msg = "the timed-out dense-block sweep did not set the status word"; }
        for (size_t i = 0; rc == SIM_OK && i < N2; i++)
            if (back2[i].x != h2[i].x || back2[i].y != h2[i].y) { rc = SIM_EINVAL; msg = "the aborted sweep wrote the state"; }
    }
    if (rc == SIM_OK && ck(cudaMemset(d_st, 0, sizeof(int)), "memset") &&
        ck(launch_dense_chunk(d_a2, n2, d_prog, d_st, st), "sweep launch") &&
        ck(cudaStreamSynchronize(st), "sweep sync") &&
        ck(cudaMemcpy(&flag, d_st, sizeof(int), cudaMemcpyDeviceToHost), "status read") &&
        ck(cudaMemcpy(back2.data(), d_a2, N2 * sizeof(float2), cudaMemcpyDeviceToHost), "state read")) {
        if (flag != 0) { rc = SIM_ETIMEOUT; msg = "a normal dense-block sweep timed out after the self-test"; }
        for (size_t i = 0; rc == SIM_OK && i < N2; i++) {
            const float2 want = h2[i ^ 1];
            if (std::fabs(back2[i].x - want.x) > 1e-6f * (1.f + std::fabs(want.x)) ||
                std::fabs(back2[i].y - want.y) > 1e-6f * (1.f + std::fabs(want.y))) {
                rc = SIM_EINVAL;
                msg = "the dense-block sweep after the self-test is wrong";
            }
        }
    }
    if (st) cudaStreamSynchronize(st);
    if (d_a) cudaFree(d_a);
    if (d_u) cudaFree(d_u);
    if (d_a2) cudaFree(d_a2);
    if (d_prog) cudaFree(d_prog);
    if (d_st) cudaFree(d_st);
    if (st) cudaStreamDestroy(st);
    if (!msg.empty()) return fail(nullptr, rc, msg);
    return rc;
}

const char *sim_last_error(const sim_t *s) { return s ? s->err.c_str() : g_err.c_str(); }

static int create_common(int n, sim_dtype dt, void *buf, size_t bytes, void *stream, bool own, sim_t **out)
{
    if (!out) return fail(nullptr, SIM_EINVAL, "null output handle");
    *out = nullptr;
    int rc = check_n(n, dt);
    if (rc) return rc;
    sim_t *s = new (std::nothrow) sim_t();
    if (!s) return fail(nullptr, SIM_ENOMEM, "host allocation failed");
    s->n = n;
    s->dt = dt;
    s->state_bytes = ((size_t)1 << n) * amp_bytes(dt);
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) { cuda_fail(nullptr, e, "cudaGetDevice"); delete s; return SIM_ECUDA; }
    if (own) {
        size_t fr = 0, tot = 0;
        e = cudaMemGetInfo(&fr, &tot);
        if (e != cudaSuccess) { cuda_fail(nullptr, e, "cudaMemGetInfo"); delete s; return SIM_ECUDA; }
        if (s->state_bytes + (64ull << 20) > fr) {
            delete s;
            return fail(nullptr, SIM_ENOMEM, "state vector does not fit in free device memory");
        }
        e = dev_malloc((void **)&s->state, s->state_bytes);
        if (e != cudaSuccess) { delete s; return cuda_fail(nullptr, e, "cudaMalloc(state)"); }
        s->own_state = true;
        e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { free_all(s); return cuda_fail(nullptr, e, "cudaStreamCreate"); }
        s->own_stream = true;
    } else {
        if (!buf) { delete s; return fail(nullptr, SIM_EINVAL, "null device buffer"); }
        if (bytes < s->state_bytes) { delete s; return fail(nullptr, SIM_EINVAL, "device buffer too small"); }
        if (((uintptr_t)buf & 255) != 0) { delete s; return fail(nullptr, SIM_EINVAL, "device buffer must be 256-byte aligned"); }
        s->state = buf;
        s->stream = (cudaStream_t)stream;
    }
    rc = alloc_aux(s);
    if (rc) { std::string m = s->err; free_all(s); return fail(nullptr, rc, m); }
    s->reset_pending = true;
    s->basis = 0;
    *out = s;
    return SIM_OK;
}

int sim_create(int n_qubits, sim_dtype dtype, sim_t **out)
{
    return create_common(n_qubits, dtype, nullptr, 0, nullptr, true, out);
}

int sim_create_on(int n_qubits, sim_dtype dtype, void *dev_buf, size_t bytes, void *cuda_stream, sim_t **out)
{
    return create_common(n_qubits, dtype, dev_buf, bytes, cuda_stream, false, out);
}

}  // extern "C"

int svs_rebind(sim_t *s, int n, sim_dtype dt, void *buf, size_t bytes)
{
    if (!s || s->own_state) return fail(s, SIM_EINVAL, "rebind needs a handle on a caller buffer");
    int rc = check_n(n, dt);
    if (rc) return rc;
    const size_t need = ((size_t)1 << n) * amp_bytes(dt);
    if (!buf || bytes < need) return fail(s, SIM_EINVAL, "buffer too small");
    s->n = n;
    s->dt = dt;
    s->state = buf;
    s->state_bytes = need;
    s->product = true;
    s->basis = 0;
    s->reset_pending = true;
    return SIM_OK;
}

extern "C" {

int sim_destroy(sim_t *s)
{
    if (!s) return fail(nullptr, SIM_EINVAL, "null handle");
    free_all(s);
    return SIM_OK;
}

int sim_reset(sim_t *s, uint64_t basis)
{
    if (!s) return fail(nullptr, SIM_EINVAL, "null handle");
    if (s->n < 64 && (basis >> s->n) != 0) return fail(s, SIM_EINVAL, "basis index out of range");
    s->product = true;
    s->basis = basis;
    s->reset_pending = true;
    return SIM_OK;
}

int sim_sync(sim_t *s)
{
    if (!s) return fail(nullptr, SIM_EINVAL, "null handle");
    if (int rc = materialize(s)) return rc;
    CK(s, cudaStreamSynchronize(s->stream));
    return check_status(s);
}

int sim_state_device(sim_t *s, void **dev_ptr, void **stream)
{
    if (!s) return fail(nullptr, SIM_EINVAL, "null handle");
    if (int rc = materialize(s)) return rc;
    if (dev_ptr) *dev_ptr = s->state;
    if (stream) *stream = (void *)s->stream;
    return SIM_OK;
}

int sim_last_plan_stats(const sim_t *s, sim_plan_stats *out)
{
    if (!s || !out) return fail(nullptr, SIM_EINVAL, "null argument");
    *out = s->stats;
    return SIM_OK;
}

}  // extern "C"

// ------------------------------------------------------------ executor
static size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

struct Blob {
    std::vector<unsigned char> b;
    size_t add(const void *p, size_t n)
    {
        size_t off = align16(b.size());
        b.resize(off + n);
        std::memcpy(b.data() + off, p, n);
        return off;
    }
};

static void add_complex(Blob &bl, const std::vector<cd> &v, bool f64, size_t &off)
{
    if (f64) {
        std::vector<double> d(2 * v.size());
        for (size_t i = 0; i < v.size(); i++) { d[2 * i] = v[i].real(); d[2 * i + 1] = v[i].imag(); }
        off = bl.add(d.data(), d.size() * 8);
    } else {
        std::vector<float> d(2 * v.size());
        for (size_t i = 0; i < v.size(); i++) { d[2 * i] = (float)v[i].real(); d[2 * i + 1] = (float)v[i].imag(); }
        off = bl.add(d.data(), d.size() * 4);
    }
}

static int ensure_sub(sim_t *s, int id, int nq)
{
    if ((int)s->sub.size() <= id) { s->sub.resize(id + 1, nullptr); s->sub_bytes.resize(id + 1, 0); }
    size_t need = ((size_t)1 << nq) * amp_bytes(s->dt);
    if (s->sub_bytes[id] < need) {
        if (s->sub[id]) { CK(s, cudaStreamSynchronize(s->stream)); CK(s, cudaFree(s->sub[id])); s->sub[id] = nullptr; }
        CK(s, dev_malloc((void **)&s->sub[id], need));
        s->sub_bytes[id] = need;
    }
    return SIM_OK;
}

static void *buf_ptr(sim_t *s, int id) { return id == 0 ? s->state : s->sub[id]; }

static int execute(sim_t *s, const Plan &p, bool jit)
{
    const bool f64 = s->dt == SIM_C128;
    if (s->reset_pending) {
        // a booster plan writes the whole state with its final tensor product
        // before anything reads it; otherwise write |basis> first
        bool overwritten = false;
        for (const Op &o : p.ops)
            if (o.buf == 0) { overwritten = o.kind == OPK_TENSOR; break; }
        if (!overwritten) {
            if (int rc = materialize(s)) return rc;
        }
        s->reset_pending = false;
    }
    // 1. plan constants: matrices, diagonal factors and device programs
    Blob bl;
    std::vector<size_t> off(p.ops.size(), 0);
    std::vector<std::vector<int>> nzidx(p.ops.size());
    for (size_t i = 0; i < p.ops.size(); i++) {
        const Op &o = p.ops[i];
        if (o.kind == OPK_DENSE_TC) {
            add_complex(bl, o.gate.M, true, off[i]);   // FP64; the kernels round as their arithmetic needs
        } else if (o.kind == OPK_GATE) {
            add_complex(bl, o.gate.M, f64, off[i]);
        } else if (o.kind == OPK_GATE_DIAG) {
            std::vector<cd> f;
            for (int c = 0; c < (1 << o.gate.k); c++) {
                uint64_t x = 0;
                for (int j = 0; j < o.gate.k; j++) if ((c >> j) & 1) x |= 1ull << o.gate.q[j];
                uint64_t w = 0;
                for (const Term &t : o.gate.terms) if ((x & t.mask) == t.mask) w += t.w;
                if (w != 0) { nzidx[i].push_back(c); f.push_back(phase_of(w)); }
            }
            if (!f.empty()) add_complex(bl, f, f64, off[i]);
        } else if (o.kind == OPK_PHASE_SMALL) {
            std::vector<uint64_t> tw;
            for (const Term &t : o.terms) { tw.push_back(t.mask); tw.push_back(t.w); }
            if (tw.empty()) tw.assign(2, 0);
            off[i] = bl.add(tw.data(), tw.size() * 8);
        } else if (o.kind == OPK_CHUNK || o.kind == OPK_DIAG || o.kind == OPK_DENSE_CHUNK) {
            off[i] = bl.add(o.words.data(), o.words.size() * 4);
        }
    }
    for (size_t b = 1; b < p.buf_qubits.size(); b++) {
        int rc = ensure_sub(s, (int)b, p.buf_qubits[b]);
        if (rc) return rc;
    }
    size_t need = std::max<size_t>(align16(bl.b.size()), 256);
    if (s->pin_pending) { CK(s, cudaEventSynchronize(s->pin_ev)); s->pin_pending = false; }
    if (s->pin_bytes < need) {
        if (s->h_pin) CK(s, cudaFreeHost(s->h_pin));
        s->h_pin = nullptr;
        size_t nb = std::max(need, (size_t)1 << 20);
        CK(s, cudaMallocHost((void **)&s->h_pin, nb));
        s->pin_bytes = nb;
    }
    if (s->const_bytes < need) {
        if (s->d_const) { CK(s, cudaStreamSynchronize(s->stream)); CK(s, cudaFree(s->d_const)); }
        s->d_const = nullptr;
        size_t nb = std::max(need, (size_t)1 << 20);
        CK(s, dev_malloc((void **)&s->d_const, nb));
        s->const_bytes = nb;
    }
    if (!bl.b.empty()) {
        std::memcpy(s->h_pin, bl.b.data(), bl.b.size());
        CK(s, cudaMemcpyAsync(s->d_const, s->h_pin, bl.b.size(), cudaMemcpyHostToDevice, s->stream));
        CK(s, cudaEventRecord(s->pin_ev, s->stream));
        s->pin_pending = true;
    }
    // specialised chunk kernels: compile the programs not cached yet (all of
    // them at once, in parallel) before the first launch
    // (a program whose numbers exceed the kernel-argument space keeps the
    // interpreter kernel: its handle has no kernel)
    std::vector<long> jit_of(p.ops.size(), -1);
    std::vector<JitHandle> jh;
    if (jit) {
        std::vector<JitProg> progs;
        for (size_t i = 0; i < p.ops.size(); i++) {
            const Op &o = p.ops[i];
            if (o.kind == OPK_CHUNK && jit_supported(f64, o.prog.C, o.prog.RB)) {
                jit_of[i] = (long)progs.size();
                const bool fed = i > 0 && p.ops[i - 1].fused;
                progs.push_back({&o.words, fed ? JIT_CHUNK_FED : JIT_CHUNK});
            } else if (o.kind == OPK_DIAG && jit_supported_diag(f64, (int)o.words[prog::H_RB])) {
                jit_of[i] = (long)progs.size();
                progs.push_back({&o.words, JIT_DIAG});
            }
        }
        std::string err;
        if (!progs.empty() && !jit_prepare(progs, jh, err)) return fail(s, SIM_ECUDA, err);
        for (size_t i = 0; i < p.ops.size(); i++)
            if (jit_of[i] >= 0 && !jh[(size_t)jit_of[i]].k) jit_of[i] = -1;
    }
    // 2. launches (Algorithm 5)
    for (size_t i = 0; i < p.ops.size(); i++) {
        const Op &o = p.ops[i];
        if (o.fused) continue;   // a tensor product computed by the next sweep's loads
        void *a = buf_ptr(s, o.buf);
        const unsigned char *cst = s->d_const + off[i];
        TensorSrc src;
        const bool fed = i > 0 && p.ops[i - 1].fused;
        if (fed) {
            const Op &t = p.ops[i - 1];
            src.hi = buf_ptr(s, t.buf_hi);
            src.lo = buf_ptr(s, t.buf_lo);
            src.n_lo = t.n_lo;
        }
        if (fault_launch_fails()) return cuda_fail(s, cudaErrorLaunchOutOfResources, "kernel launch (injected fault)");
        cudaError_t e = cudaSuccess;
        long pe = prof_begin(s, o.buf);
        switch (o.kind) {
        case OPK_INIT_BASIS: e = launch_init_basis(a, o.n, f64, o.basis, s->stream); break;
        case OPK_GATE: e = launch_gate_dense(a, o.n, f64, o.gate.k, o.gate.q, cst, s->stream); break;
        case OPK_DENSE_TC:
            e = launch_dense5(a, o.n, f64, o.precision, o.gate.q, cst, s->d_status, s->stream);
            break;
        case OPK_GATE_DIAG:
            e = launch_gate_diag(a, o.n, f64, o.gate.k, o.gate.q, (int)nzidx[i].size(), nzidx[i].data(), cst,
                                 s->stream);
            break;
        case OPK_DIAG:
            if (jit_of[i] >= 0)
                e = launch_diag_jit(jh[(size_t)jit_of[i]], a, o.n, o.words, (const uint32_t *)cst,
                                    prog::smem_bytes(o.words.data(), true), src, s->stream);
            else
                e = launch_diag_sweep(a, o.n, f64, (const uint32_t *)cst, prog::smem_bytes(o.words.data(), true),
                                      src, s->stream);
            break;
        case OPK_PHASE_SMALL:
            e = launch_phase_small(a, o.n, f64, (const uint64_t *)cst, (int)o.terms.size(), s->stream);
            break;
        case OPK_CHUNK:
            if (jit_of[i] >= 0)
                e = launch_chunk_jit(jh[(size_t)jit_of[i]], a, o.n, o.words, (const uint32_t *)cst,
                                     prog::smem_bytes(o.words.data(), false), src, s->stream);
            else
                e = launch_chunk(a, o.n, f64, o.prog.C, o.prog.RB, (const uint32_t *)cst,
                                 prog::smem_bytes(o.words.data(), false), src, s->stream);
            break;
        case OPK_TENSOR:
            e = launch_tensor(a, buf_ptr(s, o.buf_hi), o.n_hi, buf_ptr(s, o.buf_lo), o.n_lo, f64, s->stream);
            break;
        case OPK_DENSE_CHUNK:
            e = f64 ? cudaErrorInvalidValue
                    : launch_dense_chunk(a, o.n, (const uint32_t *)cst, s->d_status, s->stream);
            break;
        }
        if (e != cudaSuccess) return cuda_fail(s, e, "kernel launch");
        double amps = (double)((uint64_t)1 << o.n), sz = f64 ? 16.0 : 8.0;
        double by = (o.kind == OPK_TENSOR || o.kind == OPK_INIT_BASIS || fed) ? amps * sz : 2.0 * amps * sz;
        prof_end(s, pe, profile_kind(o.kind) + (o.buf ? 8 : 0), by);
    }
    if (s->prof_on) s->prof.h2d_bytes += bl.b.size();
    return SIM_OK;
}

extern "C" {

int sim_apply_circuit(sim_t *s, const sim_gate *gates, size_t n, const sim_options *opt)
{
    if (!s) return fail(nullptr, SIM_EINVAL, "null handle");
    if (n > 0 && !gates) return fail(s, SIM_EINVAL, "null gate array");
    sim_options o;
    if (opt) o = *opt;
    else fill_default_options(o);
    Plan p;
    std::string err;
    uint64_t basis = s->product ? s->basis : UINT64_MAX;
    try {
        if (!make_plan(s->n, s->dt, basis, gates, n, o, p, err)) return fail(s, SIM_EINVAL, err);
    } catch (const std::bad_alloc &) {
        return fail(s, SIM_ENOMEM, "host allocation failed while planning");
    }
    int rc = execute(s, p, (o.flags & SIM_F_JIT) != 0);
    if (rc) return rc;
    s->stats = p.stats;
    if (n > 0) s->product = false;
    return SIM_OK;
}

int sim_norm(sim_t *s, double *out)
{
    if (!s || !out) return fail(s, SIM_EINVAL, "null argument");
    if (int rc = materialize(s)) return rc;
    CK(s, launch_norm(s->state, s->n, s->dt == SIM_C128, s->d_part, s->d_out, s->stream));
    CK(s, cudaMemcpyAsync(out, s->d_out, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    return check_status(s);
}

int sim_expectation(sim_t *s, const uint64_t *masks, size_t nt, double *out)
{
    if (!s || (nt && (!masks || !out))) return fail(s, SIM_EINVAL, "null argument");
    for (size_t i = 0; i < nt; i++)
        if (s->n < 64 && (masks[i] >> s->n)) return fail(s, SIM_EINVAL, "Z mask has bits above n");
    if (int rc = materialize(s)) return rc;
    for (size_t b = 0; b < nt; b += 16) {
        int cnt = (int)std::min<size_t>(16, nt - b);
        CK(s, cudaMemcpyAsync(s->d_masks, masks + b, sizeof(uint64_t) * cnt, cudaMemcpyHostToDevice, s->stream));
        CK(s, launch_expect_z(s->state, s->n, s->dt == SIM_C128, s->d_masks, cnt, s->d_part, s->d_out, s->stream));
        CK(s, cudaMemcpyAsync(out + b, s->d_out, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s->stream));
        CK(s, cudaStreamSynchronize(s->stream));
    }
    return SIM_OK;
}

int sim_probabilities(sim_t *s, double *out)
{
    if (!s || !out) return fail(s, SIM_EINVAL, "null argument");
    if (int rc = materialize(s)) return rc;
    size_t N = (size_t)1 << s->n;
    double *d = nullptr;
    CK(s, cudaMallocAsync((void **)&d, N * sizeof(double), s->stream));
    cudaError_t e = launch_probs(s->state, s->n, s->dt == SIM_C128, d, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, N * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    cudaFreeAsync(d, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "probabilities");
    CK(s, cudaStreamSynchronize(s->stream));
    return check_status(s);
}

static int topk_scratch(sim_t *s)
{
    size_t need = topk_scratch_bytes(1024) + 2 * 1024 * 8;
    if (s->topk_bytes < need) {
        if (s->d_topk) { CK(s, cudaStreamSynchronize(s->stream)); CK(s, cudaFree(s->d_topk)); }
        s->d_topk = nullptr;
        CK(s, dev_malloc((void **)&s->d_topk, need));
        s->topk_bytes = need;
    }
    return SIM_OK;
}

// Top-k of the state into host idx/prob.  `join`: an event recorded on
// another stream (the combined read-out's <Z> sums, nz values at dz) that
// the handle's stream waits for before the first copies, so both run while
// one synchronisation waits for both; the sums are copied to zout.
static int top_k_into(sim_t *s, int k, uint64_t *idx, double *prob, cudaEvent_t join, double *zout,
                      const double *dz, int nz)
{
    int kk = (int)std::min<uint64_t>((uint64_t)k, (uint64_t)1 << s->n);
    unsigned char *base = (unsigned char *)s->d_topk;
    uint64_t *di = (uint64_t *)(base + topk_scratch_bytes(1024));
    double *dp = (double *)(di + 1024);
    // first with warps that keep only their best kTopWarpKeep candidates;
    // again with the exact kernel if a warp slice could have lost one
    const int keep = kk > kTopWarpKeep ? kTopWarpKeep : 0;
    int64_t slice = 0;
    for (int pass = 0; pass < 2; pass++) {
        CK(s, launch_topk(s->state, s->n, s->dt == SIM_C128, kk, base, di, dp, s->stream, pass ? 0 : keep,
                          pass ? nullptr : &slice));
        if (join && pass == 0) {
            CK(s, cudaStreamWaitEvent(s->stream, join, 0));
            CK(s, cudaMemcpyAsync(zout, dz, sizeof(double) * nz, cudaMemcpyDeviceToHost, s->stream));
        }
        CK(s, cudaMemcpyAsync(idx, di, sizeof(uint64_t) * kk, cudaMemcpyDeviceToHost, s->stream));
        CK(s, cudaMemcpyAsync(prob, dp, sizeof(double) * kk, cudaMemcpyDeviceToHost, s->stream));
        CK(s, cudaStreamSynchronize(s->stream));
        if (pass || !topk_warp_suspect(idx, kk, slice, keep)) break;
    }
    for (int i = kk; i < k; i++) { idx[i] = UINT64_MAX; prob[i] = -1.0; }
    return SIM_OK;
}

int sim_top_k(sim_t *s, int k, uint64_t *idx, double *prob)
{
    if (!s || !idx || !prob) return fail(s, SIM_EINVAL, "null argument");
    if (k < 1 || k > 1024) return fail(s, SIM_EINVAL, "k must be in 1..1024");
    if (int rc = materialize(s)) return rc;
    if (int rc = topk_scratch(s)) return rc;
    return top_k_into(s, k, idx, prob, nullptr, nullptr, nullptr, 0);
}

int sim_top_k_expectation(sim_t *s, int k, uint64_t *idx, double *prob, const uint64_t *masks, size_t nt,
                          double *out)
{
    if (!s || !idx || !prob || (nt && (!masks || !out))) return fail(s, SIM_EINVAL, "null argument");
    if (k < 1 || k > 1024) return fail(s, SIM_EINVAL, "k must be in 1..1024");
    for (size_t i = 0; i < nt; i++)
        if (s->n < 64 && (masks[i] >> s->n)) return fail(s, SIM_EINVAL, "Z mask has bits above n");
    if (int rc = materialize(s)) return rc;
    if (int rc = topk_scratch(s)) return rc;
    if (nt == 0) return top_k_into(s, k, idx, prob, nullptr, nullptr, nullptr, 0);
    if (!s->aux) {
        CK(s, cudaStreamCreateWithFlags(&s->aux, cudaStreamNonBlocking));
        CK(s, cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming));
        CK(s, cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming));
    }
    // the first 16 strings' sums on the second stream, beside the top-k
    const int c0 = (int)std::min<size_t>(16, nt);
    CK(s, cudaEventRecord(s->ev_fork, s->stream));
    CK(s, cudaStreamWaitEvent(s->aux, s->ev_fork, 0));
    CK(s, cudaMemcpyAsync(s->d_masks, masks, sizeof(uint64_t) * c0, cudaMemcpyHostToDevice, s->aux));
    CK(s, launch_expect_z(s->state, s->n, s->dt == SIM_C128, s->d_masks, c0, s->d_part, s->d_out, s->aux));
    CK(s, cudaEventRecord(s->ev_join, s->aux));
    if (int rc = top_k_into(s, k, idx, prob, s->ev_join, out, s->d_out, c0)) return rc;
    // further strings, 16 at a time, after
    for (size_t b = 16; b < nt; b += 16) {
        int cnt = (int)std::min<size_t>(16, nt - b);
        CK(s, cudaMemcpyAsync(s->d_masks, masks + b, sizeof(uint64_t) * cnt, cudaMemcpyHostToDevice, s->stream));
        CK(s, launch_expect_z(s->state, s->n, s->dt == SIM_C128, s->d_masks, cnt, s->d_part, s->d_out, s->stream));
        CK(s, cudaMemcpyAsync(out + b, s->d_out, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s->stream));
        CK(s, cudaStreamSynchronize(s->stream));
    }
    return SIM_OK;
}

int sim_get_state(sim_t *s, void *host, size_t bytes)
{
    if (!s || !host) return fail(s, SIM_EINVAL, "null argument");
    if (bytes != s->state_bytes) return fail(s, SIM_EINVAL, "byte count must equal 2^n * bytes per amplitude");
    if (int rc = materialize(s)) return rc;
    CK(s, cudaMemcpyAsync(host, s->state, bytes, cudaMemcpyDeviceToHost, s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    return check_status(s);
}

int sim_set_state(sim_t *s, const void *host, size_t bytes)
{
    if (!s || !host) return fail(s, SIM_EINVAL, "null argument");
    if (bytes != s->state_bytes) return fail(s, SIM_EINVAL, "byte count must equal 2^n * bytes per amplitude");
    s->reset_pending = false;
    CK(s, cudaMemcpyAsync(s->state, host, bytes, cudaMemcpyHostToDevice, s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    s->product = false;
    return SIM_OK;
}

int sim_profile_enable(sim_t *s, int on)
{
    if (!s) return fail(nullptr, SIM_EINVAL, "null handle");
    CK(s, cudaStreamSynchronize(s->stream));
    s->prof_pend.clear();
    s->ev_used = 0;
    if (on) s->prof = sim_profile{};
    s->prof_on = on != 0;
    s->prof_all = on != 2;
    return SIM_OK;
}

int sim_profile_read(sim_t *s, sim_profile *out)
{
    if (!s || !out) return fail(s, SIM_EINVAL, "null argument");
    CK(s, cudaStreamSynchronize(s->stream));
    for (const sim_t::Pend &p : s->prof_pend) {
        float ms = 0;
        CK(s, cudaEventElapsedTime(&ms, s->ev_pool[p.e0], s->ev_pool[p.e0 + 1]));
        s->prof.launches[p.kind & 15]++;
        s->prof.ms[p.kind & 15] += ms;
        s->prof.bytes[p.kind & 15] += p.bytes;
    }
    s->prof_pend.clear();
    s->ev_used = 0;
    *out = s->prof;
    return SIM_OK;
}

int sim_plan_json(int n, sim_dtype dt, uint64_t basis, const sim_gate *gates, size_t ng, const sim_options *opt,
                  char *buf, size_t buflen, size_t *needed)
{
    int rc = check_n(n, dt);
    if (rc) return rc;
    if (ng > 0 && !gates) return fail(nullptr, SIM_EINVAL, "null gate array");
    sim_options o;
    if (opt) o = *opt;
    else fill_default_options(o);
    Plan p;
    std::string err;
    try {
        if (!make_plan(n, dt, basis, gates, ng, o, p, err)) return fail(nullptr, SIM_EINVAL, err);
    } catch (const std::bad_alloc &) {
        return fail(nullptr, SIM_ENOMEM, "host allocation failed while planning");
    }
    std::string js = plan_json(p);
    if (needed) *needed = js.size() + 1;
    if (!buf || buflen < js.size() + 1) return fail(nullptr, SIM_ENOMEM, "buffer too small for the plan");
    std::memcpy(buf, js.c_str(), js.size() + 1);
    return SIM_OK;
}

int sim_jit_info(uint64_t *programs, double *compile_ms)
{
    const size_t n = jit_cache_size(compile_ms, nullptr);
    if (programs) *programs = n;
    return SIM_OK;
}

int sim_jit_cache(int max_kernels, uint64_t *kernels, uint64_t *compiles)
{
    if (max_kernels < 0) return fail(nullptr, SIM_EINVAL, "max_kernels must be >= 0");
    if (max_kernels > 0) jit_set_cache_limit((size_t)max_kernels);
    const size_t k = jit_cache_size(nullptr, compiles);
    if (kernels) *kernels = k;
    return SIM_OK;
}

// the specialised sweeps of a plan: generate (and optionally compile) each
static int jit_plan_sources(int n, sim_dtype dt, uint64_t basis, const sim_gate *gates, size_t ng,
                            const sim_options *opt, bool compile, int *n_programs, std::string *text)
{
    int rc = check_n(n, dt);
    if (rc) return rc;
    if (ng > 0 && !gates) return fail(nullptr, SIM_EINVAL, "null gate array");
    sim_options o;
    if (opt) o = *opt;
    else fill_default_options(o);
    Plan p;
    std::string err;
    try {
        if (!make_plan(n, dt, basis, gates, ng, o, p, err)) return fail(nullptr, SIM_EINVAL, err);
        int np = 0;
        for (size_t i = 0; i < p.ops.size(); i++) {
            const Op &op = p.ops[i];
            int kind = -1;
            if (op.kind == OPK_CHUNK && jit_supported(dt == SIM_C128, op.prog.C, op.prog.RB))
                kind = i > 0 && p.ops[i - 1].fused ? JIT_CHUNK_FED : JIT_CHUNK;
            if (op.kind == OPK_DIAG && jit_supported_diag(dt == SIM_C128, (int)op.words[prog::H_RB])) kind = JIT_DIAG;
            if (kind < 0) continue;
            std::string src;
            std::vector<uint32_t> vals;
            std::vector<char> cubin;
            if (!jit_source(op.words, kind, src, vals, err)) return fail(nullptr, SIM_EINVAL, err);
            if (compile && (!jit_compile(src, cubin, err) || cubin.empty()))
                return fail(nullptr, SIM_EINVAL, err.empty() ? "empty cubin" : err);
            if (text) {
                *text += "// ---- specialised sweep " + std::to_string(np) + ": " + std::to_string(vals.size()) +
                         " parameter words\n" + src;
            }
            np++;
        }
        if (n_programs) *n_programs = np;
    } catch (const std::bad_alloc &) {
        return fail(nullptr, SIM_ENOMEM, "host allocation failed while planning");
    }
    return SIM_OK;
}

int sim_jit_sources(int n, sim_dtype dt, uint64_t basis, const sim_gate *gates, size_t ng, const sim_options *opt,
                    char *buf, size_t buflen, size_t *needed)
{
    std::string text;
    int rc = jit_plan_sources(n, dt, basis, gates, ng, opt, false, nullptr, &text);
    if (rc) return rc;
    if (needed) *needed = text.size() + 1;
    if (!buf || buflen < text.size() + 1) return fail(nullptr, SIM_ENOMEM, "buffer too small for the sources");
    std::memcpy(buf, text.c_str(), text.size() + 1);
    return SIM_OK;
}

int sim_jit_check(int n, sim_dtype dt, uint64_t basis, const sim_gate *gates, size_t ng, const sim_options *opt,
                  int *n_programs)
{
    return jit_plan_sources(n, dt, basis, gates, ng, opt, true, n_programs, nullptr);
}

}  // extern "C"
