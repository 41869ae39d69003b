// serve.cpp -- the serving loop (srv_* in include/svsim.h): continuous
// batching of circuit requests on one GPU.
//
//   submit  -> copy the request, validate its shape, queue it
//   batcher -> takes every queued small request (state fits one CTA's shared
//              memory), packs them into one k_batch launch on its own stream
//   workers -> n_streams threads, one stream + one reusable state buffer and
//              sim_t handle each; take the first queued large request whose
//              state footprint fits the remaining HBM budget, run the full
//              pipeline (optimizer + kernels + read-out) on it
// Requests that arrive while others run are admitted as soon as a slot and
// budget free up; batches and worker streams overlap on the device.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "batch.h"
#include "internal.h"
#include "kernels.h"

using namespace svs;
using Clock = std::chrono::steady_clock;

namespace {

struct Req {
    uint64_t ticket = 0;
    int n = 0;
    sim_dtype dt = SIM_C64;
    std::vector<sim_gate> gates;
    std::vector<double> mats;        // owned copies of the gates' matrices
    uint64_t basis = 0;
    int top_k = 0;
    std::vector<uint64_t> masks;
    size_t bytes = 0;                // state footprint
    bool small = false;
    Clock::time_point t_submit, t_start, t_done;
    bool done = false;
    srv_result res;
};

double ms_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct srv_t {
    size_t budget = 0;
    size_t in_use = 0;
    size_t peak = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> small_q, large_q;
    std::unordered_map<uint64_t, Req *> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<std::thread> threads;
    // stats
    uint64_t submitted = 0, completed = 0, failed = 0, batched = 0, batches = 0;
    std::vector<double> lat;
    bool any = false;
    Clock::time_point t_first, t_last;
};

namespace {

void finish(srv_t *s, Req *r, int status)
{
    r->t_done = Clock::now();
    r->res.status = status;
    r->res.latency_ms = ms_between(r->t_submit, r->t_done);
    r->res.queue_ms = ms_between(r->t_submit, r->t_start);
    std::lock_guard<std::mutex> lk(s->mu);
    r->done = true;
    s->completed++;
    if (status != SIM_OK) s->failed++;
    s->lat.push_back(r->res.latency_ms);
    s->t_last = r->t_done;
    s->cv_done.notify_all();
}

// ---- batch path: many small circuits, one launch, one CTA each
void batcher_loop(srv_t *s)
{
    cudaSetDevice(s->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    uint32_t *d_blob = nullptr, *h_blob = nullptr;
    size_t blob_cap = 0;
    BatchReq *d_reqs = nullptr, *h_reqs = nullptr;
    size_t req_cap = 0;
    double *d_out = nullptr, *h_out = nullptr;
    size_t out_cap = 0;
    const int max_batch = 4 * std::max(1, device_sm_count());
    while (true) {
        std::vector<Req *> take;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->small_q.empty(); });
            if (s->small_q.empty() && s->stop) break;
            // one launch per dtype: take the leading requests of the first one's dtype
            const sim_dtype dt = s->small_q.front()->dt;
            for (auto it = s->small_q.begin(); it != s->small_q.end() && (int)take.size() < max_batch;) {
                if ((*it)->dt == dt) { take.push_back(*it); it = s->small_q.erase(it); }
                else ++it;
            }
        }
        const bool f64 = take[0]->dt == SIM_C128;
        std::vector<uint32_t> blob;
        std::vector<BatchReq> brs;
        std::vector<Req *> run;
        size_t outs = 0;
        int max_n = 1;
        for (Req *r : take) {
            r->t_start = Clock::now();
            BatchReq b{};
            std::vector<uint32_t> w;
            int nops = 0;
            std::string err;
            bool wide = false;
            if (!make_batch_ops(r->n, r->dt, r->gates.data(), r->gates.size(), w, nops, err, wide)) {
                if (wide) {   // not a batch circuit after all: full pipeline
                    std::lock_guard<std::mutex> lk(s->mu);
                    r->small = false;
                    s->large_q.push_back(r);
                    s->cv_work.notify_all();
                } else {
                    finish(s, r, SIM_EINVAL);
                }
                continue;
            }
            if (blob.size() & 1) blob.push_back(0);
            b.n = r->n;
            b.nops = nops;
            b.ops_off = (uint32_t)blob.size();
            blob.insert(blob.end(), w.begin(), w.end());
            if (blob.size() & 1) blob.push_back(0);
            b.masks_off = (uint32_t)blob.size();
            for (uint64_t m : r->masks) { blob.push_back((uint32_t)m); blob.push_back((uint32_t)(m >> 32)); }
            b.nmask = (int)r->masks.size();
            b.top_k = r->top_k;
            b.basis = r->basis;
            b.out_off = outs;
            outs += r->masks.size() + 2 * (size_t)r->top_k;
            max_n = std::max(max_n, r->n);
            brs.push_back(b);
            run.push_back(r);
        }
        if (run.empty()) continue;
        auto grow = [](size_t need, size_t &cap, auto *&dptr, auto *&hptr) {
            if (need <= cap) return cudaSuccess;
            if (dptr) cudaFree(dptr);
            if (hptr) cudaFreeHost(hptr);
            size_t nc = std::max(need, cap * 2);
            cudaError_t e = dev_malloc((void **)&dptr, nc * sizeof(*dptr));
            if (e == cudaSuccess) e = cudaMallocHost((void **)&hptr, nc * sizeof(*hptr));
            cap = e == cudaSuccess ? nc : 0;
            return e;
        };
        cudaError_t e = grow(blob.size() + 2, blob_cap, d_blob, h_blob);
        if (e == cudaSuccess) e = grow(brs.size(), req_cap, d_reqs, h_reqs);
        if (e == cudaSuccess) e = grow(outs + 1, out_cap, d_out, h_out);
        if (e == cudaSuccess) {
            std::memcpy(h_blob, blob.data(), blob.size() * 4);
            std::memcpy(h_reqs, brs.data(), brs.size() * sizeof(BatchReq));
            e = cudaMemcpyAsync(d_blob, h_blob, blob.size() * 4, cudaMemcpyHostToDevice, st);
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_reqs, h_reqs, brs.size() * sizeof(BatchReq), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = launch_batch(d_reqs, (int)brs.size(), max_n, d_blob, d_out, f64, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_out, d_out, outs * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->batches++;
            s->batched += run.size();
        }
        for (size_t i = 0; i < run.size(); i++) {
            Req *r = run[i];
            if (e != cudaSuccess) { finish(s, r, SIM_ECUDA); continue; }
            const double *o = h_out + brs[i].out_off;
            r->res.path = 0;
            r->res.n_masks = (int)r->masks.size();
            r->res.top_k = r->top_k;
            for (size_t m = 0; m < r->masks.size(); m++) r->res.expect[m] = o[m];
            for (int k = 0; k < r->top_k; k++) {
                r->res.top_p[k] = o[r->masks.size() + k];
                const double ix = o[r->masks.size() + r->top_k + k];
                r->res.top_idx[k] = ix < 0 ? UINT64_MAX : (uint64_t)ix;
            }
            finish(s, r, SIM_OK);
        }
    }
    if (d_blob) cudaFree(d_blob);
    if (h_blob) cudaFreeHost(h_blob);
    if (d_reqs) cudaFree(d_reqs);
    if (h_reqs) cudaFreeHost(h_reqs);
    if (d_out) cudaFree(d_out);
    if (h_out) cudaFreeHost(h_out);
    cudaStreamDestroy(st);
}

// ---- full-state path: optimizer + kernels on a worker stream
// Admission charges what the device really holds: in_use is the sum of the
// state buffers the workers keep (each worker keeps its largest buffer for
// the next request).  A worker may take a queued request that fits its own
// buffer, or whose footprint fits the budget once its own buffer is given
// back.  A worker with nothing it may take while requests wait releases its
// buffer, so that another worker can take them.
void worker_loop(srv_t *s)
{
    cudaSetDevice(s->device);
    cudaStream_t st = nullptr;
    const bool stream_ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
    void *buf = nullptr;
    size_t cap = 0;
    sim_t *h = nullptr;
    auto release = [&] {
        if (h) { sim_destroy(h); h = nullptr; }
        if (buf) cudaFree(buf);
        buf = nullptr;
        std::lock_guard<std::mutex> lk(s->mu);
        s->in_use -= cap;
        cap = 0;
    };
    while (true) {
        Req *r = nullptr;
        bool give_back = false;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            auto fits = [&](const Req *q) { return q->bytes <= cap || s->in_use - cap + q->bytes <= s->budget; };
            s->cv_work.wait(lk, [&] {
                if (s->stop && s->large_q.empty()) return true;
                for (Req *q : s->large_q)
                    if (fits(q)) return true;
                return cap > 0 && !s->large_q.empty();
            });
            if (s->large_q.empty()) break;
            // admission by footprint: the first queued request that fits
            for (auto it = s->large_q.begin(); it != s->large_q.end(); ++it)
                if (fits(*it)) {
                    r = *it;
                    s->large_q.erase(it);
                    break;
                }
            if (!r) {
                give_back = true;
            } else if (r->bytes > cap) {
                // the buffer grows: charged now, before it is allocated
                s->in_use += r->bytes - cap;
                s->peak = std::max(s->peak, s->in_use);
            }
        }
        if (give_back) {
            release();
            s->cv_work.notify_all();
            continue;
        }
        r->t_start = Clock::now();
        int rc = stream_ok ? SIM_OK : SIM_ECUDA;
        if (rc == SIM_OK && cap < r->bytes) {
            const size_t want = r->bytes;
            if (h) { sim_destroy(h); h = nullptr; }
            if (buf) cudaFree(buf);
            buf = nullptr;
            if (dev_malloc(&buf, want) != cudaSuccess) {
                buf = nullptr;
                rc = SIM_ENOMEM;
                std::lock_guard<std::mutex> lk(s->mu);
                s->in_use -= want;   // charged above, not held
                cap = 0;
            } else {
                cap = want;
            }
        }
        if (rc == SIM_OK && !h) rc = sim_create_on(r->n, r->dt, buf, cap, (void *)st, &h);
        if (rc == SIM_OK) rc = svs_rebind(h, r->n, r->dt, buf, cap);
        if (rc == SIM_OK) rc = sim_reset(h, r->basis);
        if (rc == SIM_OK) rc = sim_apply_circuit(h, r->gates.data(), r->gates.size(), nullptr);
        if (rc == SIM_OK && r->top_k > 0)
            rc = sim_top_k_expectation(h, r->top_k, r->res.top_idx, r->res.top_p, r->masks.data(), r->masks.size(),
                                       r->res.expect);
        else if (rc == SIM_OK && !r->masks.empty())
            rc = sim_expectation(h, r->masks.data(), r->masks.size(), r->res.expect);
        if (rc == SIM_OK) rc = sim_sync(h);
        r->res.path = 1;
        r->res.n_masks = (int)r->masks.size();
        r->res.top_k = r->top_k;
        s->cv_work.notify_all();
        finish(s, r, rc);
    }
    release();
    if (st) cudaStreamDestroy(st);
}

int sfail(int code) { return code; }

}  // namespace

extern "C" {

int srv_create(size_t budget, int n_streams, srv_t **out)
{
    if (!out || n_streams < 1 || n_streams > 64 || budget == 0) return sfail(SIM_EINVAL);
    srv_t *s = new (std::nothrow) srv_t();
    if (!s) return sfail(SIM_ENOMEM);
    if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return sfail(SIM_ECUDA); }
    s->budget = budget;
    try {
        s->threads.emplace_back(batcher_loop, s);
        for (int i = 0; i < n_streams; i++) s->threads.emplace_back(worker_loop, s);
    } catch (...) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        for (auto &t : s->threads) if (t.joinable()) t.join();
        delete s;
        return sfail(SIM_ENOMEM);
    }
    *out = s;
    return SIM_OK;
}

int srv_submit(srv_t *s, const srv_request *q, uint64_t *ticket)
{
    if (!s || !q || !ticket) return sfail(SIM_EINVAL);
    const int nmax = q->dtype == SIM_C64 ? kMaxQubitsC64 : kMaxQubitsC128;
    if ((q->dtype != SIM_C64 && q->dtype != SIM_C128) || q->n_qubits < 1 || q->n_qubits > nmax) return sfail(SIM_EINVAL);
    if (q->top_k < 0 || q->top_k > 1024 || q->n_masks > 64) return sfail(SIM_EINVAL);
    if ((q->n_gates && !q->gates) || (q->n_masks && !q->z_masks)) return sfail(SIM_EINVAL);
    if (q->n_qubits < 64 && (q->basis >> q->n_qubits)) return sfail(SIM_EINVAL);
    for (size_t i = 0; i < q->n_masks; i++)
        if (q->z_masks[i] >> q->n_qubits) return sfail(SIM_EINVAL);
    Req *r = new (std::nothrow) Req();
    if (!r) return sfail(SIM_ENOMEM);
    r->n = q->n_qubits;
    r->dt = q->dtype;
    r->basis = q->basis;
    r->top_k = q->top_k;
    r->masks.assign(q->z_masks, q->z_masks + q->n_masks);
    r->bytes = ((size_t)1 << r->n) * (r->dt == SIM_C64 ? 8 : 16);
    if (r->bytes > s->budget) { delete r; return sfail(SIM_ENOMEM); }
    // copy gates and their matrices (the caller's arrays are borrowed)
    r->gates.assign(q->gates, q->gates + q->n_gates);
    size_t md = 0;
    for (const sim_gate &g : r->gates) {
        if (!g.matrix) continue;
        const int k = g.kind == G_U1Q ? 1 : (int)g.nq;
        if (k < 1 || k > kMaxGateQubits) { delete r; return sfail(SIM_EINVAL); }
        md += g.kind == G_DIAG ? 2 * ((size_t)1 << k) : 2 * ((size_t)1 << (2 * k));
    }
    r->mats.resize(md);
    size_t o = 0;
    for (sim_gate &g : r->gates) {
        if (!g.matrix) continue;
        const int k = g.kind == G_U1Q ? 1 : (int)g.nq;
        const size_t len = g.kind == G_DIAG ? 2 * ((size_t)1 << k) : 2 * ((size_t)1 << (2 * k));
        std::memcpy(&r->mats[o], g.matrix, len * sizeof(double));
        g.matrix = &r->mats[o];
        o += len;
    }
    const int small_n = r->dt == SIM_C64 ? kBatchMaxN64 : kBatchMaxN128;
    r->small = r->n <= small_n && r->top_k <= kBatchMaxTopK;
    std::memset(&r->res, 0, sizeof(r->res));
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) { delete r; return sfail(SIM_EBUSY); }
        r->ticket = s->next_ticket++;
        s->reqs[r->ticket] = r;
        s->submitted++;
        if (!s->any) { s->any = true; s->t_first = r->t_submit; }
        (r->small ? s->small_q : s->large_q).push_back(r);
    }
    s->cv_work.notify_all();
    *ticket = r->ticket;
    return SIM_OK;
}

int srv_poll(srv_t *s, uint64_t ticket, srv_result *out, int timeout_ms)
{
    if (!s || !out) return sfail(SIM_EINVAL);
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return sfail(SIM_EINVAL);
    Req *r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_ms < 0) s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return SIM_ETIMEOUT;
    std::memcpy(out, &r->res, sizeof(srv_result));
    s->reqs.erase(it);
    delete r;
    return SIM_OK;
}

int srv_get_stats(srv_t *s, srv_stats *out)
{
    if (!s || !out) return sfail(SIM_EINVAL);
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->batched = s->batched;
    out->batches = s->batches;
    out->hbm_budget = s->budget;
    out->hbm_peak = s->peak;
    if (!s->lat.empty()) {
        std::vector<double> v = s->lat;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) { return v[std::min(v.size() - 1, (size_t)(q * (v.size() - 1) + 0.5))]; };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        out->max_ms = v.back();
        double sum = 0;
        for (double x : v) sum += x;
        out->mean_ms = sum / v.size();
        out->elapsed_s = std::chrono::duration<double>(s->t_last - s->t_first).count();
        out->circuits_per_s = out->elapsed_s > 0 ? s->completed / out->elapsed_s : 0;
    }
    return SIM_OK;
}

int srv_destroy(srv_t *s)
{
    if (!s) return sfail(SIM_EINVAL);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->threads) if (t.joinable()) t.join();
    for (auto &kv : s->reqs) delete kv.second;
    delete s;
    return SIM_OK;
}

}  // extern "C"
