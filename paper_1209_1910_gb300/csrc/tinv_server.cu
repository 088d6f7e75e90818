// tinv_server.cu -- request-queue API with continuous batching (tinv_server_* in tinv.h).
//
// Callers submit eigenvector problems of any order at any time.  A worker thread owns the GPU.
// Whenever one of its streams is free and enough SMs are free, it forms a wave from the pending
// requests: in arrival order, skipping requests that do not fit the slot limit or the memory
// budget right now (so small requests pass a large one that waits for memory; a request passed
// over too often stops the others from passing it), until the wave holds its share of the
// pending work.  The memory budget is re-read at every admission (hbm_fraction of the device
// memory free now plus what the server's own waves hold).  The wave is enqueued on its stream:
// host-to-device copy of the packed inputs, Sturm bisection for requests that came without
// eigenvalues, the batched inverse-iteration path (tinv_batch's device form, one problem table
// for the wave) with a persistent grid sized from the free SMs, and the copy of the
// eigenvectors back to pinned staging.  Up to max_inflight waves run at once, so requests that
// arrive while waves are on the GPU start as soon as a stream and SMs free up, and the waves'
// kernels and copies overlap on the device.  A completed wave's vectors are copied into the
// callers' buffers and their requests complete.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/tinv.h"
#include "tinv_internal.h"

using namespace tinvx;
using Clock = std::chrono::steady_clock;

namespace {

struct Req {
    uint64_t ticket = 0;
    int64_t n = 0;
    std::vector<double> d, e, w;  // copies taken at submit
    bool has_w = false;
    double* Z = nullptr;          // caller's host buffer, n x n
    uint64_t seed = 0;
    int32_t state = TINV_REQ_PENDING;
    bool cancel = false;          // cancelled while running: the result is dropped
    bool delivering = false;      // the result is being copied to Z: too late to cancel
    int skipped = 0;              // admissions that passed over this request
    int64_t info = 0;
    int rc = 0;
    size_t bytes = 0;             // device bytes the request adds to a wave
    Clock::time_point t_submit, t_done;
};
using ReqP = std::shared_ptr<Req>;

// Pinned staging of one stream (reused by the waves of that stream, grown on demand).
struct Staging {
    double* in = nullptr;
    size_t cap_in = 0;  // doubles
    double* z = nullptr;
    size_t cap_z = 0;
    int64_t* tab = nullptr;  // ns | off_de | info (3 x cap_tab)
    size_t cap_tab = 0;
};

struct Wave {
    std::vector<ReqP> reqs;
    int slot = 0;
    int ctas = 0;       // persistent CTAs (SMs) of the wave's cluster kernel
    size_t bytes = 0;
    int rc = 0;
    std::atomic<bool> finished{false};
    struct tinv_server* srv = nullptr;
};

bool grow_pinned(void** p, size_t* cap, size_t need, size_t elem)
{
    if (*cap >= need) return true;
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    *cap = 0;
    size_t want = need + need / 4 + 1024;
    if (cudaMallocHost(p, want * elem) != cudaSuccess) {
        *p = nullptr;
        return false;
    }
    *cap = want;
    return true;
}

// Device bytes one request adds to a wave: LU factors and pivots (33 n^2), Y and the T bound
// (16 n^2), the eigenvectors (8 n^2) and O(n) vectors.
size_t request_bytes(int64_t n)
{
    const double nn = (double)n;
    return (size_t)(57.0 * nn * nn + 256.0 * nn + 4096.0);
}

// Work estimate of a request for dividing the pending requests among waves and SMs: the
// reorthogonalization grows as (cluster size)^2 n, at most n^3.
double request_work(int64_t n)
{
    const double nn = (double)n;
    return nn * nn * nn + 1.0e6;
}

// Admissions that may pass over a pending request before it blocks the requests behind it.
constexpr int kMaxSkips = 8;

}  // namespace

struct tinv_server {
    tinv_server_cfg cfg;
    int device = 0;
    int sms = 1;
    size_t budget = 0;
    std::mutex mu;
    std::condition_variable cv_work;  // worker: new requests, finished waves, stop
    std::condition_variable cv_done;  // callers: request state changes
    std::deque<ReqP> pending;
    std::unordered_map<uint64_t, ReqP> table;
    std::vector<cudaStream_t> streams;
    std::vector<Staging> staging;
    std::vector<Wave*> inflight;
    std::vector<bool> slot_busy;
    size_t inflight_bytes = 0;
    int sms_used = 0;  // persistent CTAs of the waves in flight
    int64_t inflight_problems = 0;
    uint64_t next_ticket = 1;
    bool stopping = false;
    std::thread worker;
    // statistics
    uint64_t submitted = 0, completed = 0, cancelled = 0, failed = 0, rejected = 0, waves = 0;
    uint64_t max_inflight_seen = 0, wave_problems = 0;
    double eigvecs_done = 0.0;
    std::vector<double> lat_ms;
    bool any_submit = false;
    Clock::time_point t_first, t_last;

    void run();
    Wave* launch(std::vector<ReqP>&& reqs, int slot, int ctas);
    bool admit();
    void finish(Wave* w);
};

namespace {

void CUDART_CB wave_done_cb(void* arg)
{
    Wave* w = (Wave*)arg;
    w->finished.store(true);
    // notify under the lock so the worker cannot miss it between its check and its wait
    std::lock_guard<std::mutex> lk(w->srv->mu);
    w->srv->cv_work.notify_all();
}

}  // namespace

// Enqueue one wave on streams[slot].  Returns the wave (rc != 0 if enqueueing failed).
Wave* tinv_server::launch(std::vector<ReqP>&& reqs, int slot, int ctas)
{
    Wave* wv = new Wave;
    wv->reqs = std::move(reqs);
    wv->slot = slot;
    wv->ctas = ctas;
    wv->srv = this;
    cudaStream_t st = streams[slot];
    Staging& sg = staging[slot];
    const int64_t np = (int64_t)wv->reqs.size();
    std::vector<int64_t> ns(np), off_de(np), off_z(np);
    std::vector<uint64_t> seeds(np);
    int64_t M = 0, ZZ = 0, nmax = 1, nbis = 0;
    for (int64_t q = 0; q < np; ++q) {
        const Req& r = *wv->reqs[q];
        ns[q] = r.n;
        off_de[q] = M;
        off_z[q] = ZZ;
        seeds[q] = r.seed;
        M += r.n;
        ZZ += r.n * r.n;
        nmax = std::max(nmax, r.n);
        if (!r.has_w) ++nbis;
        wv->bytes += r.bytes;
    }
    int rc = 0;
    if (!grow_pinned((void**)&sg.in, &sg.cap_in, (size_t)(3 * M), sizeof(double)) ||
        !grow_pinned((void**)&sg.z, &sg.cap_z, (size_t)ZZ, sizeof(double)) ||
        !grow_pinned((void**)&sg.tab, &sg.cap_tab, (size_t)(3 * np), sizeof(int64_t)))
        rc = TINV_ENOMEM;
    double *dev = nullptr, *dz = nullptr;
    int64_t* dtab = nullptr;
    if (!rc) {
        double* hd = sg.in;
        double* he = sg.in + M;
        double* hw = sg.in + 2 * M;
        int64_t* tn = sg.tab;
        int64_t* toff = sg.tab + np;
        int64_t nb = 0;
        for (int64_t q = 0; q < np; ++q) {
            const Req& r = *wv->reqs[q];
            memcpy(hd + off_de[q], r.d.data(), (size_t)r.n * sizeof(double));
            if (r.n > 1) memcpy(he + off_de[q], r.e.data(), (size_t)(r.n - 1) * sizeof(double));
            he[off_de[q] + r.n - 1] = 0.0;
            if (r.has_w) {
                memcpy(hw + off_de[q], r.w.data(), (size_t)r.n * sizeof(double));
            } else {
                tn[nb] = r.n;
                toff[nb] = off_de[q];
                ++nb;
            }
        }
        cudaError_t ce = cudaMallocAsync((void**)&dev, (size_t)(3 * M) * sizeof(double), st);
        if (ce == cudaSuccess) ce = cudaMallocAsync((void**)&dz, (size_t)std::max<int64_t>(ZZ, 1) * sizeof(double), st);
        if (ce == cudaSuccess) ce = cudaMallocAsync((void**)&dtab, (size_t)(3 * np) * sizeof(int64_t), st);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(dev, sg.in, (size_t)(3 * M) * sizeof(double), cudaMemcpyHostToDevice, st);
        if (ce == cudaSuccess && nb > 0) {
            // bisection table: orders at dtab[0..nb), offsets at dtab[np..np+nb)
            ce = cudaMemcpyAsync(dtab, tn, (size_t)nb * sizeof(int64_t), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(dtab + np, toff, (size_t)nb * sizeof(int64_t), cudaMemcpyHostToDevice, st);
            int64_t nbmax = 1;
            for (int64_t i = 0; i < nb; ++i) nbmax = std::max(nbmax, tn[i]);
            if (ce == cudaSuccess)
                ce = launch_bisect(nb, dtab, dtab + np, 0, nbmax, dev, dev + M, dev + 2 * M, st);
        }
        rc = cuda_code(ce);
    }
    if (!rc) {
        tinv_opts o;
        tinv_opts_default(&o);
        o.method = cfg.method;
        o.device_ptrs = 1;
        o.stream = st;
        o.max_team = cfg.max_team;
        o.block = cfg.block;
        // each wave's persistent kernel holds one CTA on each of its SMs (a CTA fills an SM's
        // registers), and the worker keeps the grids of the waves in flight within the SM count,
        // so every wave's CTAs are co-resident
        o.grid_ctas = wv->ctas;
        rc = batch_enqueue_device(np, ns.data(), off_de.data(), off_z.data(), seeds.data(), dev,
                                  dev + M, dev + 2 * M, dz, dtab + 2 * np, o);
    }
    if (!rc) {
        cudaError_t ce = cudaMemcpyAsync(sg.z, dz, (size_t)ZZ * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(sg.tab + 2 * np, dtab + 2 * np, (size_t)np * sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, st);
        rc = cuda_code(ce);
    }
    if (dev) cudaFreeAsync(dev, st);
    if (dz) cudaFreeAsync(dz, st);
    if (dtab) cudaFreeAsync(dtab, st);
    if (!rc) rc = cuda_code(cudaLaunchHostFunc(st, wave_done_cb, wv));
    wv->rc = rc;
    if (rc) {
        cudaStreamSynchronize(st);  // nothing of this wave may still run
        wv->finished.store(true);
    }
    return wv;
}

// Copy a finished wave's vectors to the callers' buffers (no lock held).
void tinv_server::finish(Wave* wv)
{
    cudaStream_t st = streams[wv->slot];
    int rc = wv->rc;
    if (!rc) rc = cuda_code(cudaStreamSynchronize(st));
    const Staging& sg = staging[wv->slot];
    const int64_t np = (int64_t)wv->reqs.size();
    int64_t zoff = 0;
    for (int64_t q = 0; q < np; ++q) {
        Req& r = *wv->reqs[q];
        if (!rc) {
            r.info = sg.tab[2 * np + q];
            bool deliver;
            {
                // decided under the lock: from here on tinv_cancel reports the request as
                // completed, so a caller never sees a successful cancel while Z is written
                std::lock_guard<std::mutex> lk(mu);
                deliver = !r.cancel && r.info >= 0;
                r.delivering = deliver;
            }
            if (deliver) memcpy(r.Z, sg.z + zoff, (size_t)(r.n * r.n) * sizeof(double));
        }
        zoff += r.n * r.n;
    }
    const Clock::time_point now = Clock::now();
    std::lock_guard<std::mutex> lk(mu);
    for (auto& rp : wv->reqs) {
        Req& r = *rp;
        r.t_done = now;
        if (r.cancel) {
            r.state = TINV_REQ_CANCELLED;
            ++cancelled;
        } else if (rc || r.info < 0) {
            r.state = TINV_REQ_FAILED;
            r.rc = rc ? rc : (int)r.info;
            ++failed;
        } else {
            r.state = TINV_REQ_DONE;
            ++completed;
            eigvecs_done += (double)r.n;
            lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r.t_submit).count());
            t_last = now;
        }
    }
    inflight_bytes -= wv->bytes;
    inflight_problems -= np;
    sms_used -= wv->ctas;
    slot_busy[wv->slot] = false;
    cv_done.notify_all();
}

// Form and enqueue one wave if a stream and enough SMs are free and some pending request fits.
// Called by the worker with `mu` held; releases it while the wave is enqueued.  Returns true when
// a wave was launched.
bool tinv_server::admit()
{
    if (pending.empty()) return false;
    int slot = -1, free_streams = 0;
    for (int s = 0; s < (int)streams.size(); ++s)
        if (!slot_busy[s]) {
            if (slot < 0) slot = s;
            ++free_streams;
        }
    if (slot < 0) return false;
    const int share = cfg.wave_ctas > 0 ? std::min(cfg.wave_ctas, sms)
                                        : std::max(1, sms / (int)streams.size());
    const int free_sms = sms - sms_used;
    if (free_sms < share && !inflight.empty()) return false;
    // memory budget now: hbm_fraction of the free device memory (with what the library's pool
    // keeps unused from earlier waves) plus what the waves hold
    size_t budget_now = budget;
    {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
            budget_now = (size_t)(cfg.hbm_fraction * (double)(free_b + lib_pool_idle() + inflight_bytes));
    }
    double pend_work = 0.0;
    for (const ReqP& r : pending) pend_work += request_work(r->n);
    // this wave's share of the pending work: the free streams divide it
    const double target = pend_work / (double)free_streams;
    std::vector<ReqP> take, passed;
    size_t bytes = 0;
    double work = 0.0;
    for (auto it = pending.begin(); it != pending.end() && work < target;) {
        ReqP r = *it;
        const bool first = take.empty() && inflight.empty();
        bool fits = first;
        if (!first)
            fits = inflight_problems + (int64_t)take.size() + 1 <= cfg.max_slots &&
                   inflight_bytes + bytes + r->bytes <= budget_now;
        if (!fits) {
            // a request passed over by kMaxSkips waves stops the ones behind it from passing it
            if (r->skipped >= kMaxSkips) break;
            passed.push_back(r);
            ++it;
            continue;
        }
        it = pending.erase(it);
        r->state = TINV_REQ_RUNNING;
        bytes += r->bytes;
        work += request_work(r->n);
        take.push_back(r);
    }
    if (take.empty()) return false;
    for (ReqP& r : passed) ++r->skipped;
    // SMs: the wave's share of the free SMs by work; one stream's share stays free for later
    // arrivals while other streams are free and requests remain, unless this is the last one
    const double rest = pend_work - work;
    int ctas = free_sms;
    if (free_streams > 1 && pend_work > 0.0)
        ctas = (int)llround((double)free_sms * work / pend_work);
    if (free_streams > 1 && rest <= 0.0) ctas = free_sms - share;
    ctas = std::max(std::min(share, free_sms), std::min(ctas, free_sms));
    ctas = std::max(1, ctas);
    slot_busy[slot] = true;
    inflight_bytes += bytes;
    inflight_problems += (int64_t)take.size();
    sms_used += ctas;
    ++waves;
    wave_problems += take.size();
    cv_done.notify_all();  // states changed to running
    mu.unlock();
    Wave* w = launch(std::move(take), slot, ctas);
    mu.lock();
    inflight.push_back(w);
    max_inflight_seen = std::max<uint64_t>(max_inflight_seen, inflight.size());
    return true;
}

void tinv_server::run()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        // completions
        std::vector<Wave*> done;
        for (size_t i = 0; i < inflight.size();) {
            if (inflight[i]->finished.load()) {
                done.push_back(inflight[i]);
                inflight.erase(inflight.begin() + (long)i);
            } else {
                ++i;
            }
        }
        if (!done.empty()) {
            lk.unlock();
            for (Wave* w : done) {
                finish(w);
                delete w;
            }
            lk.lock();
            continue;
        }
        // admission (takes and releases the lock around the wave's enqueueing)
        if (admit()) continue;
        if (stopping && pending.empty() && inflight.empty()) break;
        // sleep until something changes (a bounded wait guards against a lost wake-up)
        cv_work.wait_for(lk, std::chrono::milliseconds(inflight.empty() ? 50 : 2));
    }
}

extern "C" {

void tinv_server_cfg_default(tinv_server_cfg* c)
{
    if (!c) return;
    memset(c, 0, sizeof(*c));
    c->max_slots = 4096;
    c->max_inflight = 4;
    c->hbm_fraction = 0.5;
    c->method = TINV_CWY;
    c->max_pending = 65536;
}

int tinv_server_create(const tinv_server_cfg* cfg, tinv_server** out)
{
    if (!out) return -2;
    *out = nullptr;
    tinv_server_cfg c;
    if (cfg)
        c = *cfg;
    else
        tinv_server_cfg_default(&c);
    if (c.max_slots <= 0) c.max_slots = 4096;
    if (c.max_inflight <= 0) c.max_inflight = 2;
    if (c.max_pending <= 0) c.max_pending = 65536;
    if (!(c.hbm_fraction > 0.0)) c.hbm_fraction = 0.5;
    if (c.hbm_fraction > 0.95) return -1;
    if (c.max_inflight > 8) return -1;
    if (c.method != TINV_CWY && c.method != TINV_MGS) return -1;
    if (cudaSetDevice(c.device) != cudaSuccess) return TINV_ENODEV;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return TINV_ENODEV;
    tinv_server* s = new tinv_server;
    s->cfg = c;
    s->device = c.device;
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, c.device);
    if (s->sms < 1) s->sms = 1;
    s->budget = (size_t)(c.hbm_fraction * (double)free_b);
    s->streams.resize((size_t)c.max_inflight, nullptr);
    s->staging.resize((size_t)c.max_inflight);
    s->slot_busy.assign((size_t)c.max_inflight, false);
    for (auto& st : s->streams) {
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (auto& t : s->streams)
                if (t) cudaStreamDestroy(t);
            delete s;
            return TINV_ECUDA;
        }
    }
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return 0;
}

int tinv_submit(tinv_server* srv, int64_t n, const double* d, const double* e, const double* w,
                double* Z, uint64_t seed, uint64_t* ticket)
{
    if (!srv) return -1;
    if (n < 1) return -2;
    if (!d) return -3;
    if (n > 1 && !e) return -4;
    if (!Z) return -6;
    if (!ticket) return -8;
    for (int64_t i = 0; i < n; ++i)
        if (!isfinite(d[i])) return -3;
    for (int64_t i = 0; i + 1 < n; ++i)
        if (!isfinite(e[i])) return -4;
    if (w) {
        for (int64_t i = 0; i < n; ++i)
            if (!isfinite(w[i]) || (i > 0 && !(w[i] >= w[i - 1]))) return -5;
    }
    auto r = std::make_shared<Req>();
    r->n = n;
    r->d.assign(d, d + n);
    if (n > 1) r->e.assign(e, e + n - 1);
    r->has_w = w != nullptr;
    if (w) r->w.assign(w, w + n);
    r->Z = Z;
    r->seed = seed;
    r->bytes = request_bytes(n);
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stopping) return TINV_ECANCELED;
    if (r->bytes > srv->budget) {
        ++srv->rejected;
        return TINV_ENOTSUP;  // larger than the whole memory budget
    }
    if ((int64_t)srv->pending.size() >= srv->cfg.max_pending) {
        ++srv->rejected;
        return TINV_EAGAIN;
    }
    r->ticket = srv->next_ticket++;
    r->t_submit = Clock::now();
    if (!srv->any_submit) {
        srv->any_submit = true;
        srv->t_first = r->t_submit;
    }
    srv->table[r->ticket] = r;
    srv->pending.push_back(r);
    ++srv->submitted;
    *ticket = r->ticket;
    srv->cv_work.notify_all();
    return 0;
}

int tinv_poll(tinv_server* srv, uint64_t ticket, int32_t* state)
{
    if (!srv) return -1;
    if (!state) return -3;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->table.find(ticket);
    if (it == srv->table.end()) return -2;
    *state = it->second->state;
    return 0;
}

int tinv_wait(tinv_server* srv, uint64_t ticket, int32_t timeout_ms, int64_t* info)
{
    if (!srv) return -1;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->table.find(ticket);
    if (it == srv->table.end()) return -2;
    ReqP r = it->second;
    auto final_state = [&] {
        return r->state == TINV_REQ_DONE || r->state == TINV_REQ_CANCELLED ||
               r->state == TINV_REQ_FAILED;
    };
    if (timeout_ms < 0) {
        srv->cv_done.wait(lk, final_state);
    } else if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), final_state)) {
        return TINV_ETIMEDOUT;
    }
    srv->table.erase(ticket);
    if (r->state == TINV_REQ_CANCELLED) return TINV_ECANCELED;
    if (r->state == TINV_REQ_FAILED) return r->rc;
    if (info) *info = r->info;
    return 0;
}

int tinv_cancel(tinv_server* srv, uint64_t ticket)
{
    if (!srv) return -1;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->table.find(ticket);
    if (it == srv->table.end()) return -2;
    Req& r = *it->second;
    if (r.state == TINV_REQ_PENDING) {
        for (auto p = srv->pending.begin(); p != srv->pending.end(); ++p)
            if ((*p)->ticket == ticket) {
                srv->pending.erase(p);
                break;
            }
        r.state = TINV_REQ_CANCELLED;
        r.t_done = Clock::now();
        ++srv->cancelled;
        srv->cv_done.notify_all();
        return 0;
    }
    if (r.state == TINV_REQ_RUNNING) {
        if (r.delivering) return 1;  // its result is being written to Z: it completes
        r.cancel = true;             // the GPU work finishes; its result is not written to Z
        return 0;
    }
    return r.state == TINV_REQ_CANCELLED ? TINV_ECANCELED : 1;  // 1: already finished
}

int tinv_server_stats(tinv_server* srv, tinv_stats* out)
{
    if (!srv) return -1;
    if (!out) return -2;
    std::lock_guard<std::mutex> lk(srv->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = srv->submitted;
    out->completed = srv->completed;
    out->cancelled = srv->cancelled;
    out->failed = srv->failed;
    out->rejected = srv->rejected;
    out->waves = srv->waves;
    out->max_inflight_seen = srv->max_inflight_seen;
    out->pending = srv->pending.size();
    out->inflight_waves = srv->inflight.size();
    out->mean_wave_problems = srv->waves ? (double)srv->wave_problems / (double)srv->waves : 0.0;
    if (!srv->lat_ms.empty()) {
        std::vector<double> v = srv->lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            const double x = p * (double)(v.size() - 1);
            const size_t i = (size_t)x;
            const double f = x - (double)i;
            return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double s = 0.0;
        for (double x : v) s += x;
        out->mean_ms = s / (double)v.size();
        const double span = std::chrono::duration<double>(srv->t_last - srv->t_first).count();
        if (span > 0.0) {
            out->problems_per_s = (double)srv->completed / span;
            out->eigvecs_per_s = srv->eigvecs_done / span;
        }
    }
    return 0;
}

int tinv_server_destroy(tinv_server* srv)
{
    if (!srv) return -1;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stopping = true;
        srv->cv_work.notify_all();
    }
    if (srv->worker.joinable()) srv->worker.join();
    for (auto& st : srv->streams) {
        if (st) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
    }
    for (auto& sg : srv->staging) {
        if (sg.in) cudaFreeHost(sg.in);
        if (sg.z) cudaFreeHost(sg.z);
        if (sg.tab) cudaFreeHost(sg.tab);
    }
    {
        // wake any caller still waiting on a request of this server
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->cv_done.notify_all();
    }
    delete srv;
    return 0;
}

}  // extern "C"
