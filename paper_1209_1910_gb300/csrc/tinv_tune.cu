// tinv_tune.cu -- autotuner and tune cache for the cluster kernel's launch parameters: the team
// cap (tinv_tune), the cap and the block size of the blocked compact-WY path together
// (tinv_tune_auto), and both for a batch keyed by its size profile (tinv_tune_batch).
//
// A cluster with m_c members is processed by a team of G CTAs that split every member sweep of
// Alg. 4 (the passes over Y of Sec. 3.3.2 and the solve) and meet at team barriers.  A larger
// team has more FP64 units but waits longer at every barrier for its slowest CTA; the automatic
// rule gives each cluster a share of the grid proportional to its m_c^2 n work (capped at n/16
// and kTeamMax).  The tuner measures instead: it times tinv_ex on the caller's problem once per
// candidate cap and keeps the fastest, and caches the choice for the problem's shape.  The cache
// can be written to and read from a text file (tinv_tune_save / tinv_tune_load, or the file named
// by the environment variable TINV_TUNE_CACHE), keyed by the device's name and SM count so that a
// file carries over between processes and machines with the same GPU.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/tinv.h"
#include "tinv_internal.h"

using namespace tinvx;

namespace {

// What was tuned: the cap alone (tinv_tune), the cap and the block size of one problem
// (tinv_tune_auto), or both for a batch (tinv_tune_batch).
enum TuneKind : int32_t { kTuneCap = 0, kTuneAuto = 1, kTuneBatch = 2 };

// The device model and the shape of a problem as far as the team schedule sees it.  For a batch
// n is the total order, m the number of problems, nclu a hash of the problems' sizes (the count
// of each power-of-two order class) and largest the largest order.
struct TuneKey {
    int32_t kind;
    std::string dev;  // device name (tabs and line breaks replaced by '_')
    int32_t sms, method, grid, block_in;
    int64_t n, m, nclu, largest;
    bool operator<(const TuneKey& b) const
    {
        return std::tie(kind, dev, sms, method, grid, block_in, n, m, nclu, largest) <
               std::tie(b.kind, b.dev, b.sms, b.method, b.grid, b.block_in, b.n, b.m, b.nclu, b.largest);
    }
};

struct TuneVal {
    int32_t max_team;
    int32_t block;
    float ms;
};

std::mutex g_mu;
std::map<TuneKey, TuneVal> g_cache;  // guarded by g_mu
bool g_env_loaded = false;          // guarded by g_mu

constexpr const char* kFileTagV1 = "# tinv tune cache v1";
constexpr const char* kFileTag = "# tinv tune cache v2";

// File format v2: the tag line, then one entry per line, tab-separated: kind (0 cap, 1 cap and
// block, 2 batch), device name, SM count, method, grid cap, block of the options, n, m, clusters
// with >= 2 members (batch: size-profile hash), largest cluster (batch: largest order), chosen
// cap, chosen block, milliseconds.  Files of v1 (no kind and no blocks) are read as kind 0.
int save_locked(const char* path)
{
    FILE* f = fopen(path, "w");
    if (!f) return -2;
    int ok = fprintf(f, "%s\n", kFileTag) > 0;
    for (const auto& kv : g_cache) {
        const TuneKey& k = kv.first;
        ok = ok && fprintf(f, "%d\t%s\t%d\t%d\t%d\t%d\t%lld\t%lld\t%lld\t%lld\t%d\t%d\t%.6g\n", k.kind,
                           k.dev.c_str(), k.sms, k.method, k.grid, k.block_in, (long long)k.n,
                           (long long)k.m, (long long)k.nclu, (long long)k.largest,
                           kv.second.max_team, kv.second.block, (double)kv.second.ms) > 0;
    }
    ok = (fclose(f) == 0) && ok;
    return ok ? 0 : -2;
}

// Merges the file's entries into the cache; returns the number read, -2 (unreadable or not a
// cache file) or -3 (a malformed entry: the entries before it are kept).
int load_locked(const char* path)
{
    FILE* f = fopen(path, "r");
    if (!f) return -2;
    char line[1024];
    int version = 0;
    if (fgets(line, sizeof line, f)) {
        if (strncmp(line, kFileTag, strlen(kFileTag)) == 0)
            version = 2;
        else if (strncmp(line, kFileTagV1, strlen(kFileTagV1)) == 0)
            version = 1;
    }
    if (!version) {
        fclose(f);
        return -2;
    }
    int count = 0, rc = 0;
    while (fgets(line, sizeof line, f)) {
        if (line[0] == '\n' || line[0] == '\0') continue;
        TuneKey k;
        k.kind = kTuneCap;
        k.block_in = 0;
        char* name = line;
        if (version == 2) {
            int kind;
            int used = 0;
            if (sscanf(line, "%d\t%n", &kind, &used) != 1 || used == 0 || kind < kTuneCap || kind > kTuneBatch) {
                rc = -3;
                break;
            }
            k.kind = kind;
            name = line + used;
        }
        char* tab = strchr(name, '\t');
        if (!tab || tab == name) {
            rc = -3;
            break;
        }
        k.dev.assign(name, (size_t)(tab - name));
        long long n, m, nclu, largest;
        int sms, method, grid, mt, bin = 0, bout = 0;
        double ms;
        char tail;
        bool bad;
        if (version == 2)
            bad = sscanf(tab + 1, "%d\t%d\t%d\t%d\t%lld\t%lld\t%lld\t%lld\t%d\t%d\t%lf %c", &sms, &method,
                         &grid, &bin, &n, &m, &nclu, &largest, &mt, &bout, &ms, &tail) != 11;
        else
            bad = sscanf(tab + 1, "%d\t%d\t%d\t%lld\t%lld\t%lld\t%lld\t%d\t%lf %c", &sms, &method, &grid, &n,
                         &m, &nclu, &largest, &mt, &ms, &tail) != 9;
        const bool batch = k.kind == kTuneBatch;
        if (bad || sms <= 0 || grid < 0 || n < 0 || m < 0 || (!batch && m > n) || nclu < 0 ||
            largest < 0 || (!batch && largest > m) || mt < 0 || mt > kTeamMax || !(ms >= 0.0 && ms < 1e30) ||
            bin < 0 || bin > kBlockMax || bout < 0 || bout > kBlockMax ||
            (method != TINV_CWY && method != TINV_MGS)) {
            rc = -3;
            break;
        }
        k.sms = sms;
        k.method = method;
        k.grid = grid;
        k.block_in = bin;
        k.n = n;
        k.m = m;
        k.nclu = nclu;
        k.largest = largest;
        g_cache[k] = TuneVal{mt, bout, (float)ms};
        ++count;
    }
    fclose(f);
    return rc ? rc : count;
}

// The file named by TINV_TUNE_CACHE is read once, before the first lookup.
void load_env_locked()
{
    if (g_env_loaded) return;
    g_env_loaded = true;
    const char* p = getenv("TINV_TUNE_CACHE");
    if (p && *p) load_locked(p);
}

std::string device_name(int dev, int* sms)
{
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        *sms = 0;
        return std::string("unknown");
    }
    *sms = prop.multiProcessorCount;
    std::string s(prop.name);
    for (char& c : s)
        if (c == '\t' || c == '\n' || c == '\r') c = '_';
    return s.empty() ? std::string("unknown") : s;
}

// Clusters with >= 2 members and the largest cluster, from the plan's head indices (members of
// a cluster are consecutive and share their head).
void signature(const std::vector<int32_t>& head, int64_t* nclu, int64_t* largest)
{
    int64_t count = 0, big = 1, run = 0;
    for (size_t j = 0; j < head.size(); ++j) {
        if (head[j] == (int32_t)j) {
            if (run >= 2) ++count;
            run = 1;
        } else {
            ++run;
        }
        big = run > big ? run : big;
    }
    if (run >= 2) ++count;
    *nclu = count;
    *largest = head.empty() ? 0 : big;
}

}  // namespace

extern "C" void tinv_tune_clear(void)
{
    std::lock_guard<std::mutex> g(g_mu);
    g_cache.clear();
}

extern "C" int tinv_tune_save(const char* path)
{
    if (!path) return -1;
    std::lock_guard<std::mutex> g(g_mu);
    return save_locked(path);
}

extern "C" int tinv_tune_load(const char* path)
{
    if (!path) return -1;
    std::lock_guard<std::mutex> g(g_mu);
    return load_locked(path);
}

namespace {

// One warm-up call and `reps` timed calls of `run` (each enqueues one call on st) between CUDA
// events; the mean device milliseconds, or an error code (a bounded wait that expired in the last
// call, read from the device status word dinfo, fails the tuning).
template <class Run>
int time_calls(Run run, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1, int32_t reps,
               const int64_t* dinfo, int64_t ninfo, float* out_ms)
{
    int rc = run();  // warm-up
    if (!rc) rc = cuda_code(cudaEventRecord(ev0, st));
    for (int32_t r = 0; r < reps && !rc; ++r) rc = run();
    if (!rc) rc = cuda_code(cudaEventRecord(ev1, st));
    if (!rc) rc = cuda_code(cudaEventSynchronize(ev1));
    if (!rc && dinfo) {
        std::vector<int64_t> info((size_t)ninfo);
        rc = cuda_code(cudaMemcpy(info.data(), dinfo, (size_t)ninfo * sizeof(int64_t), cudaMemcpyDeviceToHost));
        for (int64_t q = 0; q < ninfo && !rc; ++q)
            if (info[(size_t)q] < 0) rc = (int)info[(size_t)q];
    }
    float t = 0.0f;
    if (!rc) rc = cuda_code(cudaEventElapsedTime(&t, ev0, ev1));
    *out_ms = t / (float)reps;
    return rc;
}

// Caps that can bind for a grid of P CTAs and orders up to nmax: 2, 4, 8, ... below the grid,
// nmax/16 and kTeamMax.
std::vector<int32_t> cap_candidates(int32_t P, int64_t nmax)
{
    std::vector<int32_t> cand;
    for (int32_t c = 2; c < P && (int64_t)c <= nmax / 16 && c <= kTeamMax; c *= 2) cand.push_back(c);
    return cand;
}

// The two-stage search of tinv_tune_auto / tinv_tune_batch: the block size first (one member at
// a time, blocks of 4 and of 8) with the automatic caps, then the caps with the chosen block.  A
// candidate replaces the current choice only when it is at least 1% faster.  `timed(cap, block,
// &ms)` runs and times one candidate.
template <class Timed>
int two_stage(Timed timed, bool cwy, bool teams, int32_t P, int64_t nmax, int32_t* cap,
              int32_t* block, float* ms)
{
    float best = 0.0f;
    int rc = timed(0, 0, &best);
    int32_t bpick = 0, cpick = 0;
    if (!rc && cwy && teams) {
        for (int32_t b : {4, 8, 16}) {
            float t = 0.0f;
            rc = timed(0, b, &t);
            if (rc) break;
            if (t < 0.99f * best) {
                best = t;
                bpick = b;
            }
        }
        const float base = best;
        for (int32_t c : cap_candidates(P, nmax)) {
            if (rc) break;
            float t = 0.0f;
            rc = timed(c, bpick, &t);
            if (!rc && t < best && t < 0.99f * base) {
                best = t;
                cpick = c;
            }
        }
    }
    *cap = cpick;
    *block = bpick;
    *ms = best;
    return rc;
}

}  // namespace

extern "C" int tinv_tune(int64_t n, const double* d, const double* e, int64_t m, const double* w,
                         const tinv_opts* o, int32_t reps, int32_t* max_team, float* ms,
                         int32_t* cached)
{
    tinv_opts op;
    if (o)
        op = *o;
    else
        tinv_opts_default(&op);
    if (n < 0) return -1;
    if (n > 0 && !d) return -2;
    if (n > 1 && !e) return -3;
    if (m < 0 || m > n) return -4;
    if (m > 0 && !w) return -5;
    if (op.method != TINV_CWY && op.method != TINV_MGS) return -6;
    if (reps < 1) return -7;
    if (!max_team) return -8;
    if (!op.device_ptrs) {
        if (!all_finite(d, n) || (n > 1 && !all_finite(e, n - 1))) return -2;
        if (!all_finite(w, m) || !ascending(w, m)) return -5;
    }
    *max_team = 0;
    if (ms) *ms = 0.0f;
    if (cached) *cached = 0;
    if (n <= 1 || m == 0) return 0;
    if (n > (int64_t)INT32_MAX / 2 || m > (int64_t)INT32_MAX / 2) return TINV_ENOTSUP;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TINV_ENODEV;
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return TINV_ENODEV;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int rc = 0;
    {
        DevBuf bd, be, bw, bz, bwp, bhead, bscal, bws, binfo;
        const double *pd = d, *pe = e, *pw = w;
        cudaError_t ce = cudaSuccess;
        if (!op.device_ptrs) {
            ce = bd.alloc((size_t)n * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = be.alloc((size_t)(n - 1) * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = bw.alloc((size_t)m * sizeof(double), st, true);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(bd.p, d, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(be.p, e, (size_t)(n - 1) * sizeof(double), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(bw.p, w, (size_t)m * sizeof(double), cudaMemcpyHostToDevice, st);
            pd = (const double*)bd.p;
            pe = (const double*)be.p;
            pw = (const double*)bw.p;
        }
        // the options of every call below: device pointers on the tuner's stream, and none of
        // the caller's outputs
        tinv_opts po = op;
        po.device_ptrs = 1;
        po.stream = (void*)st;
        po.workspace = nullptr;
        po.workspace_bytes = 0;
        po.iters = nullptr;
        po.info = nullptr;
        po.counters = nullptr;
        po.phase_ms = nullptr;
        po.table_ready = 0;
        po.max_team = 0;
        if (ce == cudaSuccess) ce = bwp.alloc((size_t)m * sizeof(double), st, true);
        if (ce == cudaSuccess) ce = bhead.alloc((size_t)m * sizeof(int32_t), st, true);
        if (ce == cudaSuccess) ce = bscal.alloc(3 * sizeof(double), st, true);
        rc = cuda_code(ce);
        if (!rc)
            rc = tinv_plan(n, pd, pe, m, pw, (double*)bwp.p, (int32_t*)bhead.p, (double*)bscal.p, &po);
        std::vector<int32_t> head((size_t)m);
        if (!rc) {
            ce = cudaMemcpyAsync(head.data(), bhead.p, (size_t)m * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
            rc = cuda_code(ce);
        }
        TuneKey key;
        key.kind = kTuneCap;
        key.block_in = opts_block(op);
        key.dev = device_name(dev, &key.sms);
        key.method = op.method;
        key.grid = op.grid_ctas;
        key.n = n;
        key.m = m;
        key.nclu = key.largest = 0;
        bool hit = false;
        if (!rc) {
            signature(head, &key.nclu, &key.largest);
            std::lock_guard<std::mutex> g(g_mu);
            load_env_locked();
            auto it = g_cache.find(key);
            if (it != g_cache.end()) {
                *max_team = it->second.max_team;
                if (ms) *ms = it->second.ms;
                if (cached) *cached = 1;
                hit = true;
            }
        }
        if (!rc && !hit) {
            // candidates: the automatic rule, then caps that can bind (below the grid and n/16);
            // teams exist only for CWY clusters of >= 2 members
            std::vector<int32_t> cand{0};
            const int32_t P = chain_grid(op.grid_ctas, n);
            if (op.method == TINV_CWY && key.nclu > 0)
                for (int32_t c = 2; c < P && (int64_t)c <= n / 16 && c <= kTeamMax; c *= 2) cand.push_back(c);
            const size_t need = tinv_workspace_size(n, m, &po);
            ce = bz.alloc((size_t)n * (size_t)m * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = bws.alloc(need, st, true);
            if (ce == cudaSuccess) ce = binfo.alloc(sizeof(int64_t), st, true);
            if (ce == cudaSuccess) ce = cudaEventCreate(&ev0);
            if (ce == cudaSuccess) ce = cudaEventCreate(&ev1);
            rc = cuda_code(ce);
            po.workspace = bws.p;
            po.workspace_bytes = need;
            po.info = (int64_t*)binfo.p;  // status of the last call: a timed-out wait fails the tuning
            float best = 0.0f, automs = 0.0f;
            int32_t pick = 0;
            // with device pointers tinv_ex returns 0 once the work is enqueued, or an error
            auto run = [&]() {
                const int r = tinv_ex(n, pd, pe, m, pw, (double*)bz.p, n, &po, nullptr);
                return r > 0 ? 0 : r;
            };
            for (size_t i = 0; i < cand.size() && !rc; ++i) {
                po.max_team = cand[i];
                rc = run();  // warm-up
                if (!rc) rc = cuda_code(cudaEventRecord(ev0, st));
                for (int32_t r = 0; r < reps && !rc; ++r) rc = run();
                if (!rc) rc = cuda_code(cudaEventRecord(ev1, st));
                if (!rc) rc = cuda_code(cudaEventSynchronize(ev1));
                int64_t info = 0;
                if (!rc) rc = cuda_code(cudaMemcpy(&info, binfo.p, sizeof(int64_t), cudaMemcpyDeviceToHost));
                if (!rc && info < 0) rc = (int)info;
                float t = 0.0f;
                if (!rc) rc = cuda_code(cudaEventElapsedTime(&t, ev0, ev1));
                if (rc) break;
                t /= (float)reps;
                if (cand[i] == 0) {
                    automs = best = t;
                } else if (t < best && t < 0.99f * automs) {
                    // a cap replaces the automatic rule only when it is at least 1% faster
                    best = t;
                    pick = cand[i];
                }
            }
            if (!rc) {
                *max_team = pick;
                if (ms) *ms = best;
                std::lock_guard<std::mutex> g(g_mu);
                g_cache[key] = TuneVal{pick, key.block_in, best};
                const char* p = getenv("TINV_TUNE_CACHE");
                if (p && *p) save_locked(p);  // best effort: the choice is returned either way
            }
        }
        cudaStreamSynchronize(st);
    }
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    cudaStreamDestroy(st);
    return rc;
}

namespace {

// 64-bit FNV-1a hash of the count of problems in each power-of-two order class (the batch's
// size profile), kept to 62 bits so that it reads back as a non-negative integer.
int64_t size_profile(int64_t nprob, const int64_t* n)
{
    int64_t cls[64] = {};
    for (int64_t q = 0; q < nprob; ++q) {
        int b = 0;
        for (int64_t v = n[q]; v > 1; v >>= 1) ++b;
        cls[b]++;
    }
    uint64_t h = 1469598103934665603ull;
    for (int b = 0; b < 64; ++b) {
        for (int k = 0; k < 8; ++k) {
            h ^= (uint64_t)((cls[b] >> (8 * k)) & 0xff);
            h *= 1099511628211ull;
        }
    }
    return (int64_t)(h >> 2);
}

int tuned_out(tinv_tuning* out, int32_t cap, int32_t block, float ms, int32_t cached)
{
    memset(out, 0, sizeof(*out));
    out->max_team = cap;
    out->block = block;
    out->ms = ms;
    out->cached = cached;
    return 0;
}

}  // namespace

extern "C" int tinv_tune_auto(int64_t n, const double* d, const double* e, int64_t m, const double* w,
                              const tinv_opts* o, int32_t reps, tinv_tuning* out)
{
    tinv_opts op;
    if (o)
        op = *o;
    else
        tinv_opts_default(&op);
    if (n < 0) return -1;
    if (n > 0 && !d) return -2;
    if (n > 1 && !e) return -3;
    if (m < 0 || m > n) return -4;
    if (m > 0 && !w) return -5;
    if (op.method != TINV_CWY && op.method != TINV_MGS) return -6;
    if (reps < 1) return -7;
    if (!out) return -8;
    if (!op.device_ptrs) {
        if (!all_finite(d, n) || (n > 1 && !all_finite(e, n - 1))) return -2;
        if (!all_finite(w, m) || !ascending(w, m)) return -5;
    }
    tuned_out(out, 0, 0, 0.0f, 0);
    if (n <= 1 || m == 0) return 0;
    if (n > (int64_t)INT32_MAX / 2 || m > (int64_t)INT32_MAX / 2) return TINV_ENOTSUP;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TINV_ENODEV;
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return TINV_ENODEV;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int rc = 0;
    {
        DevBuf bd, be, bw, bz, bwp, bhead, bscal, bws, binfo;
        const double *pd = d, *pe = e, *pw = w;
        cudaError_t ce = cudaSuccess;
        if (!op.device_ptrs) {
            ce = bd.alloc((size_t)n * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = be.alloc((size_t)(n - 1) * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = bw.alloc((size_t)m * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(bd.p, d, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(be.p, e, (size_t)(n - 1) * sizeof(double), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(bw.p, w, (size_t)m * sizeof(double), cudaMemcpyHostToDevice, st);
            pd = (const double*)bd.p;
            pe = (const double*)be.p;
            pw = (const double*)bw.p;
        }
        tinv_opts po = op;
        po.device_ptrs = 1;
        po.stream = (void*)st;
        po.workspace = nullptr;
        po.workspace_bytes = 0;
        po.iters = nullptr;
        po.info = nullptr;
        po.counters = nullptr;
        po.phase_ms = nullptr;
        po.table_ready = 0;
        po.max_team = 0;
        po.block = 0;
        if (ce == cudaSuccess) ce = bwp.alloc((size_t)m * sizeof(double), st, true);
        if (ce == cudaSuccess) ce = bhead.alloc((size_t)m * sizeof(int32_t), st, true);
        if (ce == cudaSuccess) ce = bscal.alloc(3 * sizeof(double), st, true);
        rc = cuda_code(ce);
        if (!rc) rc = tinv_plan(n, pd, pe, m, pw, (double*)bwp.p, (int32_t*)bhead.p, (double*)bscal.p, &po);
        std::vector<int32_t> head((size_t)m);
        if (!rc) {
            ce = cudaMemcpyAsync(head.data(), bhead.p, (size_t)m * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
            rc = cuda_code(ce);
        }
        TuneKey key;
        key.kind = kTuneAuto;
        key.block_in = 0;
        key.dev = device_name(dev, &key.sms);
        key.method = op.method;
        key.grid = op.grid_ctas;
        key.n = n;
        key.m = m;
        key.nclu = key.largest = 0;
        bool hit = false;
        if (!rc) {
            signature(head, &key.nclu, &key.largest);
            std::lock_guard<std::mutex> g(g_mu);
            load_env_locked();
            auto it = g_cache.find(key);
            if (it != g_cache.end()) {
                tuned_out(out, it->second.max_team, it->second.block, it->second.ms, 1);
                hit = true;
            }
        }
        if (!rc && !hit) {
            tinv_opts pmax = po;
            pmax.block = kBlockMax;  // the largest layout of all candidates
            const size_t need = tinv_workspace_size(n, m, &pmax);
            ce = bz.alloc((size_t)n * (size_t)m * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = bws.alloc(need, st, true);
            if (ce == cudaSuccess) ce = binfo.alloc(sizeof(int64_t), st, true);
            if (ce == cudaSuccess) ce = cudaEventCreate(&ev0);
            if (ce == cudaSuccess) ce = cudaEventCreate(&ev1);
            rc = cuda_code(ce);
            po.workspace = bws.p;
            po.workspace_bytes = need;
            po.info = (int64_t*)binfo.p;
            auto timed = [&](int32_t cap, int32_t block, float* t) {
                po.max_team = cap;
                po.block = block;
                auto run = [&]() {
                    const int r = tinv_ex(n, pd, pe, m, pw, (double*)bz.p, n, &po, nullptr);
                    return r > 0 ? 0 : r;
                };
                return time_calls(run, st, ev0, ev1, reps, (const int64_t*)binfo.p, 1, t);
            };
            int32_t cap = 0, block = 0;
            float best = 0.0f;
            if (!rc)
                rc = two_stage(timed, op.method == TINV_CWY, key.nclu > 0, chain_grid(op.grid_ctas, n), n,
                               &cap, &block, &best);
            if (!rc) {
                tuned_out(out, cap, block, best, 0);
                std::lock_guard<std::mutex> g(g_mu);
                g_cache[key] = TuneVal{cap, block, best};
                const char* p = getenv("TINV_TUNE_CACHE");
                if (p && *p) save_locked(p);
            }
        }
        cudaStreamSynchronize(st);
    }
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    cudaStreamDestroy(st);
    return rc;
}

extern "C" int tinv_tune_batch(int64_t nprob, const int64_t* n, const int64_t* off_de,
                               const int64_t* off_z, const double* d, const double* e,
                               const double* w, const tinv_opts* o, int32_t reps, tinv_tuning* out)
{
    tinv_opts op;
    if (o)
        op = *o;
    else
        tinv_opts_default(&op);
    if (nprob < 0) return -1;
    if (nprob > 0 && (!n || !off_de || !off_z)) return !n ? -2 : (!off_de ? -3 : -4);
    if (nprob > 0 && (!d || !e || !w)) return !d ? -5 : (!e ? -6 : -7);
    if (op.method != TINV_CWY && op.method != TINV_MGS) return -8;
    if (reps < 1) return -9;
    if (!out) return -10;
    tuned_out(out, 0, 0, 0.0f, 0);
    int64_t de_len = 0, z_len = 0, total = 0, nmax = 0;
    for (int64_t q = 0; q < nprob; ++q) {
        if (n[q] < 0 || off_de[q] < 0 || off_z[q] < 0) return n[q] < 0 ? -2 : (off_de[q] < 0 ? -3 : -4);
        de_len = std::max(de_len, off_de[q] + n[q]);
        z_len = std::max(z_len, off_z[q] + n[q] * n[q]);
        total += n[q];
        nmax = std::max(nmax, n[q]);
    }
    if (total == 0) return 0;
    if (!op.device_ptrs) {
        for (int64_t q = 0; q < nprob; ++q) {
            if (n[q] == 0) continue;
            if (!all_finite(d + off_de[q], n[q])) return -5;
            if (n[q] > 1 && !all_finite(e + off_de[q], n[q] - 1)) return -6;
            if (!all_finite(w + off_de[q], n[q]) || !ascending(w + off_de[q], n[q])) return -7;
        }
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TINV_ENODEV;
    TuneKey key;
    key.kind = kTuneBatch;
    key.block_in = 0;
    key.dev = device_name(dev, &key.sms);
    key.method = op.method;
    key.grid = op.grid_ctas;
    key.n = total;
    key.m = nprob;
    key.nclu = size_profile(nprob, n);
    key.largest = nmax;
    {
        std::lock_guard<std::mutex> g(g_mu);
        load_env_locked();
        auto it = g_cache.find(key);
        if (it != g_cache.end()) return tuned_out(out, it->second.max_team, it->second.block, it->second.ms, 1);
    }
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return TINV_ENODEV;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int rc = 0;
    {
        DevBuf bd, be, bw, bz, bws, binfo;
        const double *pd = d, *pe = e, *pw = w;
        cudaError_t ce = cudaSuccess;
        if (!op.device_ptrs) {
            ce = bd.alloc((size_t)de_len * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = be.alloc((size_t)de_len * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = bw.alloc((size_t)de_len * sizeof(double), st, true);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(bd.p, d, (size_t)de_len * sizeof(double), cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(bw.p, w, (size_t)de_len * sizeof(double), cudaMemcpyHostToDevice, st);
            // e of problem q has n_q - 1 entries: copy per problem (the packed array may end
            // one entry short of de_len)
            for (int64_t q = 0; q < nprob && ce == cudaSuccess; ++q)
                if (n[q] > 1)
                    ce = cudaMemcpyAsync((double*)be.p + off_de[q], e + off_de[q], (size_t)(n[q] - 1) * sizeof(double),
                                         cudaMemcpyHostToDevice, st);
            pd = (const double*)bd.p;
            pe = (const double*)be.p;
            pw = (const double*)bw.p;
        }
        tinv_opts po = op;
        po.device_ptrs = 1;
        po.stream = (void*)st;
        po.iters = nullptr;
        po.info = nullptr;
        po.counters = nullptr;
        po.phase_ms = nullptr;
        po.table_ready = 0;
        po.max_team = 0;
        po.block = kBlockMax;
        const size_t need = tinv_batch_workspace_size(nprob, n, &po);  // the largest layout
        po.block = 0;
        if (ce == cudaSuccess) ce = bz.alloc((size_t)std::max<int64_t>(z_len, 1) * sizeof(double), st, true);
        if (ce == cudaSuccess) ce = bws.alloc(need, st, true);
        if (ce == cudaSuccess) ce = binfo.alloc((size_t)nprob * sizeof(int64_t), st, true);
        if (ce == cudaSuccess) ce = cudaEventCreate(&ev0);
        if (ce == cudaSuccess) ce = cudaEventCreate(&ev1);
        rc = cuda_code(ce);
        po.workspace = bws.p;
        po.workspace_bytes = need;
        auto timed = [&](int32_t cap, int32_t block, float* t) {
            po.max_team = cap;
            po.block = block;
            auto run = [&]() {
                const int r = tinv_batch(nprob, n, off_de, off_z, pd, pe, pw, (double*)bz.p,
                                         (int64_t*)binfo.p, &po);
                return r > 0 ? 0 : r;
            };
            return time_calls(run, st, ev0, ev1, reps, (const int64_t*)binfo.p, nprob, t);
        };
        int32_t cap = 0, block = 0;
        float best = 0.0f;
        if (!rc)
            rc = two_stage(timed, op.method == TINV_CWY, true, chain_grid(op.grid_ctas, nmax), nmax, &cap,
                           &block, &best);
        if (!rc) {
            tuned_out(out, cap, block, best, 0);
            std::lock_guard<std::mutex> g(g_mu);
            g_cache[key] = TuneVal{cap, block, best};
            const char* p = getenv("TINV_TUNE_CACHE");
            if (p && *p) save_locked(p);
        }
        cudaStreamSynchronize(st);
    }
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    cudaStreamDestroy(st);
    return rc;
}
