// tinv_tune.cu -- autotuner and tune cache for the cluster kernel's team cap.
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

#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/tinv.h"
#include "tinv_internal.h"

using namespace tinvx;

namespace {

// The device model and the shape of a problem as far as the team schedule sees it.
struct TuneKey {
    std::string dev;  // device name (tabs and line breaks replaced by '_')
    int32_t sms, method, grid;
    int64_t n, m, nclu, largest;
    bool operator<(const TuneKey& b) const
    {
        return std::tie(dev, sms, method, grid, n, m, nclu, largest) <
               std::tie(b.dev, b.sms, b.method, b.grid, b.n, b.m, b.nclu, b.largest);
    }
};

struct TuneVal {
    int32_t max_team;
    float ms;
};

std::mutex g_mu;
std::map<TuneKey, TuneVal> g_cache;  // guarded by g_mu
bool g_env_loaded = false;          // guarded by g_mu

constexpr const char* kFileTag = "# tinv tune cache v1";

// File format: the tag line, then one entry per line, tab-separated: device name, SM count,
// method, grid cap, n, m, clusters with >= 2 members, largest cluster, chosen cap, milliseconds.
int save_locked(const char* path)
{
    FILE* f = fopen(path, "w");
    if (!f) return -2;
    int ok = fprintf(f, "%s\n", kFileTag) > 0;
    for (const auto& kv : g_cache) {
        const TuneKey& k = kv.first;
        ok = ok && fprintf(f, "%s\t%d\t%d\t%d\t%lld\t%lld\t%lld\t%lld\t%d\t%.6g\n", k.dev.c_str(),
                           k.sms, k.method, k.grid, (long long)k.n, (long long)k.m,
                           (long long)k.nclu, (long long)k.largest, kv.second.max_team,
                           (double)kv.second.ms) > 0;
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
    if (!fgets(line, sizeof line, f) || strncmp(line, kFileTag, strlen(kFileTag)) != 0) {
        fclose(f);
        return -2;
    }
    int count = 0, rc = 0;
    while (fgets(line, sizeof line, f)) {
        if (line[0] == '\n' || line[0] == '\0') continue;
        char* tab = strchr(line, '\t');
        if (!tab || tab == line) {
            rc = -3;
            break;
        }
        TuneKey k;
        k.dev.assign(line, (size_t)(tab - line));
        long long n, m, nclu, largest;
        int sms, method, grid, mt;
        double ms;
        char tail;
        if (sscanf(tab + 1, "%d\t%d\t%d\t%lld\t%lld\t%lld\t%lld\t%d\t%lf %c", &sms, &method, &grid, &n,
                   &m, &nclu, &largest, &mt, &ms, &tail) != 9 ||
            sms <= 0 || grid < 0 || n < 0 || m < 0 || m > n || nclu < 0 || largest < 0 ||
            largest > m || mt < 0 || mt > kTeamMax || !(ms >= 0.0 && ms < 1e30) ||
            (method != TINV_CWY && method != TINV_MGS)) {
            rc = -3;
            break;
        }
        k.sms = sms;
        k.method = method;
        k.grid = grid;
        k.n = n;
        k.m = m;
        k.nclu = nclu;
        k.largest = largest;
        g_cache[k] = TuneVal{mt, (float)ms};
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
                g_cache[key] = TuneVal{pick, best};
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
