// jz_aux.cu -- host-side services around the replica-gluing kernels (none has
// a counterpart in the paper): the persisted autotune cache, the per-job
// JSON-lines record of the server, cancellation and resumable runs.
#include <cuda_runtime.h>

#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <tuple>

#include "jz_host.h"

using namespace jzh;

// ------------------------------------------------------------ tune cache --
namespace {
using TuneKey = std::tuple<std::string, int, int, int, int, int>;   // gpu, d, L, L_t, n, bucket

int traj_bucket(int n_traj)
{
    int b = 0;
    while ((1LL << (b + 1)) <= (long long)n_traj) ++b;
    return b;
}

// GPU names go into JSON strings: keep printable ASCII without quotes or
// backslashes (device names have none; anything else becomes '_').
std::string clean_name(const char* s)
{
    std::string out;
    for (; s && *s; ++s) {
        const char c = *s;
        out += (c >= 32 && c < 127 && c != '"' && c != '\\') ? c : '_';
    }
    return out;
}
}  // namespace

struct jz_tune_cache {
    std::map<TuneKey, int> entries;
};

extern "C" {

int jz_tune_cache_create(jz_tune_cache** out)
{
    if (!out) return ISING_ERR_ARG;
    *out = new (std::nothrow) jz_tune_cache();
    return *out ? ISING_OK : ISING_ERR_NOMEM;
}

void jz_tune_cache_free(jz_tune_cache* c) { delete c; }

int jz_tune_cache_put(jz_tune_cache* c, const char* gpu, int d, int L, int L_t, int n_replica,
                      int n_traj, int cta_threads)
{
    if (!c || !gpu || (d != 2 && d != 3) || L < 2 || L_t < 2 || n_traj < 1 || cta_threads < 0)
        return ISING_ERR_ARG;
    const int n = n_replica == 0 ? 2 : n_replica;
    c->entries[TuneKey(clean_name(gpu), d, L, L_t, n, traj_bucket(n_traj))] = cta_threads;
    return ISING_OK;
}

int jz_tune_cache_get(const jz_tune_cache* c, const char* gpu, int d, int L, int L_t,
                      int n_replica, int n_traj, int* cta_threads)
{
    if (!c || !gpu || !cta_threads || n_traj < 1) return ISING_ERR_ARG;
    const int n = n_replica == 0 ? 2 : n_replica;
    auto it = c->entries.find(TuneKey(clean_name(gpu), d, L, L_t, n, traj_bucket(n_traj)));
    if (it == c->entries.end()) return ISING_ERR_NOT_FOUND;
    *cta_threads = it->second;
    return ISING_OK;
}

int jz_tune_cache_size(const jz_tune_cache* c, int* n)
{
    if (!c || !n) return ISING_ERR_ARG;
    *n = (int)c->entries.size();
    return ISING_OK;
}

int jz_tune_cache_save(const jz_tune_cache* c, const char* path)
{
    if (!c || !path) return ISING_ERR_ARG;
    FILE* f = std::fopen(path, "w");
    if (!f) return ISING_ERR_NOT_FOUND;
    std::fprintf(f, "{\"version\": 1, \"entries\": [\n");
    size_t i = 0;
    for (const auto& e : c->entries) {
        const TuneKey& k = e.first;
        std::fprintf(f,
                     "{\"gpu\": \"%s\", \"d\": %d, \"L\": %d, \"L_t\": %d, \"n_replica\": %d, "
                     "\"traj_bucket\": %d, \"cta_threads\": %d}%s\n",
                     std::get<0>(k).c_str(), std::get<1>(k), std::get<2>(k), std::get<3>(k),
                     std::get<4>(k), std::get<5>(k), e.second,
                     ++i < c->entries.size() ? "," : "");
    }
    std::fprintf(f, "]}\n");
    return std::fclose(f) == 0 ? ISING_OK : ISING_ERR_NOT_FOUND;
}

int jz_tune_cache_load(jz_tune_cache* c, const char* path)
{
    if (!c || !path) return ISING_ERR_ARG;
    FILE* f = std::fopen(path, "r");
    if (!f) return ISING_ERR_NOT_FOUND;
    char line[1024];
    bool header = false, closed = false;
    std::map<TuneKey, int> got;
    int rc = ISING_OK;
    while (std::fgets(line, sizeof line, f)) {
        if (std::strncmp(line, "{\"version\": 1, \"entries\": [", 27) == 0) {
            header = true;
            continue;
        }
        if (std::strncmp(line, "]}", 2) == 0) {
            closed = true;
            continue;
        }
        char gpu[256];
        int d, L, Lt, n, b, t;
        if (!header || closed ||
            std::sscanf(line,
                        "{\"gpu\": \"%255[^\"]\", \"d\": %d, \"L\": %d, \"L_t\": %d, "
                        "\"n_replica\": %d, \"traj_bucket\": %d, \"cta_threads\": %d}",
                        gpu, &d, &L, &Lt, &n, &b, &t) != 7 ||
            (d != 2 && d != 3) || L < 2 || Lt < 2 || n < 2 || b < 0 || b > 40 || t < 0) {
            rc = ISING_ERR_ARG;
            break;
        }
        got[TuneKey(gpu, d, L, Lt, n, b)] = t;
    }
    std::fclose(f);
    if (rc == ISING_OK && (!header || !closed)) rc = ISING_ERR_ARG;
    if (rc == ISING_OK)
        for (const auto& e : got) c->entries[e.first] = e.second;
    return rc;
}

int ising_autotune_cached(ising_ctx* ctx, jz_tune_cache* c, const jz_params* p, int* threads,
                          int* hit)
{
    if (!ctx || !c || !p) return ISING_ERR_ARG;
    int rc = check_params(p);
    if (rc) return rc;
    if (hit) *hit = 0;
    if (p->update == 1) return ising_autotune(ctx, p, threads);   // fixed CTA, nothing cached
    int t = 0;
    if (jz_tune_cache_get(c, ctx->gpu_name.c_str(), p->d, p->L, p->L_t, nrep_of(*p), p->n_traj,
                          &t) == ISING_OK &&
        (rc = ising_set_threads(ctx, p->d, p->L, p->L_t, t)) == ISING_OK) {
        if (hit) *hit = 1;
        if (threads) *threads = t;
        return ISING_OK;
    }
    if ((rc = ising_autotune(ctx, p, &t))) return rc;
    if ((rc = jz_tune_cache_put(c, ctx->gpu_name.c_str(), p->d, p->L, p->L_t, nrep_of(*p),
                                p->n_traj, t)))
        return rc;
    if (threads) *threads = t;
    return ISING_OK;
}

// ------------------------------------------------------------ JSON lines --
int jz_result_json(uint64_t job_id, const jz_params* p, const jz_result* r, char* buf, size_t n)
{
    if (!p || !r || !buf || n == 0) return ISING_ERR_ARG;
    const double latency = r->done_s - r->submit_s;
    const double on_device = r->done_s - r->start_s;
    const bool ok = r->status == ISING_OK;
    // non-finite values (a failed job) are written as null
    auto num = [](double v, char* out, size_t m) {
        if (std::isfinite(v)) std::snprintf(out, m, "%.17g", v);
        else std::snprintf(out, m, "null");
    };
    char lr[32], ds[32], de[32], rate[32];
    num(ok ? r->log_ratio : NAN, lr, sizeof lr);
    num(ok ? r->delta_S2 : NAN, ds, sizeof ds);
    num(ok ? r->delta_S2_err : NAN, de, sizeof de);
    num(ok && on_device > 0 ? (double)r->updates / on_device : NAN, rate, sizeof rate);
    const int len = std::snprintf(
        buf, n,
        "{\"job\": %llu, \"d\": %d, \"L\": %d, \"L_t\": %d, \"beta\": %.17g, \"l\": %d, "
        "\"n_step\": %d, \"n_sweep\": %d, \"n_therm\": %d, \"n_traj\": %d, \"direction\": %d, "
        "\"update\": %d, \"therm_update\": %d, \"protocol\": %d, \"n_replica\": %d, "
        "\"whole\": %d, \"seed\": %llu, "
        "\"status\": %d, \"log_ratio\": %s, \"delta_S2\": %s, \"delta_S2_err\": %s, "
        "\"submit_s\": %.6f, \"start_s\": %.6f, \"done_s\": %.6f, \"latency_s\": %.6f, "
        "\"spin_updates\": %lld, \"spin_updates_per_s\": %s}",
        (unsigned long long)job_id, p->d, p->L, p->L_t, p->beta, p->l, p->n_step, p->n_sweep,
        p->n_therm, p->n_traj, p->direction, p->update, p->therm_update, p->protocol,
        nrep_of(*p), p->whole,
        (unsigned long long)p->seed, r->status, lr, ds, de, r->submit_s, r->start_s, r->done_s,
        latency, r->updates, rate);
    if (len < 0 || (size_t)len >= n) return ISING_ERR_ARG;
    return len;
}

// --------------------------------------------------- cancellation, resume --
int ising_cancel(ising_ctx* ctx)
{
    if (!ctx) return ISING_ERR_ARG;
    ctx->cancel.store(1);
    return ISING_OK;
}

int ising_cancel_reset(ising_ctx* ctx)
{
    if (!ctx) return ISING_ERR_ARG;
    ctx->cancel.store(0);
    return ISING_OK;
}

int jarzynski_run_resumable(ising_ctx* ctx, const jz_params* p, int steps_per_segment,
                            int max_segments, int* k_done, int64_t* work_io, int8_t* spins_io)
{
    if (!ctx || !p || !k_done || !work_io || !spins_io || steps_per_segment < 1 ||
        max_segments < 0)
        return ISING_ERR_ARG;
    int rc = check_params(p);
    if (rc) return rc;
    if (*k_done < 0 || *k_done > p->n_step) return ISING_ERR_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ISING_ERR_CUDA;
    cudaEvent_t ev[2];
    if (cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming) != cudaSuccess) return ISING_ERR_CUDA;
    if (cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return ISING_ERR_CUDA;
    }
    int k = *k_done, segs = 0, prev_end = *k_done;
    rc = ISING_OK;
    while (k < p->n_step) {
        if (max_segments > 0 && segs >= max_segments) {
            rc = ISING_ERR_PENDING;
            break;
        }
        if (ctx->cancel.load()) {
            rc = ISING_ERR_CANCELLED;
            break;
        }
        const int k_end = k + steps_per_segment < p->n_step ? k + steps_per_segment : p->n_step;
        if ((rc = jarzynski_run_segment(ctx, p, k, k_end, work_io, spins_io))) break;
        if ((rc = cuda_err(cudaEventRecord(ev[segs & 1], ctx->stream)))) break;
        // at most two segments in flight: wait for the one before this one
        if (segs > 0) {
            if ((rc = cuda_err(cudaEventSynchronize(ev[(segs - 1) & 1])))) break;
            *k_done = prev_end;
        }
        prev_end = k_end;
        k = k_end;
        ++segs;
    }
    // segments run in stream order: once the stream is idle every enqueued one is done
    const int sync = cuda_err(cudaStreamSynchronize(ctx->stream));
    if (sync == ISING_OK && rc != ISING_ERR_CUDA) *k_done = k;
    if (rc == ISING_OK) rc = sync;
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    return rc;
}

}  // extern "C"
