// jz_records.cpp -- the library's host-only records, plain C++ with no CUDA
// (none has a counterpart in the paper): the persisted autotune cache (JSON
// file keyed by GPU name, d, L, L_t, n and the log2 trajectory bucket) and the
// per-job JSON line of the server.  Kept free of the CUDA runtime so that it
// also builds, for tests, with host sanitizers.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <tuple>

#include "../../include/isingjz.h"

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
// backslashes (device names have none; anything else becomes '_'), at most
// kMaxName characters, the longest name the loader reads back.
constexpr size_t kMaxName = 255;
std::string clean_name(const char* s)
{
    std::string out;
    for (; s && *s && out.size() < kMaxName; ++s) {
        const char c = *s;
        out += (c >= 32 && c < 127 && c != '"' && c != '\\') ? c : '_';
    }
    return out;
}
}  // namespace

// One cache line as jz_tune_cache_save writes it:
// {"gpu": "<name>", "d": D, "L": L, "L_t": T, "n_replica": N, "traj_bucket": B,
//  "cta_threads": C} with an optional trailing comma.  Names may be empty;
// every number must be a decimal integer within [0, 2^31).  False on any
// other text.
bool parse_line(const char* line, std::string* gpu, int v[6])
{
    static const char* const keys[6] = {"\"d\": ", "\"L\": ", "\"L_t\": ", "\"n_replica\": ",
                                        "\"traj_bucket\": ", "\"cta_threads\": "};
    const char* s = line;
    auto lit = [&s](const char* w) {
        const size_t n = std::strlen(w);
        if (std::strncmp(s, w, n) != 0) return false;
        s += n;
        return true;
    };
    if (!lit("{\"gpu\": \"")) return false;
    const char* q = std::strchr(s, '"');
    if (!q || (size_t)(q - s) > kMaxName) return false;
    gpu->assign(s, (size_t)(q - s));
    s = q + 1;
    for (int i = 0; i < 6; ++i) {
        if (!lit(", ") || !lit(keys[i])) return false;
        long long x = 0;
        int digits = 0;
        for (; *s >= '0' && *s <= '9' && digits < 10; ++s, ++digits) x = 10 * x + (*s - '0');
        if (digits == 0 || (*s >= '0' && *s <= '9') || x > 0x7FFFFFFFLL) return false;
        v[i] = (int)x;
    }
    if (!lit("}")) return false;
    lit(",");
    return std::strcmp(s, "\n") == 0 || *s == '\0';
}

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
        std::string gpu;
        int v[6];
        if (!header || closed || !parse_line(line, &gpu, v) || (v[0] != 2 && v[0] != 3) ||
            v[1] < 2 || v[2] < 2 || v[3] < 2 || v[4] > 40) {
            rc = ISING_ERR_ARG;
            break;
        }
        got[TuneKey(gpu, v[0], v[1], v[2], v[3], v[4])] = v[5];
    }
    std::fclose(f);
    if (rc == ISING_OK && (!header || !closed)) rc = ISING_ERR_ARG;
    if (rc == ISING_OK)
        for (const auto& e : got) c->entries[e.first] = e.second;
    return rc;
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
    char beta[32], lr[32], ds[32], de[32], rate[32];
    num(p->beta, beta, sizeof beta);
    num(ok ? r->log_ratio : NAN, lr, sizeof lr);
    num(ok ? r->delta_S2 : NAN, ds, sizeof ds);
    num(ok ? r->delta_S2_err : NAN, de, sizeof de);
    num(ok && on_device > 0 ? (double)r->updates / on_device : NAN, rate, sizeof rate);
    const int len = std::snprintf(
        buf, n,
        "{\"job\": %llu, \"d\": %d, \"L\": %d, \"L_t\": %d, \"beta\": %s, \"l\": %d, "
        "\"n_step\": %d, \"n_sweep\": %d, \"n_therm\": %d, \"n_traj\": %d, \"direction\": %d, "
        "\"update\": %d, \"therm_update\": %d, \"protocol\": %d, \"n_replica\": %d, "
        "\"whole\": %d, \"seed\": %llu, "
        "\"status\": %d, \"log_ratio\": %s, \"delta_S2\": %s, \"delta_S2_err\": %s, "
        "\"submit_s\": %.6f, \"start_s\": %.6f, \"done_s\": %.6f, \"latency_s\": %.6f, "
        "\"spin_updates\": %lld, \"spin_updates_per_s\": %s}",
        (unsigned long long)job_id, p->d, p->L, p->L_t, beta, p->l, p->n_step, p->n_sweep,
        p->n_therm, p->n_traj, p->direction, p->update, p->therm_update, p->protocol,
        p->n_replica == 0 ? 2 : p->n_replica, p->whole,
        (unsigned long long)p->seed, r->status, lr, ds, de, r->submit_s, r->start_s, r->done_s,
        latency, r->updates, rate);
    if (len < 0 || (size_t)len >= n) return ISING_ERR_ARG;
    return len;
}

// --------------------------------------------------- cancellation, resume --
}  // extern "C"
