// jz_serve.cu -- continuous-batching server for c-function jobs.
//
// One host worker thread owns the device side.  It admits queued jobs in
// arrival order while a stream slot is free and the job's device memory fits
// the budget, launches each admitted job on its slot's stream (the job's
// trajectories, then its estimator, then the copies of the results into
// pinned host memory), and polls the slots' completion events; a finished slot
// immediately takes the next queued job, so jobs arriving while others run are
// overlapped on the device.  Device memory is allocated stream-ordered
// (cudaMallocAsync / cudaFreeAsync on the slot's stream), so admitting and
// retiring jobs never synchronises the device.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "jz_host.h"

using namespace jzh;

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    jz_params p{};
    size_t need = 0;          // device bytes while running
    bool done = false;
    bool cancel = false;      // jz_cancel on a running job: discard its results
    jz_result res{};
    std::vector<int64_t> work;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    uint64_t job = 0;
    std::vector<uint32_t> tcut;        // host table build area
    uint32_t* h_tcut = nullptr;        // pinned staging
    size_t h_tcut_cap = 0;             // words
    jz::JobDesc* h_desc = nullptr;     // pinned descriptors: the job's, then its
    size_t h_desc_cap = 0;             // thermalisation launches' (capacity)
    double* h_est = nullptr;           // pinned, 3 doubles
    int64_t* h_work = nullptr;         // pinned
    size_t h_work_cap = 0;             // entries
};

// Threshold words of a job: per step 8d switched-site thresholds (Metropolis)
// or the two switched bond thresholds (Swendsen-Wang).
size_t tcut_words(const jz_params& p)
{
    return (size_t)p.n_step * (p.update == 1 ? 2 : 8 * p.d);
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// A job's device memory, in order (byte offsets, 256-byte aligned): its
// thresholds, its job descriptors (its own, then one per thermalisation
// launch), W_int, the estimator's output, and for therm_update = 1 the
// thermalised spins (n_traj V bytes) and, when the Swendsen-Wang state does
// not fit shared memory, the HBM slices of one thermalisation chunk (one
// resident wave of trajectories, wave[d - 2]).
struct JobMem {
    size_t desc = 0, work = 0, est = 0, spins = 0, lattice = 0, total = 0;
    long long chunk = 0;      // trajectories per thermalisation launch (0: none)
    size_t n_desc = 1;
    bool therm_hbm = false;
};

JobMem job_mem(const jz_params& p, const long long wave[2])
{
    JobMem m;
    const jz::Geom g = make_geom(p.d, p.L, p.L_t, nrep_of(p));
    const size_t V = (size_t)g.nrep * g.Lt * g.Ly * g.L;
    const bool hybrid = sw_therm(p);
    m.therm_hbm = hybrid && !sw_fits(g);
    if (hybrid) {
        m.chunk = m.therm_hbm ? std::min<long long>(p.n_traj, wave[p.d - 2]) : p.n_traj;
        m.n_desc = 1 + (size_t)((p.n_traj + m.chunk - 1) / m.chunk);
    }
    size_t o = round256(tcut_words(p) * sizeof(uint32_t));
    m.desc = o;
    o += round256(m.n_desc * sizeof(jz::JobDesc));
    m.work = o;
    o += round256((size_t)p.n_traj * sizeof(int64_t));
    m.est = o;
    o += 256;
    m.spins = o;
    o += hybrid ? round256((size_t)p.n_traj * V) : 0;
    m.lattice = o;
    o += m.therm_hbm ? (size_t)m.chunk * jz::sw_smem_bytes(g) : 0;
    m.total = o;
    return m;
}

int grow_pinned(void** p, size_t* cap, size_t want, size_t elem)
{
    if (want <= *cap) return ISING_OK;
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMallocHost(p, want * elem) != cudaSuccess) {
        cudaGetLastError();
        return ISING_ERR_NOMEM;
    }
    *cap = want;
    return ISING_OK;
}

}  // namespace

struct jz_server {
    ising_ctx* ctx = nullptr;
    size_t budget = 0, used = 0;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::map<uint64_t, std::unique_ptr<Job>> jobs;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread worker;
    Clock::time_point t0;
    long long wave[2] = {1, 1};   // resident HBM Swendsen-Wang CTAs on the device, 2D and 3D
    FILE* log = nullptr;      // jz_server_set_log: one JSON line per finished job

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
    void run();
    int launch(Slot& s, Job& j);
    void finish(uint64_t id, Job& j);
};

// Marks a job finished (lock held): wakes its waiters and logs its line.
void jz_server::finish(uint64_t id, Job& j)
{
    j.done = true;
    if (log) {
        char line[1024];
        if (jz_result_json(id, &j.p, &j.res, line, sizeof line) > 0) {
            std::fputs(line, log);
            std::fputc('\n', log);
            std::fflush(log);
        }
    }
    cv_done.notify_all();
}

// The thermalisation launches of a job (none without therm_update = 1), on
// its slot's stream: descriptors 1 .. n_desc - 1, one chunk each.
int therm_launches(const jz_params& p, const jz::Geom& g, const jz::PhiloxKeys& K,
                   const jz::JobDesc* d_desc, const JobMem& m, uint32_t* d_lat, const Slot& s)
{
    for (size_t c = 1; c < m.n_desc; ++c) {
        const int rc = cuda_err(jz::launch_sw(p.d, g, K, d_desc + c, 1, s.h_desc[c].n_traj,
                                              s.stream, d_lat));
        if (rc) return rc;
    }
    return ISING_OK;
}

// Enqueues one job on its slot's stream.  Called without the lock; the job
// record is stable (held by unique_ptr) and not touched by other threads
// while it is running.
int jz_server::launch(Slot& s, Job& j)
{
    const jz_params& p = j.p;
    const jz::Geom g = make_geom(p.d, p.L, p.L_t, nrep_of(p));
    const size_t n_tcut = tcut_words(p);
    int rc;
    const JobMem m = job_mem(p, wave);
    if ((rc = grow_pinned((void**)&s.h_tcut, &s.h_tcut_cap, n_tcut, sizeof(uint32_t))) ||
        (rc = grow_pinned((void**)&s.h_work, &s.h_work_cap, (size_t)p.n_traj, sizeof(int64_t))) ||
        (rc = grow_pinned((void**)&s.h_desc, &s.h_desc_cap, m.n_desc, sizeof(jz::JobDesc))))
        return rc;
    s.tcut.assign(n_tcut, 0);
    jz::JobDesc& J = *s.h_desc;
    std::memset(&J, 0, sizeof J);
    if (p.update == 1) build_bond_tables(p, J.tb, s.tcut, 0);
    else build_tables(p, J.tb, s.tcut, 0);
    std::memcpy(s.h_tcut, s.tcut.data(), n_tcut * sizeof(uint32_t));
    char* d = nullptr;
    if ((rc = cuda_err(cudaMallocAsync((void**)&d, j.need, s.stream)))) return rc;
    uint32_t* d_tcut = (uint32_t*)d;
    jz::JobDesc* d_desc = (jz::JobDesc*)(d + m.desc);
    long long* d_work = (long long*)(d + m.work);
    double* d_est = (double*)(d + m.est);
    int8_t* d_spins = (int8_t*)(d + m.spins);
    uint32_t* d_lat = m.therm_hbm ? (uint32_t*)(d + m.lattice) : nullptr;
    const bool hybrid = sw_therm(p);
    const long long V = (long long)g.nrep * g.Lt * g.Ly * g.L;
    J.l = p.l;
    J.n_step = p.n_step;
    J.n_sweep = p.n_sweep;
    J.n_therm = p.n_therm;
    J.dir = p.direction;
    J.prot = p.protocol == 2 ? 2 : 1;
    cut_range(p, &J.g0, &J.g1);
    J.k_begin = 0;
    J.k_end = p.n_step;
    J.n_traj = p.n_traj;
    J.traj0 = p.traj0;
    J.cta0 = 0;
    J.tcut = d_tcut;
    J.w_out = d_work;
    J.spins_out = nullptr;
    if (hybrid) {
        // Swendsen-Wang thermalisation (no protocol steps) into d_spins, one
        // launch per chunk of trajectories, from which the Metropolis
        // protocol starts
        jz::JobDesc T = J;
        std::vector<uint32_t> bt((size_t)2 * p.n_step);
        build_bond_tables(p, T.tb, bt, 0);
        T.k_end = 0;
        for (size_t c = 1; c < m.n_desc; ++c) {
            const long long off = (long long)(c - 1) * m.chunk;
            jz::JobDesc& C = s.h_desc[c];
            C = T;
            C.n_traj = (int)std::min<long long>(m.chunk, p.n_traj - off);
            C.traj0 = T.traj0 + off;
            C.w_out = d_work + off;
            C.spins_out = d_spins + off * V;
        }
        J.start_in = 1;
        J.spins_in = d_spins;
    }
    const jz::PhiloxKeys K = key_schedule(p.seed);
    const jz::LaunchShape sh = p.update == 1 ? shape_for(g, 0) : ctx_shape(ctx, p.d, g, p.n_traj);
    const int B = p.n_traj < 32 ? p.n_traj : 32;
    if ((rc = cuda_err(cudaMemcpyAsync(d_tcut, s.h_tcut, n_tcut * sizeof(uint32_t),
                                       cudaMemcpyHostToDevice, s.stream))) ||
        (rc = cuda_err(cudaMemcpyAsync(d_desc, s.h_desc, m.n_desc * sizeof(jz::JobDesc),
                                       cudaMemcpyHostToDevice, s.stream))) ||
        (rc = therm_launches(p, g, K, d_desc, m, d_lat, s)) ||
        (rc = cuda_err(p.update == 1   // Swendsen-Wang: one trajectory per CTA
                           ? jz::launch_sw(p.d, g, K, d_desc, 1, p.n_traj, s.stream)
                           : jz::launch_traj(p.d, g, K, d_desc, 1,
                                             (p.n_traj + sh.teams - 1) / sh.teams, sh,
                                             s.stream))) ||
        (rc = cuda_err(jz::launch_estimator(d_work, p.n_traj, p.beta / (double)p.n_step,
                                            p.direction, B, d_est, s.stream))) ||
        (rc = cuda_err(cudaMemcpyAsync(s.h_est, d_est, 3 * sizeof(double),
                                       cudaMemcpyDeviceToHost, s.stream))) ||
        (rc = cuda_err(cudaMemcpyAsync(s.h_work, d_work, (size_t)p.n_traj * sizeof(int64_t),
                                       cudaMemcpyDeviceToHost, s.stream)))) {
        cudaFreeAsync(d, s.stream);
        return rc;
    }
    cudaFreeAsync(d, s.stream);
    return cuda_err(cudaEventRecord(s.done, s.stream));
}

void jz_server::run()
{
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        bool any_busy = false;
        // retire finished jobs
        for (Slot& s : slots) {
            if (!s.busy) continue;
            const cudaError_t e = cudaEventQuery(s.done);
            if (e == cudaErrorNotReady) {
                any_busy = true;
                continue;
            }
            Job& j = *jobs[s.job];
            const Range nv("jz retire");
            if (e == cudaSuccess && j.cancel) {
                j.res.status = ISING_ERR_CANCELLED;
            } else if (e == cudaSuccess) {
                j.res.status = ISING_OK;
                j.res.log_ratio = s.h_est[0];
                j.res.delta_S2 = s.h_est[1];
                j.res.delta_S2_err = s.h_est[2];
                j.work.assign(s.h_work, s.h_work + j.p.n_traj);
            } else {
                cudaGetLastError();
                j.res.status = ISING_ERR_CUDA;
            }
            j.res.done_s = now();
            used -= j.need;
            s.busy = false;
            finish(s.job, j);
        }
        // admit in arrival order while a slot and the budget allow
        while (!queue.empty() && !stop) {
            const uint64_t head = queue.front();
            Job& j = *jobs[head];
            if (j.need > budget) {
                j.res.status = ISING_ERR_NOMEM;
                j.res.start_s = j.res.done_s = now();
                queue.pop_front();
                finish(head, j);
                continue;
            }
            Slot* free_slot = nullptr;
            for (Slot& s : slots)
                if (!s.busy) {
                    free_slot = &s;
                    break;
                }
            if (!free_slot || used + j.need > budget) break;
            const uint64_t id = queue.front();
            queue.pop_front();
            used += j.need;
            free_slot->busy = true;
            free_slot->job = id;
            j.res.start_s = now();
            lk.unlock();
            int rc;
            {
                const Range nv("jz admit");
                rc = launch(*free_slot, j);
            }
            lk.lock();
            if (rc) {
                cudaStreamSynchronize(free_slot->stream);
                cudaGetLastError();
                j.res.status = rc;
                j.res.done_s = now();
                used -= j.need;
                free_slot->busy = false;
                finish(id, j);
            } else {
                any_busy = true;
            }
        }
        if (stop && !any_busy) break;
        if (any_busy)
            cv_work.wait_for(lk, std::chrono::microseconds(50));
        else
            cv_work.wait(lk, [&] { return stop || !queue.empty(); });
    }
}

extern "C" {

int jz_server_create(ising_ctx* ctx, size_t hbm_budget_bytes, int max_inflight, jz_server** out)
{
    if (!ctx || !out || hbm_budget_bytes == 0 || max_inflight < 1 || max_inflight > 64)
        return ISING_ERR_ARG;
    *out = nullptr;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ISING_ERR_CUDA;
    std::unique_ptr<jz_server> s(new (std::nothrow) jz_server());
    if (!s) return ISING_ERR_NOMEM;
    s->ctx = ctx;
    s->budget = hbm_budget_bytes;
    s->slots.resize(max_inflight);
    for (Slot& sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            grow_pinned((void**)&sl.h_desc, &sl.h_desc_cap, 2, sizeof(jz::JobDesc)) != ISING_OK ||
            cudaMallocHost((void**)&sl.h_est, 4 * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            for (Slot& t : s->slots) {
                if (t.stream) cudaStreamDestroy(t.stream);
                if (t.done) cudaEventDestroy(t.done);
                if (t.h_desc) cudaFreeHost(t.h_desc);
                if (t.h_est) cudaFreeHost(t.h_est);
            }
            return ISING_ERR_CUDA;
        }
    }
    s->t0 = Clock::now();
    s->wave[0] = jz::sw_hbm_wave(2);
    s->wave[1] = jz::sw_hbm_wave(3);
    jz_server* raw = s.release();
    raw->worker = std::thread([raw] { raw->run(); });
    *out = raw;
    return ISING_OK;
}

int jz_submit(jz_server* s, const jz_params* p, uint64_t* job_id)
{
    if (!s || !p || !job_id) return ISING_ERR_ARG;
    int rc = check_params(p);
    if (rc) return rc;
    const jz::Geom g = make_geom(p->d, p->L, p->L_t, nrep_of(*p));
    if (p->update == 1 ? !sw_fits(g) : !shape_fits(g)) return ISING_ERR_UNSUPPORTED;
    std::unique_ptr<Job> j(new (std::nothrow) Job());
    if (!j) return ISING_ERR_NOMEM;
    j->p = *p;
    j->need = job_mem(*p, s->wave).total;
    j->res.status = ISING_ERR_PENDING;
    j->res.updates = (long long)p->n_traj * ((long long)g.nrep * p->L_t * g.Ly * p->L) *
                     ((long long)p->n_therm + (long long)p->n_step * p->n_sweep);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return ISING_ERR_ARG;
        const uint64_t id = s->next_id++;
        j->res.submit_s = s->now();
        s->jobs[id] = std::move(j);
        s->queue.push_back(id);
        *job_id = id;
    }
    s->cv_work.notify_one();
    return ISING_OK;
}

int jz_poll(jz_server* s, uint64_t job_id, jz_result* out)
{
    if (!s || !out) return ISING_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return ISING_ERR_NOT_FOUND;
    if (!it->second->done) return ISING_ERR_PENDING;
    *out = it->second->res;
    return ISING_OK;
}

int jz_wait(jz_server* s, uint64_t job_id, double timeout_s, jz_result* out)
{
    if (!s || !out || !(timeout_s >= 0)) return ISING_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return ISING_ERR_NOT_FOUND;
    Job* j = it->second.get();
    const auto limit = std::chrono::duration<double>(timeout_s);
    if (!s->cv_done.wait_for(lk, std::chrono::duration_cast<Clock::duration>(limit),
                             [&] { return j->done; }))
        return ISING_ERR_TIMEOUT;
    *out = j->res;
    return ISING_OK;
}

int jz_server_work(jz_server* s, uint64_t job_id, int64_t* work_out)
{
    if (!s || !work_out) return ISING_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return ISING_ERR_NOT_FOUND;
    if (!it->second->done) return ISING_ERR_PENDING;
    if (it->second->res.status != ISING_OK) return it->second->res.status;
    std::memcpy(work_out, it->second->work.data(), it->second->work.size() * sizeof(int64_t));
    return ISING_OK;
}

int jz_cancel(jz_server* s, uint64_t job_id)
{
    if (!s) return ISING_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return ISING_ERR_NOT_FOUND;
    Job& j = *it->second;
    if (j.done) return ISING_OK;   // a finished job keeps its result
    for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
        if (*q == job_id) {       // still queued: dropped before admission
            s->queue.erase(q);
            j.res.status = ISING_ERR_CANCELLED;
            j.res.start_s = j.res.done_s = s->now();
            s->finish(job_id, j);
            return ISING_OK;
        }
    j.cancel = true;               // on the device: runs to its end, results discarded
    return ISING_OK;
}

int jz_server_set_log(jz_server* s, const char* path)
{
    if (!s) return ISING_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->log) std::fclose(s->log);
    s->log = nullptr;
    if (!path) return ISING_OK;
    s->log = std::fopen(path, "a");
    return s->log ? ISING_OK : ISING_ERR_NOT_FOUND;
}

void jz_server_free(jz_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        // queued jobs are dropped: their waiters see ISING_ERR_CANCELLED
        for (uint64_t id : s->queue) {
            Job& j = *s->jobs[id];
            j.res.status = ISING_ERR_CANCELLED;
            j.res.start_s = j.res.done_s = s->now();
            s->finish(id, j);
        }
        s->queue.clear();
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->ctx->device);
    for (Slot& t : s->slots) {
        cudaStreamSynchronize(t.stream);
        cudaStreamDestroy(t.stream);
        cudaEventDestroy(t.done);
        if (t.h_desc) cudaFreeHost(t.h_desc);
        if (t.h_est) cudaFreeHost(t.h_est);
        if (t.h_tcut) cudaFreeHost(t.h_tcut);
        if (t.h_work) cudaFreeHost(t.h_work);
    }
    if (s->log) std::fclose(s->log);
    delete s;
}

}  // extern "C"
