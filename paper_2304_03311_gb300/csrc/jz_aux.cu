// jz_aux.cu -- host-side services around the replica-gluing kernels (none has
// a counterpart in the paper): the autotuner backed by the persisted cache,
// cancellation and resumable runs.  The cache itself and the per-job JSON
// line are plain C++ in jz_records.cpp.
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

extern "C" {

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
