// jz_batch.cu -- uneven batches in one persistent launch, and the batched
// FP64 estimator.
//
// persistent_kernel: a grid sized to the GPU's resident capacity; each CTA
// repeatedly takes the next work item from a device counter.  An item is
// (job, first trajectory): the CTA splits into `teams` teams of the job's
// team size and each team runs one whole trajectory of that job (jz_traj.cuh)
// on its own slice of shared memory.  Items are ordered by cost, largest
// first, so the long trajectories start early and the tail is short.  Jobs
// of every lattice shape (2D and 3D, any L, L_t) share the launch.
#include <cstdint>

#include "jz_device.cuh"
#include "jz_traj.cuh"

namespace jz {

constexpr int kMaxTeams = 64;

template <int D, bool FAST, class Bar>
__device__ __forceinline__ void run_item(const BatchJob& B, const PhiloxKeys& K, int traj_lo,
                                         uint32_t* S, const uint32_t* tab, int* s_work, Bar bar)
{
    const TeamJob tj = team_job(B.J, B.g.Ly);
    int team, tid;
    team_of(B.sh, &team, &tid);
    if (!B.sh.warp && tid >= B.sh.team_threads) team = -1;   // CTA larger than the team
    const int n_here = min(B.sh.teams, B.J.n_traj - traj_lo);
    const bool has = team >= 0 && team < n_here;
    if (!has) tid = -1;
    const int tm = has ? team : 0;
    uint32_t* St = S + (size_t)tm * B.lattice_words;
    const long long local = (long long)traj_lo + tm;
    const long long V = (long long)B.g.nrep * B.g.Lt * B.g.Ly * B.g.L;
    // therm_update = 1: the job starts from its thermalised spins
    const int8_t* sin = (has && tj.start_in) ? B.J.spins_in + local * V : nullptr;
    const int dE = run_trajectory<D, FAST, 0, 0>(B.g, K, tj, B.J.traj0 + local, St, tab, tid,
                                                 B.sh.team_threads, bar, sin);
    if (has && dE != 0) atomicAdd(&s_work[tm], dE);
    __syncthreads();
    if (has && tid == 0)
        B.J.w_out[local] = (long long)(tj.dir > 0 ? s_work[tm] : -s_work[tm]) *
                           (tj.prot == 2 ? B.g.Ly : 1);
    if (has && B.J.spins_out != nullptr)
        export_spins<D>(B.g, St,
                        B.J.spins_out + local * (long long)(B.g.nrep * B.g.Lt * B.g.Ly * B.g.L),
                        tid, B.sh.team_threads);
}

template <int D, bool FAST>
__device__ __forceinline__ void run_item_any(const BatchJob& B, const PhiloxKeys& K, int traj_lo,
                                             uint32_t* S, const uint32_t* tab, int* s_work)
{
    if (B.sh.warp) run_item<D, FAST>(B, K, traj_lo, S, tab, s_work, WarpBarrier{});
    else run_item<D, FAST>(B, K, traj_lo, S, tab, s_work, CtaBarrier{});
}

__global__ void __launch_bounds__(512)
persistent_kernel(const BatchJob* __restrict__ jobs, const int2* __restrict__ items, int n_items,
                  unsigned int* __restrict__ counter, const PhiloxKeys K)
{
    extern __shared__ uint32_t S[];
    __shared__ int s_item;
    __shared__ int s_work[kMaxTeams];
    __shared__ uint32_t s_tab[8];
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const int2 item = items[it];
        const BatchJob& B = jobs[item.x];
        if (threadIdx.x < 8)
            s_tab[threadIdx.x] = threadIdx.x < (unsigned)B.D ? B.J.tb[threadIdx.x] : 0u;
        if (threadIdx.x < kMaxTeams) s_work[threadIdx.x] = 0;
        __syncthreads();
        if (B.D == 2) {
            if (B.fast) run_item_any<2, true>(B, K, item.y, S, s_tab, s_work);
            else run_item_any<2, false>(B, K, item.y, S, s_tab, s_work);
        } else {
            if (B.fast) run_item_any<3, true>(B, K, item.y, S, s_tab, s_work);
            else run_item_any<3, false>(B, K, item.y, S, s_tab, s_work);
        }
        __syncthreads();   // shared memory and s_item are reused by the next item
    }
}

// ---------------------------------------------------------- batched estimator --
constexpr int kMaxJackBlocksB = 64;

// One CTA per job: ln <e^-W> as a max-shifted log-sum-exp per jackknife block,
// then the full and leave-one-block-out estimates (Appendix A, eq.
// Jarzynski_theorem).  out[3j + 0] = ln <e^-W>, [3j + 1] = Delta S_2,
// [3j + 2] = jackknife error of Delta S_2.
__global__ void __launch_bounds__(256)
estimator_batch_kernel(const EstJob* __restrict__ jobs, double* __restrict__ out)
{
    __shared__ double s_max[kMaxJackBlocksB], s_sum[kMaxJackBlocksB];
    __shared__ int s_lo[kMaxJackBlocksB + 1];
    __shared__ double s_theta[kMaxJackBlocksB + 1];
    const EstJob E = jobs[blockIdx.x];
    const int B = E.n_blocks, n = E.n;
    const int size = n / B;
    if ((int)threadIdx.x <= B) s_lo[threadIdx.x] = (int)threadIdx.x == B ? n : threadIdx.x * size;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_warps = blockDim.x >> 5;
    for (int b = warp; b < B; b += n_warps) {
        const int lo = s_lo[b], hi = s_lo[b + 1];
        double m = -INFINITY;
        for (int i = lo + lane; i < hi; i += 32) m = fmax(m, -E.scale * (double)E.w[i]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
        double acc = 0.0;
        for (int i = lo + lane; i < hi; i += 32) acc += exp(-E.scale * (double)E.w[i] - m);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        if (lane == 0) { s_max[b] = m; s_sum[b] = acc; }
    }
    __syncthreads();
    estimator_finish(s_max, s_sum, s_lo, B, n, E.direction, s_theta, out + 3 * blockIdx.x);
}

// ------------------------------------------------------------------ launchers --
// The attribute is set to the per-CTA maximum (not this plan's size) so that
// graphs captured for larger plans stay launchable after smaller ones; the
// kernel's static shared memory comes out of the same opt-in limit.
cudaError_t persistent_prepare(size_t smem, int threads, int* blocks_per_sm)
{
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, persistent_kernel);
    if (e != cudaSuccess) return e;
    const int max_dyn = optin - (int)fa.sharedSizeBytes;
    if ((long long)smem > max_dyn) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             max_dyn);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, persistent_kernel,
                                                          threads, smem);
}

cudaError_t launch_persistent(const BatchJob* jobs, const int2* items, int n_items,
                              unsigned int* counter, const PhiloxKeys& K, int grid, int threads,
                              size_t smem, cudaStream_t st)
{
    persistent_kernel<<<grid, threads, smem, st>>>(jobs, items, n_items, counter, K);
    return cudaGetLastError();
}

cudaError_t launch_estimator_batch(const EstJob* jobs, int n_jobs, double* out, cudaStream_t st)
{
    estimator_batch_kernel<<<n_jobs, 256, 0, st>>>(jobs, out);
    return cudaGetLastError();
}

cudaError_t bounds_status_batch(unsigned int out[2], bool clear)
{
#ifdef JZ_BOUNDS_CHECK
    cudaError_t e = cudaMemcpyFromSymbol(out, jz_bounds_status, 2 * sizeof(unsigned int));
    if (e == cudaSuccess && clear) {
        const unsigned int z[2] = {0u, 0u};
        e = cudaMemcpyToSymbol(jz_bounds_status, z, sizeof z);
    }
    return e;
#else
    out[0] = out[1] = 0u;
    (void)clear;
    return cudaSuccess;
#endif
}

}  // namespace jz
