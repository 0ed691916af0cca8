// jz_kernels.cu -- the per-trajectory launch of the Jarzynski replica-gluing
// method (one CTA per trajectory, see jz_traj.cuh) and the FP64 estimator.
#include <cstdint>

#include "jz_device.cuh"
#include "jz_traj.cuh"

namespace jz {

// Finds the job owning CTA b: the last j with jobs[j].cta0 <= b.
__device__ __forceinline__ int find_job(const JobDesc* __restrict__ jobs, int n_jobs, long long b)
{
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&jobs[mid].cta0) <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

constexpr int kMaxTeams = 64;

// One CTA runs `teams` trajectories of the job that owns it (sh.teams per
// CTA; warp teams sync with __syncwarp, a CTA team with __syncthreads).  The
// lattices live in shared memory, or, when they do not fit there (gS !=
// nullptr), in this CTA's own slice of an HBM buffer (L1/L2-cached).  HBM
// is a compile-time choice so that the shared-memory variant keeps 32-bit
// shared addressing.  The specialised variants (CW > 0) are capped at 64
// registers so that two 512-thread CTAs fit on an SM; the generic variant
// keeps the full register file of one CTA, and so does the 2D GW = 1 variant,
// whose one-row pipeline holds the next half-sweep's Philox blocks.
template <int D, bool FAST, int CW, int CLY, bool WARP, bool HBM, int CLT = 0, int CTS = 0>
__global__ void __launch_bounds__(512, (CW > 1 || (CW == 1 && D == 3)) ? 2 : 1)
traj_kernel(const Geom g, const PhiloxKeys K, const JobDesc* __restrict__ jobs, int n_jobs,
            const LaunchShape sh, uint32_t* __restrict__ gS)
{
    extern __shared__ uint32_t S_shared[];
    uint32_t* S = HBM ? gS + (size_t)blockIdx.x * sh.teams * (2 * g.NR * g.GW) : S_shared;
    __shared__ int s_work[kMaxTeams];
    __shared__ uint32_t s_tab[8];

    const int j = find_job(jobs, n_jobs, (long long)blockIdx.x);
    const JobDesc& J = jobs[j];
    const TeamJob tj = team_job(J, g.Ly);
    const long long cta_local = (long long)blockIdx.x - __ldg(&J.cta0);
    int team, tid;
    team_of(sh, &team, &tid);
    const long long local = cta_local * sh.teams + (team < 0 ? 0 : team);
    const bool has = team >= 0 && local < __ldg(&J.n_traj);
    if (!has) tid = -1;
    const int tm = team < 0 ? 0 : team;
    uint32_t* St = S + (size_t)tm * (2 * g.NR * g.GW);
    if (threadIdx.x < 8) s_tab[threadIdx.x] = threadIdx.x < D ? __ldg(&J.tb[threadIdx.x]) : 0u;
    if (threadIdx.x < kMaxTeams) s_work[threadIdx.x] = 0;
    __syncthreads();
    const long long traj = __ldg(&J.traj0) + local;
    const long long V = (long long)g.nrep * g.Lt * g.Ly * g.L;
    const int8_t* sin = (has && (tj.k_begin > 0 || tj.start_in)) ? J.spins_in + local * V : nullptr;
    int dE;
    // The one-row pipeline is compiled into the 2D GW = 1 variant (L <= 16),
    // the only lattice whose warp team can hold a thread per word.
    constexpr bool kRow = D == 2 && CW == 1 && WARP;
    if (kRow && sh.team_threads == g.NR * g.GW)
        dE = run_trajectory<D, FAST, CW, CLY, kRow>(g, K, tj, traj, St, s_tab, tid,
                                                    sh.team_threads, WarpBarrier{}, sin);
    else if (WARP)
        dE = run_trajectory<D, FAST, CW, CLY, false, CLT, CTS>(g, K, tj, traj, St, s_tab, tid,
                                                               sh.team_threads, WarpBarrier{}, sin);
    else
        dE = run_trajectory<D, FAST, CW, CLY>(g, K, tj, traj, St, s_tab, tid, sh.team_threads,
                                              CtaBarrier{}, sin);
    if (has && dE != 0) atomicAdd(&s_work[tm], dE);
    __syncthreads();
    if (has && tid == 0)
        J.w_out[local] = (tj.k_begin > 0 ? J.w_in[local] : 0) +
                         (long long)(tj.dir > 0 ? s_work[tm] : -s_work[tm]) *
                             (tj.prot == 2 ? g.Ly : 1);
    int8_t* sp = J.spins_out;
    if (has && sp != nullptr) export_spins<D>(g, St, sp + local * V, tid, sh.team_threads);
}

// ---------------------------------------------------------------- estimator --
// One CTA: ln <e^-W> with W_i = scale * w_int[i] as a max-shifted log-sum-exp
// per jackknife block, then the full and leave-one-block-out estimates
// (Appendix A, eq. Jarzynski_theorem; blocked jackknife).
// out[0] = ln <e^-W>, out[1] = Delta S_2, out[2] = jackknife error.
constexpr int kMaxJackBlocks = 64;

__global__ void __launch_bounds__(1024)
estimator_kernel(const long long* __restrict__ w_int, int n, double scale, int direction,
                 int n_blocks, double* __restrict__ out)
{
    __shared__ double s_max[kMaxJackBlocks], s_sum[kMaxJackBlocks];
    __shared__ int s_lo[kMaxJackBlocks + 1];
    __shared__ double s_theta[kMaxJackBlocks + 1];
    const int B = n_blocks;
    const int size = n / B;
    if (threadIdx.x <= B) s_lo[threadIdx.x] = threadIdx.x == B ? n : threadIdx.x * size;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_warps = blockDim.x >> 5;
    for (int b = warp; b < B; b += n_warps) {
        const int lo = s_lo[b], hi = s_lo[b + 1];
        double m = -INFINITY;
        for (int i = lo + lane; i < hi; i += 32) m = fmax(m, -scale * (double)w_int[i]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
        double acc = 0.0;
        for (int i = lo + lane; i < hi; i += 32) acc += exp(-scale * (double)w_int[i] - m);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        if (lane == 0) { s_max[b] = m; s_sum[b] = acc; }
    }
    __syncthreads();
    estimator_finish(s_max, s_sum, s_lo, B, n, direction, s_theta, out);
}

// ------------------------------------------------------------ host launchers --
size_t traj_smem_bytes(const Geom& g) { return (size_t)2 * g.NR * g.GW * sizeof(uint32_t); }

using TrajFn = void (*)(const Geom, const PhiloxKeys, const JobDesc*, int, const LaunchShape,
                       uint32_t*);

template <int D, bool FAST, int CW, int CLY, int CLT = 0, int CTS = 0>
static TrajFn pick_traj(const LaunchShape& sh, bool hbm)
{
    return hbm ? (sh.warp ? traj_kernel<D, FAST, CW, CLY, true, true>
                          : traj_kernel<D, FAST, CW, CLY, false, true>)
               : (sh.warp ? traj_kernel<D, FAST, CW, CLY, true, false, CLT, CTS>
                          : traj_kernel<D, FAST, CW, CLY, false, false>);
}

// Shapes with compile-time row geometry: 2D L = 16 and 64 (GW = 1, 4) and 3D
// L = 16 (GW = 1, L_y = 16); the 2D L = L_t = 64 warp teams (eight time slices
// per thread) also fix L_t and the slice step.  Every other shape runs the
// generic instantiation.
static TrajFn select_traj(int D, const Geom& g, const LaunchShape& sh, bool hbm)
{
    const bool fast = (g.Lh % 8) == 0;
    if (D == 2) {
        if (fast && g.GW == 4 && g.Lt == 64 && sh.warp && sh.team_threads == 32 && !hbm)
            return pick_traj<2, true, 4, 1, 64, 8>(sh, hbm);
        if (fast && g.GW == 4) return pick_traj<2, true, 4, 1>(sh, hbm);
        if (fast && g.GW == 1) return pick_traj<2, true, 1, 1>(sh, hbm);
        return fast ? pick_traj<2, true, 0, 0>(sh, hbm) : pick_traj<2, false, 0, 0>(sh, hbm);
    }
    if (fast && g.GW == 1 && g.Ly == 16) return pick_traj<3, true, 1, 16>(sh, hbm);
    return fast ? pick_traj<3, true, 0, 0>(sh, hbm) : pick_traj<3, false, 0, 0>(sh, hbm);
}

// Lets kern take up to the per-CTA maximum of dynamic shared memory.  The
// attribute is raised once to that maximum, never lowered, so that launches
// and occupancy queries of the same kernel from several host threads with
// different lattice sizes cannot narrow it under one another.
static cudaError_t open_smem(TrajFn kern)
{
    cudaFuncAttributes fa;
    int dev = 0, optin = 0;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const int max_dyn = optin - (int)fa.sharedSizeBytes;
    if (fa.maxDynamicSharedSizeBytes >= max_dyn) return cudaSuccess;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn);
}

cudaError_t launch_traj(int D, const Geom& g, const PhiloxKeys& K, const JobDesc* jobs,
                        int n_jobs, long long n_cta, const LaunchShape& sh, cudaStream_t st,
                        uint32_t* gS)
{
    const size_t smem = gS ? 0 : traj_smem_bytes(g) * sh.teams;
    const TrajFn kern = select_traj(D, g, sh, gS != nullptr);
    const cudaError_t e = open_smem(kern);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)n_cta, sh.cta_threads, smem, st>>>(g, K, jobs, n_jobs, sh, gS);
    return cudaGetLastError();
}

cudaError_t traj_occupancy(int D, const Geom& g, const LaunchShape& sh, int* ctas_per_sm)
{
    const TrajFn kern = select_traj(D, g, sh, false);
    const cudaError_t e = open_smem(kern);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, kern, sh.cta_threads,
                                                         traj_smem_bytes(g) * sh.teams);
}

cudaError_t bounds_status_traj(unsigned int out[2], bool clear)
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

cudaError_t launch_estimator(const long long* w_int, int n, double scale, int direction,
                             int n_blocks, double* out, cudaStream_t st)
{
    estimator_kernel<<<1, 1024, 0, st>>>(w_int, n, scale, direction, n_blocks, out);
    return cudaGetLastError();
}

}  // namespace jz
