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

struct CtaBarrier {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// One CTA runs one trajectory of the job that owns it; the CTA is the team.
template <int D, bool FAST, int CG, int CLY>
__global__ void __launch_bounds__(512)
traj_kernel(const Geom g, const PhiloxKeys K, const JobDesc* __restrict__ jobs, int n_jobs)
{
    extern __shared__ uint32_t S[];
    __shared__ int s_work;
    __shared__ uint32_t s_tab[8];

    const int j = find_job(jobs, n_jobs, (long long)blockIdx.x);
    const JobDesc& J = jobs[j];
    const TeamJob tj = team_job(J);
    const long long local = (long long)blockIdx.x - __ldg(&J.cta0);
    const long long traj = __ldg(&J.traj0) + local;
    if (threadIdx.x < 8) s_tab[threadIdx.x] = threadIdx.x < D ? __ldg(&J.tb[threadIdx.x]) : 0u;
    if (threadIdx.x == 0) s_work = 0;
    // (the first barrier inside run_trajectory orders these before any use)
    const int dE = run_trajectory<D, FAST, CG, CLY>(g, K, tj, traj, S, s_tab, (int)threadIdx.x,
                                                    (int)blockDim.x, CtaBarrier{});
    // per-trajectory integer work: warp reduction, then one shared atomic per warp
    const int wsum = __reduce_add_sync(0xFFFFFFFFu, dE);
    if ((threadIdx.x & 31) == 0 && wsum != 0) atomicAdd(&s_work, wsum);
    __syncthreads();
    if (threadIdx.x == 0) J.w_out[local] = (long long)(tj.dir > 0 ? s_work : -s_work);
    int8_t* sp = J.spins_out;
    if (sp != nullptr)
        export_spins<D>(g, S, sp + local * (long long)(2 * g.Lt * g.Ly * g.L), (int)threadIdx.x,
                        (int)blockDim.x);
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
    if (threadIdx.x != 0) return;
    const double sign = direction > 0 ? -1.0 : 1.0;
    auto lse_without = [&](int skip, int count) {
        double M = -INFINITY;
        for (int b = 0; b < B; ++b) if (b != skip) M = fmax(M, s_max[b]);
        double tot = 0.0;
        for (int b = 0; b < B; ++b) if (b != skip) tot += s_sum[b] * exp(s_max[b] - M);
        return M + log(tot) - log((double)count);
    };
    const double full = lse_without(-1, n);
    double err = 0.0;
    if (B >= 2) {
        double theta[kMaxJackBlocks];
        double mean = 0.0;
        for (int b = 0; b < B; ++b) {
            theta[b] = sign * lse_without(b, n - (s_lo[b + 1] - s_lo[b]));
            mean += theta[b];
        }
        mean /= B;
        double ss = 0.0;
        for (int b = 0; b < B; ++b) ss += (theta[b] - mean) * (theta[b] - mean);
        err = sqrt((double)(B - 1) / B * ss);
    }
    out[0] = full;
    out[1] = sign * full;
    out[2] = err;
}

// ------------------------------------------------------------ host launchers --
size_t traj_smem_bytes(const Geom& g) { return (size_t)2 * g.NR * g.G * sizeof(uint32_t); }

template <int D, bool FAST, int CG, int CLY>
static cudaError_t launch_traj_t(const Geom& g, const PhiloxKeys& K, const JobDesc* jobs,
                                 int n_jobs, long long n_cta, int threads, cudaStream_t st)
{
    const size_t smem = traj_smem_bytes(g);
    cudaError_t e = cudaFuncSetAttribute(traj_kernel<D, FAST, CG, CLY>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    traj_kernel<D, FAST, CG, CLY><<<(unsigned)n_cta, threads, smem, st>>>(g, K, jobs, n_jobs);
    return cudaGetLastError();
}

// Shapes with compile-time row geometry: 2D L = 16 and 64 (G = 2, 8) and 3D
// L = 16 (G = 2, L_y = 16); every other shape runs the generic instantiation.
cudaError_t launch_traj(int D, const Geom& g, const PhiloxKeys& K, const JobDesc* jobs,
                        int n_jobs, long long n_cta, int threads, cudaStream_t st)
{
    const bool fast = (g.Lh % 4) == 0;
    if (D == 2) {
        if (fast && g.G == 8) return launch_traj_t<2, true, 8, 1>(g, K, jobs, n_jobs, n_cta, threads, st);
        if (fast && g.G == 2) return launch_traj_t<2, true, 2, 1>(g, K, jobs, n_jobs, n_cta, threads, st);
        return fast ? launch_traj_t<2, true, 0, 0>(g, K, jobs, n_jobs, n_cta, threads, st)
                    : launch_traj_t<2, false, 0, 0>(g, K, jobs, n_jobs, n_cta, threads, st);
    }
    if (fast && g.G == 2 && g.Ly == 16)
        return launch_traj_t<3, true, 2, 16>(g, K, jobs, n_jobs, n_cta, threads, st);
    return fast ? launch_traj_t<3, true, 0, 0>(g, K, jobs, n_jobs, n_cta, threads, st)
                : launch_traj_t<3, false, 0, 0>(g, K, jobs, n_jobs, n_cta, threads, st);
}

cudaError_t launch_estimator(const long long* w_int, int n, double scale, int direction,
                             int n_blocks, double* out, cudaStream_t st)
{
    estimator_kernel<<<1, 1024, 0, st>>>(w_int, n, scale, direction, n_blocks, out);
    return cudaGetLastError();
}

}  // namespace jz
