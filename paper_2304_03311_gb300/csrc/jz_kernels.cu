// jz_kernels.cu -- the Jarzynski replica-gluing trajectory kernel and the FP64
// estimator kernel.
//
// traj_kernel: one CTA runs one trajectory from start to end with the whole
// replica lattice resident in shared memory: hot start, n_therm checkerboard
// Metropolis sweeps at the start geometry, then N protocol steps, each the work
// increment dE_k on phi_k followed by n_sweep sweeps at lambda_{k+1}
// (section 3, linear protocol; Appendix A, eq. work_in_one_MC_step and the
// remark on the update at lambda_{k+1}).  HBM is touched only for the job
// descriptor, the switched-site thresholds and the results.
//
// The work increment is gathered inside the first colour-0 half-sweep of each
// step: for every (r, y) exactly one of the switched sites (l, y, 0)^r and
// (l, y, 1)^r has colour 0, and s_i (s_self - s_glue) summed over those sites
// equals sum_{r,y} s^r(l,y,0) [s^r(l,y,1) - s^{r+1}(l,y,1)] (re-index the glue
// sum over r).  Each such site's own thread reads these values before it
// updates, and only colour-1 sites enter the products, so no extra barrier is
// needed.
#include <cstdint>

#include "jz_device.cuh"

namespace jz {

template <int D, bool FAST>
struct Sweeper {
    const Geom& g;
    uint32_t* S;             // shared spin words [2][NR][G]
    const PhiloxKeys& K;
    uint32_t traj;           // global trajectory index (counter word 2)
    uint32_t c3base;         // dir bit << 1 | l << 2
    uint32_t tb0, tb1, tb2;  // bulk thresholds by anti-aligned count

    // Glue mask: bytes of word q (row parity p) whose site has x < lg.
    __device__ __forceinline__ static uint32_t glue_mask(int lg, int p, int q)
    {
        int hg = (lg - p + 1) >> 1;                 // # of h with 2h + p < lg
        int nj = hg - 4 * q;
        nj = nj < 0 ? 0 : (nj > 4 ? 4 : nj);
        return nj == 4 ? 0xFFFFFFFFu : ((1u << (8 * nj)) - 1u);
    }

    // Half-sweep of colour c.  protocol: k >= 0 is the step index (the update
    // uses lambda_{k+1}); k < 0 is thermalisation at the start geometry with
    // lg glued columns.  record: accumulate dE_k into *dE.
    __device__ __forceinline__ void half_sweep(int c, uint32_t sweep_index, int k, int lg, int l,
                                               int n_step, int w_self, int w_glue,
                                               const uint32_t* __restrict__ tcut, bool record,
                                               int& dE)
    {
        const int G = g.G, NR = g.NR, Lt = g.Lt, Ly = g.Ly;
        const int items = NR * G;
        uint32_t* own_base = S + c * NR * G;
        const uint32_t* oth = S + (1 - c) * NR * G;
        const int stride_r = Lt * Ly;
        for (int idx = threadIdx.x; idx < items; idx += blockDim.x) {
            const int R = (int)div_magic((uint32_t)idx, (uint32_t)G, g.magic_G);
            const int q = idx - R * G;
            int y = 0, tr = R;
            if (D == 3) {
                tr = (int)div_magic((uint32_t)R, (uint32_t)Ly, g.magic_Ly);
                y = R - tr * Ly;
            }
            const int r = (int)div_magic((uint32_t)tr, (uint32_t)Lt, g.magic_Lt);
            const int t = tr - r * Lt;
            const int p = (c + t + y) & 1;

            const uint32_t own = own_base[idx];
            const int Rtm = t == 0 ? R + (Lt - 1) * Ly : R - Ly;
            const int Rtp = t == Lt - 1 ? R - (Lt - 1) * Ly : R + Ly;
            uint32_t ntm = oth[Rtm * G + q];
            uint32_t ntp = oth[Rtp * G + q];
            const uint32_t nx0 = oth[idx];
            uint32_t nx1;
            if (FAST) {
                if (p == 0) {
                    const uint32_t w = oth[R * G + (q == 0 ? G - 1 : q - 1)];
                    nx1 = __byte_perm(w, nx0, 0x6543);
                } else {
                    const uint32_t w = oth[R * G + (q == G - 1 ? 0 : q + 1)];
                    nx1 = __byte_perm(nx0, w, 0x4321);
                }
            } else {
                const uint8_t* row = reinterpret_cast<const uint8_t*>(oth + R * G);
                nx1 = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    int h = 4 * q + j;
                    if (h < g.Lh) {
                        int hn = p == 0 ? (h == 0 ? g.Lh - 1 : h - 1)
                                        : (h == g.Lh - 1 ? 0 : h + 1);
                        nx1 |= (uint32_t)row[hn] << (8 * j);
                    }
                }
            }

            // The cut: the link t = 0 -> 1 of columns x < lg joins replica r to
            // replica r+1 (n = 2: the same as r-1 from below).
            const bool cut_row = t <= 1;
            uint32_t self_w = 0, glue_w = 0;
            if (cut_row) {
                const int Rself = t == 0 ? Rtp : Rtm;
                const int Rglue = Rself + (r == 0 ? stride_r : -stride_r);
                self_w = t == 0 ? ntp : ntm;
                glue_w = oth[Rglue * G + q];
                const uint32_t m = glue_mask(lg, p, q);
                const uint32_t blended = (self_w & ~m) | (glue_w & m);
                if (t == 0) ntp = blended; else ntm = blended;
            }

            uint32_t dsum = (own ^ ntm) + (own ^ ntp) + (own ^ nx0) + (own ^ nx1);
            if (D == 3) {
                const int Rym = y == 0 ? R + Ly - 1 : R - 1;
                const int Ryp = y == Ly - 1 ? R - (Ly - 1) : R + 1;
                dsum += (own ^ oth[Rym * G + q]) + (own ^ oth[Ryp * G + q]);
            }

            const uint4 u = philox((uint32_t)idx, sweep_index, traj, (uint32_t)c | c3base, K);

            uint32_t flip = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t a = (dsum >> (8 * j)) & 0xFFu;
                uint32_t T = a == 0 ? tb0 : tb1;
                if (D == 3) T = a == 2 ? tb2 : T;
                const bool acc = (a >= (uint32_t)D) || (word_of(u, j) < T);
                flip |= (uint32_t)acc << (8 * j);
            }

            // Switched site x = l during the protocol: couplings beta (1 - lambda)
            // to its own replica, beta lambda to the next one.
            if (k >= 0 && cut_row && ((l - p) & 1) == 0 && ((l - p) >> 3) == q) {
                const int jl = ((l - p) >> 1) & 3;
                const uint32_t ob = (own >> (8 * jl)) & 1u;
                const int as = (int)(ob ^ ((self_w >> (8 * jl)) & 1u));
                const int ag = (int)(ob ^ ((glue_w >> (8 * jl)) & 1u));
                const int a_cnt = (int)((dsum >> (8 * jl)) & 0xFFu) - as;   // fixed links
                const int a = (2 * D - 1) - 2 * a_cnt;
                const int b = 1 - 2 * as;
                const int cg = 1 - 2 * ag;
                const int m = a * n_step + b * w_self + cg * w_glue;
                const int ti = (((a + 2 * D - 1) >> 1) * 2 + (b > 0)) * 2 + (cg > 0);
                const bool acc = (m <= 0) || (word_of(u, jl) < __ldg(tcut + k * (8 * D) + ti));
                flip = (flip & ~(0xFFu << (8 * jl))) | ((uint32_t)acc << (8 * jl));
                if (record) dE += b - cg;
            }
            if (!FAST) {
                const int nv = g.Lh - 4 * q;
                if (nv < 4) flip &= (1u << (8 * nv)) - 1u;
            }
            own_base[idx] = own ^ flip;
        }
    }

    __device__ __forceinline__ void hot_start()
    {
        const int items = g.NR * g.G;
        for (int c = 0; c < 2; ++c) {
            uint32_t* base = S + c * items;
            for (int idx = threadIdx.x; idx < items; idx += blockDim.x) {
                const uint4 u = philox((uint32_t)idx, 0u, traj,
                                       (uint32_t)c | c3base | (1u << 30), K);
                const int R = (int)div_magic((uint32_t)idx, (uint32_t)g.G, g.magic_G);
                const int q = idx - R * g.G;
                const int nv = g.Lh - 4 * q;
                uint32_t w = (u.x >> 31) | ((u.y >> 31) << 8) | ((u.z >> 31) << 16) |
                             ((u.w >> 31) << 24);
                if (nv < 4) w &= (1u << (8 * nv)) - 1u;
                base[idx] = w;
            }
        }
    }
};

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

template <int D, bool FAST>
__global__ void __launch_bounds__(256)
traj_kernel(const Geom g, const PhiloxKeys K, const JobDesc* __restrict__ jobs, int n_jobs)
{
    extern __shared__ uint32_t S[];
    __shared__ int s_work;

    const int j = find_job(jobs, n_jobs, (long long)blockIdx.x);
    const JobDesc& J = jobs[j];
    const int l = __ldg(&J.l);
    const int n_step = __ldg(&J.n_step);
    const int n_sweep = __ldg(&J.n_sweep);
    const int n_therm = __ldg(&J.n_therm);
    const int dir = __ldg(&J.dir);
    const long long local = (long long)blockIdx.x - __ldg(&J.cta0);
    const long long traj = __ldg(&J.traj0) + local;
    const uint32_t* tcut = J.tcut;

    Sweeper<D, FAST> sw{g, S, K, (uint32_t)traj,
                        ((uint32_t)(dir < 0) << 1) | ((uint32_t)l << 2),
                        __ldg(&J.tb[0]), __ldg(&J.tb[1]), __ldg(&J.tb[2])};
    if (threadIdx.x == 0) s_work = 0;
    sw.hot_start();
    __syncthreads();

    int dE = 0;
    // thermalisation at the start geometry: forward lambda = 0 (x < l glued),
    // reverse lambda = 1 (x <= l glued)
    const int lg_therm = dir > 0 ? l : l + 1;
    for (int s = 0; s < n_therm; ++s) {
        sw.half_sweep(0, (uint32_t)s, -1, lg_therm, l, n_step, 0, 0, tcut, false, dE);
        __syncthreads();
        sw.half_sweep(1, (uint32_t)s, -1, lg_therm, l, n_step, 0, 0, tcut, false, dE);
        __syncthreads();
    }
    uint32_t s = (uint32_t)n_therm;
    for (int k = 0; k < n_step; ++k) {
        const int kp = k + 1;
        const int w_self = dir > 0 ? n_step - kp : kp;
        const int w_glue = dir > 0 ? kp : n_step - kp;
        for (int i = 0; i < n_sweep; ++i, ++s) {
            sw.half_sweep(0, s, k, l, l, n_step, w_self, w_glue, tcut, i == 0, dE);
            __syncthreads();
            sw.half_sweep(1, s, k, l, l, n_step, w_self, w_glue, tcut, false, dE);
            __syncthreads();
        }
    }

    // per-trajectory integer work: warp reduction, then one shared atomic per warp
    const int wsum = __reduce_add_sync(0xFFFFFFFFu, dE);
    if ((threadIdx.x & 31) == 0 && wsum != 0) atomicAdd(&s_work, wsum);
    __syncthreads();
    if (threadIdx.x == 0) J.w_out[local] = (long long)(dir > 0 ? s_work : -s_work);

    int8_t* sp = J.spins_out;
    if (sp != nullptr) {
        const int V = 2 * g.Lt * g.Ly * g.L;
        int8_t* dst = sp + local * (long long)V;
        const uint8_t* bytes = reinterpret_cast<const uint8_t*>(S);
        for (int i = threadIdx.x; i < V; i += blockDim.x) {
            const int x = i % g.L;
            const int R = i / g.L;                      // (r, t, y) row
            int y = 0, tr = R;
            if (D == 3) { y = R % g.Ly; tr = R / g.Ly; }
            const int t = tr % g.Lt;
            const int c = (x + y + t) & 1;
            const uint8_t b = bytes[(size_t)(c * g.NR + R) * g.G * 4 + (x >> 1)];
            dst[i] = b ? (int8_t)-1 : (int8_t)1;
        }
    }
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

template <int D, bool FAST>
static cudaError_t launch_traj_t(const Geom& g, const PhiloxKeys& K, const JobDesc* jobs,
                                 int n_jobs, long long n_cta, int threads, cudaStream_t st)
{
    const size_t smem = traj_smem_bytes(g);
    cudaError_t e = cudaFuncSetAttribute(traj_kernel<D, FAST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    traj_kernel<D, FAST><<<(unsigned)n_cta, threads, smem, st>>>(g, K, jobs, n_jobs);
    return cudaGetLastError();
}

cudaError_t launch_traj(int D, const Geom& g, const PhiloxKeys& K, const JobDesc* jobs,
                        int n_jobs, long long n_cta, int threads, cudaStream_t st)
{
    const bool fast = (g.Lh % 4) == 0;
    if (D == 2) return fast ? launch_traj_t<2, true>(g, K, jobs, n_jobs, n_cta, threads, st)
                            : launch_traj_t<2, false>(g, K, jobs, n_jobs, n_cta, threads, st);
    return fast ? launch_traj_t<3, true>(g, K, jobs, n_jobs, n_cta, threads, st)
                : launch_traj_t<3, false>(g, K, jobs, n_jobs, n_cta, threads, st);
}

cudaError_t launch_estimator(const long long* w_int, int n, double scale, int direction,
                             int n_blocks, double* out, cudaStream_t st)
{
    estimator_kernel<<<1, 1024, 0, st>>>(w_int, n, scale, direction, n_blocks, out);
    return cudaGetLastError();
}

}  // namespace jz
