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
// Thread mapping: the CTA has G * L_y * TS threads; thread (t0, y, q) owns
// spin word q of row y of every time slice t = t0, t0 + TS, ... in both
// replicas and both colours, so all index arithmetic and the x / y wrap
// offsets are fixed per thread.  Rows t >= 2 take the bulk path; the two rows
// next to the cut (t = 0, 1) blend in the glued replica and handle the
// switched column x = l.
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

// Flip bits of the four sites of a word.  dsum byte j = a_j, the number of
// anti-aligned neighbours of site j (energy cost m = 2D - 2 a_j); tab[a] =
// T(m) for a < D.  Sites with a_j >= D (m <= 0) always flip.
template <int D>
__device__ __forceinline__ uint32_t accept4(uint32_t dsum, const uint4& u, const uint32_t* tab)
{
    uint32_t f = ((dsum + (uint32_t)(0x80 - D) * 0x01010101u) >> 7) & 0x01010101u;
    const uint32_t d4 = dsum << 2;   // byte offsets into tab
    const unsigned char* tb = reinterpret_cast<const unsigned char*>(tab);
    if (u.x < *reinterpret_cast<const uint32_t*>(tb + (d4 & 0xFFu))) f |= 1u;
    if (u.y < *reinterpret_cast<const uint32_t*>(tb + __byte_perm(d4, 0, 0x4441))) f |= 1u << 8;
    if (u.z < *reinterpret_cast<const uint32_t*>(tb + __byte_perm(d4, 0, 0x4442))) f |= 1u << 16;
    if (u.w < *reinterpret_cast<const uint32_t*>(tb + __byte_perm(d4, 0, 0x4443))) f |= 1u << 24;
    return f;
}

template <int D, bool FAST>
struct Traj {
    const Geom& g;
    uint32_t* S;              // shared spin words [2][NR * G]
    const uint32_t* tab;      // shared bulk thresholds
    const PhiloxKeys& K;
    uint32_t hi1, lo1;        // M1 * traj: round 0 of Philox for counter word 2
    uint32_t c3base;          // dir bit << 1 | l << 2
    int q, y, t0, TS;         // this thread's word, row y, first slice and slice step
    int rowW, repW;           // words per time slice / per replica
    int d_qm, d_qp;           // word offset of the x-shift neighbour word (p = 0 / 1)
    int d_ym, d_yp;           // word offsets of the rows y-1 / y+1 (3D)
    uint32_t vmask;           // bytes of word q that hold sites (ragged rows)

    __device__ __forceinline__ Traj(const Geom& g_, uint32_t* S_, const uint32_t* tab_,
                                    const PhiloxKeys& K_, uint32_t traj, uint32_t c3base_)
        : g(g_), S(S_), tab(tab_), K(K_), c3base(c3base_)
    {
        const uint64_t p1 = (uint64_t)kPhiloxM1 * traj;
        hi1 = (uint32_t)(p1 >> 32);
        lo1 = (uint32_t)p1;
        const int tid = threadIdx.x;
        q = tid % g.G;
        y = (tid / g.G) % g.Ly;
        t0 = tid / (g.G * g.Ly);
        TS = blockDim.x / (g.G * g.Ly);
        rowW = g.Ly * g.G;
        repW = g.Lt * rowW;
        d_qm = (q == 0 ? g.G - 1 : q - 1) - q;
        d_qp = (q == g.G - 1 ? 0 : q + 1) - q;
        d_ym = ((y == 0 ? g.Ly - 1 : y - 1) - y) * g.G;
        d_yp = ((y == g.Ly - 1 ? 0 : y + 1) - y) * g.G;
        const int nv = g.Lh - 4 * q;
        vmask = nv >= 4 ? 0xFFFFFFFFu : ((1u << (8 * nv)) - 1u);
    }

    // Glue mask: bytes of word q (row parity p) whose site has x < lg.
    __device__ __forceinline__ uint32_t glue_mask(int lg, int p) const
    {
        int nj = ((lg - p + 1) >> 1) - 4 * q;   // # of sites 2h + p < lg in this word
        nj = nj < 0 ? 0 : (nj > 4 ? 4 : nj);
        return nj == 4 ? 0xFFFFFFFFu : ((1u << (8 * nj)) - 1u);
    }

    // The x neighbour that is not at the same h: h-1 for p = 0, h+1 for p = 1.
    __device__ __forceinline__ uint32_t xshift(const uint32_t* oth, int w, int p, uint32_t nx0) const
    {
        if (FAST) {
            const uint32_t nb = oth[w + (p ? d_qp : d_qm)];
            return __byte_perm(nb, nx0, p ? 0x0765 : 0x6543);
        }
        const uint8_t* row = reinterpret_cast<const uint8_t*>(oth + (w - q));
        uint32_t v = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int h = 4 * q + j;
            if (h < g.Lh) {
                const int hn = p == 0 ? (h == 0 ? g.Lh - 1 : h - 1) : (h == g.Lh - 1 ? 0 : h + 1);
                v |= (uint32_t)row[hn] << (8 * j);
            }
        }
        return v;
    }

    __device__ __forceinline__ uint4 rng(int w, uint32_t sweep, uint32_t c3) const
    {
        return philox_r0(
            (uint32_t)w, sweep, hi1, lo1, c3, K);
    }

    // Bulk row (2 <= t < L_t): every link is a full-beta link.
    __device__ __forceinline__ void bulk_item(uint32_t* own_b, const uint32_t* oth, int w, int t,
                                              int p, uint32_t sweep, uint32_t c3) const
    {
        const uint32_t own = own_b[w];
        const uint32_t ntm = oth[w - rowW];
        const uint32_t ntp = oth[t == g.Lt - 1 ? w - (g.Lt - 1) * rowW : w + rowW];
        const uint32_t nx0 = oth[w];
        const uint32_t nx1 = xshift(oth, w, p, nx0);
        uint32_t dsum = (own ^ ntm) + (own ^ ntp) + (own ^ nx0) + (own ^ nx1);
        if (D == 3) dsum += (own ^ oth[w + d_ym]) + (own ^ oth[w + d_yp]);
        const uint4 u = rng(w, sweep, c3);
        uint32_t flip = accept4<D>(dsum, u, tab);
        if (!FAST) flip &= vmask;
        own_b[w] = own ^ flip;
    }

    // Rows t = 0, 1 next to the cut.  lg = columns glued across the cut; k >= 0
    // is the protocol step (the switched column then uses the step's table).
    __device__ __forceinline__ void cut_item(uint32_t* own_b, const uint32_t* oth, int w, int t,
                                             int r, int p, uint32_t sweep, uint32_t c3, int k,
                                             int lg, int l, int n_step, int w_self, int w_glue,
                                             const uint32_t* __restrict__ tcut, bool record,
                                             int& dE) const
    {
        const uint32_t own = own_b[w];
        const int other_rep = r == 0 ? repW : -repW;
        const int w_cross = t == 0 ? w + rowW : w - rowW;           // self row across the cut
        const uint32_t self_w = oth[w_cross];
        const uint32_t glue_w = oth[w_cross + other_rep];
        const uint32_t normal = oth[t == 0 ? w + (g.Lt - 1) * rowW
                                           : (g.Lt == 2 ? w - rowW : w + rowW)];
        const uint32_t m = glue_mask(lg, p);
        const uint32_t cross = (self_w & ~m) | (glue_w & m);
        const uint32_t nx0 = oth[w];
        const uint32_t nx1 = xshift(oth, w, p, nx0);
        uint32_t dsum = (own ^ normal) + (own ^ cross) + (own ^ nx0) + (own ^ nx1);
        if (D == 3) dsum += (own ^ oth[w + d_ym]) + (own ^ oth[w + d_yp]);
        const uint4 u = rng(w, sweep, c3);
        uint32_t flip = accept4<D>(dsum, u, tab);
        // Switched site x = l during the protocol: couplings beta (1 - lambda)
        // to its own replica, beta lambda to the next one.
        if (k >= 0 && ((l - p) & 1) == 0 && ((l - p) >> 3) == q) {
            const int jl = ((l - p) >> 1) & 3;
            const uint32_t ob = (own >> (8 * jl)) & 1u;
            const int as = (int)(ob ^ ((self_w >> (8 * jl)) & 1u));
            const int ag = (int)(ob ^ ((glue_w >> (8 * jl)) & 1u));
            const int a_cnt = (int)((dsum >> (8 * jl)) & 0xFFu) - as;   // fixed links
            const int a = (2 * D - 1) - 2 * a_cnt;
            const int b = 1 - 2 * as;
            const int cg = 1 - 2 * ag;
            const int mm = a * n_step + b * w_self + cg * w_glue;
            const int ti = (((a + 2 * D - 1) >> 1) * 2 + (b > 0)) * 2 + (cg > 0);
            const bool acc = (mm <= 0) || (word_of(u, jl) < __ldg(tcut + k * (8 * D) + ti));
            flip = (flip & ~(0xFFu << (8 * jl))) | ((uint32_t)acc << (8 * jl));
            if (record) dE += b - cg;
        }
        if (!FAST) flip &= vmask;
        own_b[w] = own ^ flip;
    }

    __device__ __forceinline__ void half_sweep(int c, uint32_t sweep, int k, int lg, int l,
                                               int n_step, int w_self, int w_glue,
                                               const uint32_t* __restrict__ tcut, bool record,
                                               int& dE) const
    {
        const int cw = g.NR * g.G;
        uint32_t* own_b = S + c * cw;
        const uint32_t* oth = S + (1 - c) * cw;
        const uint32_t c3 = (uint32_t)c | c3base;
        const int w0 = t0 * rowW + y * g.G + q;
        for (int r = 0; r < 2; ++r) {
            int w = r * repW + w0;
            for (int t = t0; t < g.Lt; t += TS, w += TS * rowW) {
                const int p = (c + t + y) & 1;
                if (t >= 2)
                    bulk_item(own_b, oth, w, t, p, sweep, c3);
                else
                    cut_item(own_b, oth, w, t, r, p, sweep, c3, k, lg, l, n_step, w_self, w_glue,
                             tcut, record, dE);
            }
        }
    }

    __device__ __forceinline__ void hot_start() const
    {
        const int cw = g.NR * g.G;
        const int w0 = t0 * rowW + y * g.G + q;
        for (int c = 0; c < 2; ++c) {
            uint32_t* base = S + c * cw;
            const uint32_t c3 = (uint32_t)c | c3base | (1u << 30);
            for (int r = 0; r < 2; ++r) {
                int w = r * repW + w0;
                for (int t = t0; t < g.Lt; t += TS, w += TS * rowW) {
                    const uint4 u = rng(w, 0u, c3);
                    const uint32_t v = (u.x >> 31) | ((u.y >> 31) << 8) | ((u.z >> 31) << 16) |
                                       ((u.w >> 31) << 24);
                    base[w] = v & vmask;
                }
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
__global__ void __launch_bounds__(512)
traj_kernel(const Geom g, const PhiloxKeys K, const JobDesc* __restrict__ jobs, int n_jobs)
{
    extern __shared__ uint32_t S[];
    __shared__ int s_work;
    __shared__ uint32_t s_tab[8];

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

    if (threadIdx.x < 8) s_tab[threadIdx.x] = threadIdx.x < D ? __ldg(&J.tb[threadIdx.x]) : 0u;
    if (threadIdx.x == 0) s_work = 0;
    const Traj<D, FAST> tr(g, S, s_tab, K, (uint32_t)traj,
                           ((uint32_t)(dir < 0) << 1) | ((uint32_t)l << 2));
    tr.hot_start();
    __syncthreads();

    int dE = 0;
    // thermalisation at the start geometry: forward lambda = 0 (x < l glued),
    // reverse lambda = 1 (x <= l glued)
    const int lg_therm = dir > 0 ? l : l + 1;
    for (int s = 0; s < n_therm; ++s) {
        tr.half_sweep(0, (uint32_t)s, -1, lg_therm, l, n_step, 0, 0, tcut, false, dE);
        __syncthreads();
        tr.half_sweep(1, (uint32_t)s, -1, lg_therm, l, n_step, 0, 0, tcut, false, dE);
        __syncthreads();
    }
    uint32_t s = (uint32_t)n_therm;
    for (int k = 0; k < n_step; ++k) {
        const int kp = k + 1;
        const int w_self = dir > 0 ? n_step - kp : kp;
        const int w_glue = dir > 0 ? kp : n_step - kp;
        for (int i = 0; i < n_sweep; ++i, ++s) {
            tr.half_sweep(0, s, k, l, l, n_step, w_self, w_glue, tcut, i == 0, dE);
            __syncthreads();
            tr.half_sweep(1, s, k, l, l, n_step, w_self, w_glue, tcut, false, dE);
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
            int y = 0, trow = R;
            if (D == 3) { y = R % g.Ly; trow = R / g.Ly; }
            const int t = trow % g.Lt;
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
