// jz_sw.cu -- Swendsen-Wang cluster update of the replica lattice (the update
// of the paper's own GPU code, section 3) inside a Jarzynski transformation.
//
// One CTA (256 threads in 2D, 512 in 3D) runs one trajectory.  Shared memory holds, for the V = n L_t L_y L
// sites of the replica lattice in natural order i = ((r L_t + t) L_y + y) L + x:
//   lab[V]   int32 cluster labels (lab[i] <= i always: a forest whose roots are
//            the smallest site index of their cluster)
//   sp[VW]   spin bits, bit i of the lattice = 1 for spin -1
//   bx, bt, bg, by [VW]  bond bits of the current sweep by direction
//   fz[VW]   flip bits of the current sweep, bit i for site i
//   bq       per warp 32 queued bonds
// Warps work on chunks of 32 consecutive sites.  One sweep is three phases
// separated by CTA barriers:
//   B1 every site draws one Philox block (i, s, traj, dir<<1 | l<<2 | 2<<30);
//      word w in {+x, +t same replica, +y, +t into replica r+1} activates that
//      forward link when both spins are equal and the word is below the link's
//      bond threshold floor(2^32 (1 - e^{-2K})).  +x bonds between lanes of
//      one chunk form runs found by one ballot; each site's label is set to
//      its run's first site.  The other active bonds become bits.  Block b
//      of the flip stream (b, s, traj, dir<<1 | l<<2 | 3<<30) gives the flip
//      bits of sites 128 b ... 128 b + 127 (words 0..3, bit i & 31).
//   B2 the recorded bonds, queued per warp and taken 32 at a time, merge
//      clusters by lock-free union (the larger root is hooked under the
//      smaller one, so the root of a cluster is its smallest site index);
//   CD every site finds its root (halving the path it walks) and flips iff the
//      root's flip bit is set: each cluster flips with probability 1/2, independently of
//      the others and of its bonds (a ballot assembles 32 sites into one spin
//      word).
// The cluster partition, hence the minimum-index root of every cluster, does
// not depend on the order of the unions, so the result is the same bit for bit
// as a sequential union-find over the same bonds.
//
// Termination: a label always points to a site with a smaller or equal index
// (equal only at a root), so every find walks a strictly decreasing chain (at
// most V steps) and every retry of a union restarts from a strictly smaller
// site.
#include <cstdint>

#include "jz_device.cuh"
#include "jz_host.h"

namespace jz {

namespace {

// Threads per CTA (one trajectory): 256 in 2D, 512 in 3D, whose extra +y
// bonds make the union phase longer (measured on 2D 64^2 and 3D 16^3).
__host__ __device__ constexpr int sw_threads(int D) { return D == 3 ? 512 : 256; }

// Minimum CTAs per SM for the register allocation.  0 for the shared-memory
// variants leaves the choice to the compiler (40 registers; on the 2D L = 64
// scan 7.5e10 site updates/s against 7.0e10 when sized for five CTAs, 48
// registers); the HBM variants are sized so that they do not spill.
__host__ __device__ constexpr int sw_min_ctas(int D, bool hbm)
{
    return hbm ? (D == 3 ? 3 : 5) : 0;
}

// Division by a fixed divisor d >= 1 for numerators n < 2^31 (Granlund and
// Montgomery, PLDI'94): with s = ceil(log2 d) and m = floor(2^32 (2^s - d) / d)
// + 1, n / d = (umulhi(m, n) + n) >> s.
struct FastDiv {
    uint32_t d, m, s;
};

FastDiv make_fastdiv(uint32_t d)
{
    uint32_t s = 0;
    while ((1ull << s) < d) ++s;
    const uint64_t m = (((1ull << s) - d) << 32) / d + 1;
    return FastDiv{d, (uint32_t)m, s};
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f)
{
    return (__umulhi(f.m, n) + n) >> f.s;
}

struct SwGeom {
    int L, Lt, Ly;
    int nrep;     // replicas n
    int V;        // sites of the replica lattice
    int VW;       // 32-bit words of one site bit array, ceil(V / 32)
    int SL;       // sites of one time slice, L_y * L
    int VR;       // sites of one replica, L_t * SL
    int G;        // Philox blocks per colour row of the hot start, ceil(L / 8)
    FastDiv dL, dLy, dLt;
};

struct Site {
    int x, y, t, r, row;
};

template <int D>
__device__ __forceinline__ Site decode(int i, const SwGeom& g)
{
    Site s;
    s.row = (int)fdiv((uint32_t)i, g.dL);
    s.x = i - s.row * g.L;
    int tr = s.row;
    s.y = 0;
    if (D == 3) {
        tr = (int)fdiv((uint32_t)s.row, g.dLy);
        s.y = s.row - tr * g.Ly;
    }
    s.r = (int)fdiv((uint32_t)tr, g.dLt);
    s.t = tr - s.r * g.Lt;
    return s;
}

// Offset from site i at t = 1 to its glued partner's replica: r+1 mod n.
__device__ __forceinline__ int glue_offset(const SwGeom& g, int r)
{
    return r == g.nrep - 1 ? -(g.nrep - 1) * g.VR : g.VR;
}

// Spin bit of site i < V (checked in bounds-checked builds).
__device__ __forceinline__ int spin_bit(const uint32_t* sp, int i, int V)
{
    return in_bounds(i, V, 20) ? (int)((sp[i >> 5] >> (i & 31)) & 1u) : 0;
}

// Root of a with path halving: every visited node is re-pointed to its
// grandparent.  A plain store is enough: the new parent is an ancestor of the
// node, and a hook that a concurrent union made on that node is only ever
// overwritten after the union has moved on to join the node's old tree.
__device__ __forceinline__ int find_root(volatile int* lab, int a, int V)
{
    for (;;) {
        if (!in_bounds(a, V, 21)) return 0;
        const int p = lab[a];
        if (p == a) return a;
        if (!in_bounds(p, V, 22)) return 0;
        const int gp = lab[p];
        if (gp == p) return p;
        lab[a] = gp;
        a = gp;
    }
}

__device__ __forceinline__ void merge(int* lab, int a, int b, int V)
{
    volatile int* vl = lab;
    for (;;) {
        a = find_root(vl, a, V);
        b = find_root(vl, b, V);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(&lab[a], b);   // hook root a under b < a
        if (old == a) return;
        a = old;                                 // a was hooked meanwhile: retry from its parent
    }
}

template <int D, bool HBM>
__global__ void __launch_bounds__(sw_threads(D), sw_min_ctas(D, HBM))
sw_kernel(const SwGeom g, const PhiloxKeys K, const JobDesc* __restrict__ jobs, int n_jobs,
          uint32_t* __restrict__ gS, size_t g_words)
{
    // the trajectory's state: shared memory, or this CTA's slice of an HBM
    // buffer when it does not fit (HBM, a compile-time choice so that the
    // shared-memory variant keeps 32-bit shared addressing)
    extern __shared__ uint32_t smem_shared[];
    uint32_t* smem = HBM ? gS + (size_t)blockIdx.x * g_words : smem_shared;
    int* lab = (int*)smem;
    uint32_t* sp = smem + g.V;
    uint32_t* bx = sp + g.VW;       // +x bonds leaving a warp chunk or its row
    uint32_t* bt = bx + g.VW;       // +t bonds inside one replica
    uint32_t* bg = bt + g.VW;       // +t bonds into replica r+1
    uint32_t* by = bg + g.VW;       // +y bonds (3D)
    uint32_t* fz = by + (D == 3 ? g.VW : 0);   // flip bits
    int* s_bq = (int*)(fz + g.VW);  // per warp 32 queued bonds (phase B2)

    // the job owning this CTA: the last j with jobs[j].cta0 <= blockIdx.x
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&jobs[mid].cta0) <= (long long)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const JobDesc& J = jobs[lo];
    const long long local = (long long)blockIdx.x - __ldg(&J.cta0);
    const int l = __ldg(&J.l), dir = __ldg(&J.dir);
    const int g0 = __ldg(&J.g0), g1 = __ldg(&J.g1);   // switching columns [g0, g1)
    const int n_step = __ldg(&J.n_step), n_sweep = __ldg(&J.n_sweep);
    const int n_therm = __ldg(&J.n_therm);
    const int prot = __ldg(&J.prot);
    const int den = prot == 2 ? n_step / g.Ly : n_step;   // steps of one column's run
    const uint32_t t_full = __ldg(&J.tb[0]);
    const uint32_t* bonds = J.tcut;          // [n_step][2]: self, glue thresholds
    const uint32_t traj = (uint32_t)(__ldg(&J.traj0) + local);
    const uint64_t p1 = (uint64_t)kPhiloxM1 * traj;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t c3 = ((uint32_t)(dir < 0) << 1) | ((uint32_t)l << 2);

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n_warps = blockDim.x >> 5;
    const int chunk = n_warps * 32;

    // hot start: spin -1 iff the top bit of the site's word of the colour-row
    // Philox block (row G + h/4, 0, traj, colour | dir<<1 | l<<2 | 1<<30), h = x/2;
    // a resumed segment (k_begin > 0) loads the stored configuration instead
    const int k_begin = __ldg(&J.k_begin), k_end = __ldg(&J.k_end);
    const int8_t* sin = k_begin > 0 ? J.spins_in + local * (long long)g.V : nullptr;
    for (int base = warp * 32; base < g.V; base += chunk) {
        const int i = base + lane;
        int bit = 0;
        if (i < g.V && sin) {
            bit = sin[i] < 0;
        } else if (i < g.V) {
            const Site s = decode<D>(i, g);
            const int h = s.x >> 1;
            const uint32_t colour = (uint32_t)((s.x + s.y + s.t) & 1);
            const uint4 u = philox_r0((uint32_t)(s.row * g.G + (h >> 2)), 0u, hi1, lo1,
                                      colour | c3 | (1u << 30), K);
            bit = (int)(word_of(u, h & 3) >> 31);
        }
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, bit);
        if (lane == 0) sp[base >> 5] = m;
    }
    __syncthreads();

    long long w = 0;
    const int sw_end = n_therm + k_end * n_sweep;
    for (int sw = k_begin > 0 ? n_therm + k_begin * n_sweep : 0; sw < sw_end; ++sw) {
        const int k = sw < n_therm ? -1 : (sw - n_therm) / n_sweep;
        const bool step_start = k >= 0 && (sw - n_therm) % n_sweep == 0;
        // protocol 2: only column y = ya moves at step k; columns before it sit
        // at the end geometry, the ones after it at the start geometry
        const int ya = (k >= 0 && prot == 2) ? k / den : -1;
        // work of step k on the configuration before its sweeps:
        // dE = sum_{r,y} s(l,y,0)^r [s(l,y,1)^r - s(l,y,1)^{r+1}] over the
        // moving columns
        if (step_start && warp == 0) {
            int e = 0;
            const int nx = g1 - g0;
            for (int q = lane; q < g.nrep * g.Ly * nx; q += 32) {
                const int ry = q / nx, x = g0 + (q - ry * nx);
                const int r = ry / g.Ly, y = ry - r * g.Ly;
                if (ya >= 0 && y != ya) continue;
                const int lo_i = (r * g.Lt * g.Ly + y) * g.L + x;
                const int up_s = lo_i + g.SL;
                const int up_g = up_s + glue_offset(g, r);
                const int s0 = 1 - 2 * spin_bit(sp, lo_i, g.V);
                e += s0 * ((1 - 2 * spin_bit(sp, up_s, g.V)) -
                           (1 - 2 * spin_bit(sp, up_g, g.V)));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xFFFFFFFFu, e, o);
            w += e;
        }
        uint32_t t_self = 0, t_glue = 0;   // the switched column's two time links
        if (k < 0) {
            if (dir > 0) t_self = t_full; else t_glue = t_full;
        } else {
            t_self = __ldg(&bonds[2 * k]);
            t_glue = __ldg(&bonds[2 * k + 1]);
        }
        const uint32_t cb = c3 | (2u << 30);
        // the sweep's flip bits: one Philox block per 128 sites, spread over
        // the lanes of every warp so that each warp runs one Philox pass
        for (int b = warp + lane * n_warps; 4 * b < g.VW; b += 32 * n_warps) {
            const uint4 u = philox_r0((uint32_t)b, (uint32_t)sw, hi1, lo1, c3 | (3u << 30), K);
            fz[4 * b] = u.x;
            if (4 * b + 1 < g.VW) fz[4 * b + 1] = u.y;
            if (4 * b + 2 < g.VW) fz[4 * b + 2] = u.z;
            if (4 * b + 3 < g.VW) fz[4 * b + 3] = u.w;
        }
        // phase B1: bond draws.  A +x bond between two lanes of one warp
        // chunk joins a run of consecutive sites; every site of a run gets the
        // run's first site as its label (a star).  All other active bonds are
        // recorded as bits for phase B2.
        for (int base = warp * 32; base < g.V; base += chunk) {
            const int i = base + lane;
            bool ax = false, at = false, ay = false, ag = false, last = true;
            if (i < g.V) {
                const Site s = decode<D>(i, g);
                const int si = spin_bit(sp, i, g.V);
                last = s.x == g.L - 1;
                const int jx = last ? i + 1 - g.L : i + 1;
                int jt = -1, jg = -1, jy = -1;
                uint32_t Tt = t_full, Tg = 0;
                if (s.t != 0) {
                    jt = s.t == g.Lt - 1 ? i + g.SL - g.VR : i + g.SL;
                } else {
                    const int js = i + g.SL;
                    const int jgl = js + glue_offset(g, s.r);
                    if (s.x >= g1) {
                        jt = js;
                    } else if (s.x < g0) {
                        jg = jgl;
                        Tg = t_full;
                    } else if (ya >= 0 && s.y != ya) {
                        if ((s.y < ya) == (dir > 0)) {
                            jg = jgl;
                            Tg = t_full;
                        } else {
                            jt = js;
                        }
                    } else {
                        jt = js;
                        Tt = t_self;
                        jg = jgl;
                        Tg = t_glue;
                    }
                }
                if (D == 3) jy = s.y == g.Ly - 1 ? i + g.L - g.SL : i + g.L;
                const uint4 u = philox_r0((uint32_t)i, (uint32_t)sw, hi1, lo1, cb, K);
                ax = u.x < t_full && spin_bit(sp, jx, g.V) == si;
                at = jt >= 0 && u.y < Tt && spin_bit(sp, jt, g.V) == si;
                if (D == 3) ay = u.z < t_full && spin_bit(sp, jy, g.V) == si;
                ag = jg >= 0 && u.w < Tg && spin_bit(sp, jg, g.V) == si;
            }
            const bool inw = ax && lane != 31 && !last;   // bond to the next lane's site
            const uint32_t m = __ballot_sync(0xFFFFFFFFu, inw);
            const uint32_t brk = ~m & ((1u << lane) - 1u);
            const int start = brk ? 32 - __clz(brk) : 0;
            if (i < g.V) lab[i] = base + start;
            const uint32_t wx = __ballot_sync(0xFFFFFFFFu, ax && !inw);
            const uint32_t wt = __ballot_sync(0xFFFFFFFFu, at);
            const uint32_t wg = __ballot_sync(0xFFFFFFFFu, ag);
            const uint32_t wy = D == 3 ? __ballot_sync(0xFFFFFFFFu, ay) : 0u;
            if (lane == 0) {
                const int q = base >> 5;
                bx[q] = wx;
                bt[q] = wt;
                bg[q] = wg;
                if (D == 3) by[q] = wy;
            }
        }
        __syncthreads();
        // phase B2: the recorded bonds merge clusters (+x bonds inside a
        // chunk are already joined by the run labels).  Each warp queues its
        // chunks' bonds as (site << 2 | direction) and merges them 32 at a
        // time, so every merge round runs on a full warp.
        {
            int* bq = s_bq + warp * 32;
            int nb = 0;
            auto merge_entry = [&](int e) {
                const int i = e >> 2, dirn = e & 3;
                const Site s = decode<D>(i, g);
                int j;
                if (dirn == 0) j = s.x == g.L - 1 ? i + 1 - g.L : i + 1;
                else if (dirn == 1) j = s.t == g.Lt - 1 ? i + g.SL - g.VR : i + g.SL;
                else if (dirn == 2) j = i + g.SL + glue_offset(g, s.r);
                else j = s.y == g.Ly - 1 ? i + g.L - g.SL : i + g.L;
                if (in_bounds(i, g.V, 23) && in_bounds(j, g.V, 24)) merge(lab, i, j, g.V);
            };
            auto push = [&](uint32_t m, int e) {   // m: the warp's mask of bonds
                const int c = __popc(m);
                if (c == 0) return;
                const bool mine = (m >> lane) & 1u;
                const int rank = __popc(m & ((1u << lane) - 1u));
                const int room = 32 - nb;
                if (mine && rank < room) bq[nb + rank] = e;
                nb += c;
                if (nb >= 32) {
                    __syncwarp();
                    merge_entry(bq[lane]);
                    __syncwarp();
                    if (mine && rank >= room) bq[rank - room] = e;
                    nb -= 32;
                }
            };
            for (int base = warp * 32; base < g.V; base += chunk) {
                const int i = base + lane;
                const int q = base >> 5;
                const uint32_t wx = bx[q], wt = bt[q], wg = bg[q];
                const uint32_t wy = D == 3 ? by[q] : 0u;
                __syncwarp();
                push(wx, i << 2);
                push(wt, (i << 2) | 1);
                push(wg, (i << 2) | 2);
                if (D == 3) push(wy, (i << 2) | 3);
            }
            __syncwarp();
            if (lane < nb) merge_entry(bq[lane]);
        }
        __syncthreads();
        // phase CD: every site flips iff its cluster's root drew a set flip
        // bit.  The walks halve the paths they take (a label only ever moves
        // to an ancestor, so concurrent walkers still reach the root), which
        // shortens the walks of later sites through them: on the 2D L = 64
        // and 3D 16^3 scans this phase then takes about a third less time
        // than with read-only walks.
        for (int base = warp * 32; base < g.V; base += chunk) {
            const int i = base + lane;
            int f = 0;
            if (i < g.V) {
                const int root = find_root((volatile int*)lab, i, g.V);
                f = (int)((fz[root >> 5] >> (root & 31)) & 1u);
            }
            const uint32_t m = __ballot_sync(0xFFFFFFFFu, f);
            if (lane == 0) sp[base >> 5] ^= m;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        J.w_out[local] = (k_begin > 0 ? J.w_in[local] : 0) +
                         (dir > 0 ? w : -w) * (prot == 2 ? g.Ly : 1);
    int8_t* so = J.spins_out;
    if (so != nullptr) {
        so += local * (long long)g.V;
        for (int i = threadIdx.x; i < g.V; i += blockDim.x)
            so[i] = spin_bit(sp, i, g.V) ? (int8_t)-1 : (int8_t)1;
    }
}

SwGeom make_swgeom(int D, const Geom& geo)
{
    SwGeom g;
    g.L = geo.L;
    g.Lt = geo.Lt;
    g.Ly = geo.Ly;
    g.SL = g.Ly * g.L;
    g.VR = g.Lt * g.SL;
    g.nrep = geo.nrep;
    g.V = g.nrep * g.VR;
    g.VW = (g.V + 31) / 32;
    g.G = geo.G;
    g.dL = make_fastdiv((uint32_t)g.L);
    g.dLy = make_fastdiv((uint32_t)g.Ly);
    g.dLt = make_fastdiv((uint32_t)g.Lt);
    (void)D;
    return g;
}

}  // namespace

int sw_cta_threads(int D) { return sw_threads(D); }

long long sw_hbm_wave(int D)
{
    int dev = 0, n_sm = 0, per_sm = 0;
    auto kern = D == 3 ? sw_kernel<3, true> : sw_kernel<2, true>;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, sw_threads(D), 0) !=
            cudaSuccess) {
        cudaGetLastError();
        return sw_min_ctas(D, true);
    }
    return (long long)n_sm * (per_sm > 0 ? per_sm : 1);
}

cudaError_t bounds_status_sw(unsigned int out[2], bool clear)
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

size_t sw_smem_bytes(const Geom& geo)
{
    const size_t V = (size_t)geo.nrep * geo.Lt * geo.Ly * geo.L;
    const int VW = (int)((V + 31) / 32);
    const int threads = sw_threads(geo.Ly > 1 ? 3 : 2);
    const size_t words = (geo.Ly > 1 ? 6 : 5) * (size_t)VW + (size_t)threads;
    return V * sizeof(int) + words * sizeof(uint32_t);
}

cudaError_t launch_sw(int D, const Geom& geo, const PhiloxKeys& K, const JobDesc* jobs,
                      int n_jobs, long long n_cta, cudaStream_t st, uint32_t* gS)
{
    const SwGeom g = make_swgeom(D, geo);
    const size_t bytes = sw_smem_bytes(geo);
    const size_t smem = gS ? 0 : bytes;
    auto kern = D == 3 ? (gS ? sw_kernel<3, true> : sw_kernel<3, false>)
                       : (gS ? sw_kernel<2, true> : sw_kernel<2, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)n_cta, sw_threads(D), smem, st>>>(g, K, jobs, n_jobs, gS,
                                                       bytes / sizeof(uint32_t));
    return cudaGetLastError();
}

}  // namespace jz
