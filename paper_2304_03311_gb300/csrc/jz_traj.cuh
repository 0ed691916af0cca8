// jz_traj.cuh -- one Jarzynski trajectory of the replica-gluing method, run
// by a team of threads over a replica lattice held in shared memory.
//
// Per trajectory (section 3, linear protocol; Appendix A, eq.
// work_in_one_MC_step and the remark on the update at lambda_{k+1}): hot
// start, n_therm checkerboard Metropolis sweeps at the start geometry, then N
// protocol steps, each the work increment dE_k on phi_k followed by n_sweep
// sweeps at lambda_{k+1}.
//
// Layout: S[colour][row R][word q], R = (r L_t + t) L_y + y, q < G = ceil(L/8);
// byte j of word q is the colour-c site h = 4q + j of the row, x = 2h + p,
// p = (c + t + y) mod 2, value 0 for spin +1 and 1 for spin -1.
//
// Team mapping: a team of G * L_y * TS threads; thread (t0, y, q) owns word q
// of row y of the time slices t0, t0 + TS, ... in both replicas and colours, so
// all its index and wrap arithmetic is fixed.  Rows t >= 2 take the bulk path;
// the rows t = 0, 1 next to the cut blend in the glued replica and handle the
// switched column x = l.  CG, CLY > 0 fix G and L_y at compile time (the
// neighbour loads then use immediate offsets); 0 reads them from Geom.
//
// The work increment is gathered inside the first colour-0 half-sweep of each
// step: for every (r, y) exactly one of the switched sites (l, y, 0)^r and
// (l, y, 1)^r has colour 0, and s_i (s_self - s_glue) summed over those sites
// equals sum_{r,y} s^r(l,y,0) [s^r(l,y,1) - s^{r+1}(l,y,1)] (re-index the glue
// sum over r).  Each such site's own thread reads these values before it
// updates, and only colour-1 sites enter the products, so no extra barrier is
// needed.
#pragma once
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

// Per-job values a team needs (read from the job descriptor once).
struct TeamJob {
    int l, n_step, n_sweep, n_therm, dir;
    const uint32_t* tcut;
};

template <int D, bool FAST, int CG = 0, int CLY = 0>
struct Traj {
    const Geom& g;
    uint32_t* S;              // this team's spin words [2][NR * G]
    const uint32_t* tab;      // shared bulk thresholds
    const PhiloxKeys& K;
    uint32_t hi1, lo1;        // M1 * traj: round 0 of Philox for counter word 2
    uint32_t c3base;          // dir bit << 1 | l << 2
    int q, y, t0, TS;         // this thread's word, row y, first slice and slice step
    int d_qm, d_qp;           // word offset of the x-shift neighbour word (p = 0 / 1)
    int d_ym, d_yp;           // word offsets of the rows y-1 / y+1 (3D)
    uint32_t vmask;           // bytes of word q that hold sites (ragged rows)

    __device__ __forceinline__ int G() const { return CG > 0 ? CG : g.G; }
    __device__ __forceinline__ int Ly() const { return D == 2 ? 1 : (CLY > 0 ? CLY : g.Ly); }
    __device__ __forceinline__ int rowW() const { return Ly() * G(); }

    // tid < 0: a thread with no sites (it still takes part in the barriers).
    __device__ __forceinline__ Traj(const Geom& g_, uint32_t* S_, const uint32_t* tab_,
                                    const PhiloxKeys& K_, uint32_t traj, uint32_t c3base_,
                                    int tid, int nthr)
        : g(g_), S(S_), tab(tab_), K(K_), c3base(c3base_)
    {
        const uint64_t p1 = (uint64_t)kPhiloxM1 * traj;
        hi1 = (uint32_t)(p1 >> 32);
        lo1 = (uint32_t)p1;
        const int col = G() * Ly();
        TS = nthr / col;
        if (tid < 0) {
            q = y = 0;
            t0 = g.Lt;
        } else {
            q = tid % G();
            y = (tid / G()) % Ly();
            t0 = tid / col;
        }
        d_qm = (q == 0 ? G() - 1 : q - 1) - q;
        d_qp = (q == G() - 1 ? 0 : q + 1) - q;
        d_ym = ((y == 0 ? Ly() - 1 : y - 1) - y) * G();
        d_yp = ((y == Ly() - 1 ? 0 : y + 1) - y) * G();
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

    // The x neighbour not at the same h: h-1 for p = 0, h+1 for p = 1.  The
    // row's other words are at o[d_qm] / o[d_qp]; o points at word q.
    __device__ __forceinline__ uint32_t xshift(const uint32_t* o, int p, uint32_t nx0) const
    {
        if (FAST) {
            const uint32_t nb = o[p ? d_qp : d_qm];
            return __byte_perm(nb, nx0, p ? 0x0765 : 0x6543);
        }
        const uint8_t* row = reinterpret_cast<const uint8_t*>(o - q);
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
        return philox_r0((uint32_t)w, sweep, hi1, lo1, c3, K);
    }

    // Bulk row, 2 <= t < L_t, all links full beta.  up: offset of the t+1 row
    // (rowW, or -(L_t - 1) rowW at t = L_t - 1).
    __device__ __forceinline__ void bulk_item(uint32_t* own_b, const uint32_t* oth, int w, int up,
                                              int p, uint32_t sweep, uint32_t c3) const
    {
        const uint32_t* o = oth + w;
        const uint32_t own = own_b[w];
        const uint32_t ntm = o[-rowW()];
        const uint32_t ntp = o[up];
        const uint32_t nx0 = o[0];
        const uint32_t nx1 = xshift(o, p, nx0);
        uint32_t dsum = (own ^ ntm) + (own ^ ntp) + (own ^ nx0) + (own ^ nx1);
        if (D == 3) dsum += (own ^ o[d_ym]) + (own ^ o[d_yp]);
        const uint4 u = rng(w, sweep, c3);
        uint32_t flip = accept4<D>(dsum, u, tab);
        if (!FAST) flip &= vmask;
        own_b[w] = own ^ flip;
    }

    // Rows t = 0, 1 next to the cut.  lg = columns glued across the cut; k >= 0
    // is the protocol step (the switched column then uses the step's table).
    __device__ __forceinline__ void cut_item(uint32_t* own_b, const uint32_t* oth, int w, int t,
                                             int r, int p, uint32_t sweep, uint32_t c3, int k,
                                             int lg, const TeamJob& J, int w_self, int w_glue,
                                             bool record, int& dE) const
    {
        const int rw = rowW();
        const int repW = g.Lt * rw;
        const uint32_t* o = oth + w;
        const uint32_t own = own_b[w];
        const int cross_off = t == 0 ? rw : -rw;                   // self row across the cut
        const uint32_t self_w = o[cross_off];
        const uint32_t glue_w = o[cross_off + (r == 0 ? repW : -repW)];
        const uint32_t normal = o[t == 0 ? (g.Lt - 1) * rw : (g.Lt == 2 ? -rw : rw)];
        const uint32_t m = glue_mask(lg, p);
        const uint32_t cross = (self_w & ~m) | (glue_w & m);
        const uint32_t nx0 = o[0];
        const uint32_t nx1 = xshift(o, p, nx0);
        uint32_t dsum = (own ^ normal) + (own ^ cross) + (own ^ nx0) + (own ^ nx1);
        if (D == 3) dsum += (own ^ o[d_ym]) + (own ^ o[d_yp]);
        const uint4 u = rng(w, sweep, c3);
        uint32_t flip = accept4<D>(dsum, u, tab);
        // Switched site x = l during the protocol: couplings beta (1 - lambda)
        // to its own replica, beta lambda to the next one.
        const int l = J.l;
        if (k >= 0 && ((l - p) & 1) == 0 && ((l - p) >> 3) == q) {
            const int jl = ((l - p) >> 1) & 3;
            const uint32_t ob = (own >> (8 * jl)) & 1u;
            const int as = (int)(ob ^ ((self_w >> (8 * jl)) & 1u));
            const int ag = (int)(ob ^ ((glue_w >> (8 * jl)) & 1u));
            const int a_cnt = (int)((dsum >> (8 * jl)) & 0xFFu) - as;   // fixed links
            const int a = (2 * D - 1) - 2 * a_cnt;
            const int b = 1 - 2 * as;
            const int cg = 1 - 2 * ag;
            const int mm = a * J.n_step + b * w_self + cg * w_glue;
            const int ti = (((a + 2 * D - 1) >> 1) * 2 + (b > 0)) * 2 + (cg > 0);
            const bool acc = (mm <= 0) || (word_of(u, jl) < __ldg(J.tcut + k * (8 * D) + ti));
            flip = (flip & ~(0xFFu << (8 * jl))) | ((uint32_t)acc << (8 * jl));
            if (record) dE += b - cg;
        }
        if (!FAST) flip &= vmask;
        own_b[w] = own ^ flip;
    }

    __device__ __forceinline__ void half_sweep(int c, uint32_t sweep, int k, int lg,
                                               const TeamJob& J, int w_self, int w_glue,
                                               bool record, int& dE) const
    {
        const int rw = rowW();
        const int Lt = g.Lt;
        const int cw = 2 * Lt * rw;
        uint32_t* own_b = S + c * cw;
        const uint32_t* oth = S + (1 - c) * cw;
        const uint32_t c3 = (uint32_t)c | c3base;
        const int stride = TS * rw;
        const int pc = (c + y) & 1;
        const int wrap_up = -(Lt - 1) * rw;
#pragma unroll 1
        for (int r = 0; r < 2; ++r) {
            int t = t0;
            int w = (r * Lt + t0) * rw + y * G() + q;
            for (; t < 2 && t < Lt; t += TS, w += stride)
                cut_item(own_b, oth, w, t, r, (pc ^ t) & 1, sweep, c3, k, lg, J, w_self, w_glue,
                         record, dE);
            if (TS & 1) {
                for (; t < Lt; t += TS, w += stride)
                    bulk_item(own_b, oth, w, t == Lt - 1 ? wrap_up : rw, (pc ^ t) & 1, sweep, c3);
            } else {
                // t keeps its parity: the x-shift direction is fixed for the row set
                const int p = (pc ^ t0) & 1;
                for (; t < Lt - TS; t += TS, w += stride)
                    bulk_item(own_b, oth, w, rw, p, sweep, c3);
                if (t < Lt) bulk_item(own_b, oth, w, t == Lt - 1 ? wrap_up : rw, p, sweep, c3);
            }
        }
    }

    __device__ __forceinline__ void hot_start() const
    {
        const int rw = rowW();
        const int cw = 2 * g.Lt * rw;
        for (int c = 0; c < 2; ++c) {
            uint32_t* base = S + c * cw;
            const uint32_t c3 = (uint32_t)c | c3base | (1u << 30);
            for (int r = 0; r < 2; ++r) {
                int w = (r * g.Lt + t0) * rw + y * G() + q;
                for (int t = t0; t < g.Lt; t += TS, w += TS * rw) {
                    const uint4 u = rng(w, 0u, c3);
                    const uint32_t v = (u.x >> 31) | ((u.y >> 31) << 8) | ((u.z >> 31) << 16) |
                                       ((u.w >> 31) << 24);
                    base[w] = v & vmask;
                }
            }
        }
    }
};

// Runs one whole trajectory with the team's threads.  Every thread of the CTA
// calls it with the same job (trip counts match across teams); tid < 0 marks
// a thread without sites.  bar() synchronises the team (all teams of a CTA
// run in lockstep, so __syncthreads serves).  Returns this thread's share of
// W_int (in units of beta/N, sign of the direction applied by the caller).
template <int D, bool FAST, int CG, int CLY, class Bar>
__device__ __forceinline__ int run_trajectory(const Geom& g, const PhiloxKeys& K, const TeamJob& J,
                                              long long traj, uint32_t* S_team,
                                              const uint32_t* tab, int tid, int nthr, Bar bar)
{
    const Traj<D, FAST, CG, CLY> tr(g, S_team, tab, K, (uint32_t)traj,
                                    ((uint32_t)(J.dir < 0) << 1) | ((uint32_t)J.l << 2), tid, nthr);
    tr.hot_start();
    bar();
    int dE = 0;
    // thermalisation at the start geometry: forward lambda = 0 (x < l glued),
    // reverse lambda = 1 (x <= l glued)
    const int lg_therm = J.dir > 0 ? J.l : J.l + 1;
    for (int s = 0; s < J.n_therm; ++s) {
        tr.half_sweep(0, (uint32_t)s, -1, lg_therm, J, 0, 0, false, dE);
        bar();
        tr.half_sweep(1, (uint32_t)s, -1, lg_therm, J, 0, 0, false, dE);
        bar();
    }
    uint32_t s = (uint32_t)J.n_therm;
    for (int k = 0; k < J.n_step; ++k) {
        const int kp = k + 1;
        const int w_self = J.dir > 0 ? J.n_step - kp : kp;
        const int w_glue = J.dir > 0 ? kp : J.n_step - kp;
        for (int i = 0; i < J.n_sweep; ++i, ++s) {
            tr.half_sweep(0, s, k, J.l, J, w_self, w_glue, i == 0, dE);
            bar();
            tr.half_sweep(1, s, k, J.l, J, w_self, w_glue, false, dE);
            bar();
        }
    }
    return dE;
}

// Writes a team's final configuration as int8 +-1 in the order [r][t][y][x].
template <int D>
__device__ __forceinline__ void export_spins(const Geom& g, const uint32_t* S_team, int8_t* dst,
                                             int tid, int nthr)
{
    const int V = 2 * g.Lt * g.Ly * g.L;
    const uint8_t* bytes = reinterpret_cast<const uint8_t*>(S_team);
    for (int i = tid; i < V; i += nthr) {
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

__device__ __forceinline__ TeamJob team_job(const JobDesc& J)
{
    TeamJob t;
    t.l = __ldg(&J.l);
    t.n_step = __ldg(&J.n_step);
    t.n_sweep = __ldg(&J.n_sweep);
    t.n_therm = __ldg(&J.n_therm);
    t.dir = __ldg(&J.dir);
    t.tcut = J.tcut;
    return t;
}

}  // namespace jz
