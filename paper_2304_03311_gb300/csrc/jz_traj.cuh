// jz_traj.cuh -- one Jarzynski trajectory of the replica-gluing method, run
// by a team of threads over a replica lattice held in shared memory.
//
// Per trajectory (section 3, linear protocol; Appendix A, eq.
// work_in_one_MC_step and the remark on the update at lambda_{k+1}): hot
// start, n_therm checkerboard Metropolis sweeps at the start geometry, then N
// protocol steps, each the work increment dE_k on phi_k followed by n_sweep
// sweeps at lambda_{k+1}.
//
// Layout: S[colour][row R][word q], R = (r L_t + t) L_y + y, q < GW = ceil(L/16);
// nibble j (bits 4j..4j+3) of word q is the colour-c site h = 8q + j of the
// row, x = 2h + p, p = (c + t + y) mod 2, value 0 for spin +1 and 1 for -1.
// A word's eight sites draw from Philox blocks 2q and 2q+1 of their row.
// Nibble-wise sums of XORs give the anti-aligned neighbour count of all eight
// sites at once (at most 6 < 16, so no carries cross nibbles).
//
// Team mapping: a team of GW * L_y * TS * RS threads; thread (r0, t0, y, q)
// owns word q of row y of the time slices t0, t0 + TS, ... in the replicas
// r0, r0 + RS, ... and both colours, so all its index and wrap arithmetic is
// fixed.  RS > 1 only when TS = L_t (a whole time column per thread slot):
// lattices so small that one replica's words leave most of a warp idle.  Rows t >= 2 take the bulk
// path; the rows t = 0, 1 next to the cut blend in the glued replica and
// handle the switched column x = l.  CW, CLY > 0 fix GW and L_y at compile
// time (neighbour loads then use immediate offsets); 0 reads them from Geom.
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

// Flip bits (bit 4j) of the eight sites of a word.  dsum nibble j = a_j, the
// number of anti-aligned neighbours of site j (energy cost m = 2D - 2 a_j);
// tab[a] = T(m) for a < D.  Sites with a_j >= D (m <= 0) always flip.  Sites
// 0..3 use the words of block ua, sites 4..7 those of block ub.
template <int D>
__device__ __forceinline__ uint32_t accept8(uint32_t dsum, const uint4& ua, const uint4& ub,
                                            const uint32_t* tab)
{
    uint32_t f = ((dsum + (uint32_t)(8 - D) * 0x11111111u) >> 3) & 0x11111111u;
    const uint32_t ev = (dsum & 0x0F0F0F0Fu) << 2;   // sites 0,2,4,6: byte offsets into tab
    const uint32_t od = (dsum >> 2) & 0x3C3C3C3Cu;   // sites 1,3,5,7
    const unsigned char* tb = reinterpret_cast<const unsigned char*>(tab);
    auto T = [&](uint32_t off) { return *reinterpret_cast<const uint32_t*>(tb + off); };
    if (ua.x < T(ev & 0xFFu)) f |= 1u;
    if (ua.y < T(od & 0xFFu)) f |= 1u << 4;
    if (ua.z < T(__byte_perm(ev, 0, 0x4441))) f |= 1u << 8;
    if (ua.w < T(__byte_perm(od, 0, 0x4441))) f |= 1u << 12;
    if (ub.x < T(__byte_perm(ev, 0, 0x4442))) f |= 1u << 16;
    if (ub.y < T(__byte_perm(od, 0, 0x4442))) f |= 1u << 20;
    if (ub.z < T(__byte_perm(ev, 0, 0x4443))) f |= 1u << 24;
    if (ub.w < T(__byte_perm(od, 0, 0x4443))) f |= 1u << 28;
    return f;
}

__device__ __forceinline__ uint32_t word8(const uint4& ua, const uint4& ub, int j)
{
    return word_of(j < 4 ? ua : ub, j & 3);
}

// Per-job values a team needs (read from the job descriptor once).
struct TeamJob {
    int l, n_step, n_sweep, n_therm, dir;
    int k_begin, k_end;   // protocol steps run; k_begin > 0 resumes from stored spins
    int start_in;         // 1: step k_begin = 0 starts from stored (thermalised) spins
    int g0, g1;   // columns x < g0 glued, g0 <= x < g1 switching, x >= g1 self
    int prot;     // 1: every switched column together; 2: one column y at a time
    int den;      // steps of one column's run: N (protocol 1), N / L_y (protocol 2)
    const uint32_t* tcut;
};

// CLT, CTS > 0: L_t and the slice step TS fixed at compile time (the 2D L = 64,
// L_t = 64 warp teams); 0 reads them from Geom and the team size.
template <int D, bool FAST, int CW = 0, int CLY = 0, int CLT = 0, int CTS = 0>
struct Traj {
    const Geom& g;
    uint32_t* S;              // this team's spin words [2][NR * GW]
    const uint32_t* tab;      // shared bulk thresholds
    const PhiloxKeys& K;
    uint32_t hi1, lo1;        // M1 * traj: round 0 of Philox for counter word 2
    uint32_t c3base;          // dir bit << 1 | l << 2
    int q, y, t0, TS;         // this thread's word, row y, first slice and slice step
    int r0, RS;               // first replica and replica step
    int d_qm, d_qp;           // word offset of the x-shift neighbour word (p = 0 / 1)
    int d_ym, d_yp;           // word offsets of the rows y-1 / y+1 (3D)
    uint32_t vmask;           // nibbles of word q that hold sites (ragged rows)
    int sh_next, sh_prev;     // ragged rows: nibble position of the wrapped x neighbour
    uint32_t m_next;

    __device__ __forceinline__ int W() const { return CW > 0 ? CW : g.GW; }

    // Word i of one colour's NR * GW lattice words (checked in bounds-checked
    // builds: an index outside the colour is recorded and the access skipped).
    __device__ __forceinline__ uint32_t ld(const uint32_t* colour, int i, int site) const
    {
        return in_bounds(i, (long long)g.NR * g.GW, site) ? colour[i] : 0u;
    }
    __device__ __forceinline__ void st(uint32_t* colour, int i, uint32_t v, int site) const
    {
        if (in_bounds(i, (long long)g.NR * g.GW, site)) colour[i] = v;
    }
    __device__ __forceinline__ int Ly() const { return D == 2 ? 1 : (CLY > 0 ? CLY : g.Ly); }
    __device__ __forceinline__ int rowW() const { return Ly() * W(); }

    // tid < 0: a thread with no sites (it still takes part in the barriers).
    __device__ __forceinline__ Traj(const Geom& g_, uint32_t* S_, const uint32_t* tab_,
                                    const PhiloxKeys& K_, uint32_t traj, uint32_t c3base_,
                                    int tid, int nthr)
        : g(g_), S(S_), tab(tab_), K(K_), c3base(c3base_)
    {
        const uint64_t p1 = (uint64_t)kPhiloxM1 * traj;
        hi1 = (uint32_t)(p1 >> 32);
        lo1 = (uint32_t)p1;
        const int col = W() * Ly();
        const int slots = nthr / col;   // threads per word column
        TS = CTS > 0 ? CTS : (slots < g.Lt ? slots : g.Lt);
        RS = slots / TS;
        if (tid < 0 || tid / col >= TS * RS) {
            q = y = 0;
            t0 = g.Lt;
            r0 = g.nrep;
        } else {
            q = tid % W();
            y = (tid / W()) % Ly();
            t0 = (tid / col) % TS;
            r0 = (tid / col) / TS;
        }
        d_qm = (q == 0 ? W() - 1 : q - 1) - q;
        d_qp = (q == W() - 1 ? 0 : q + 1) - q;
        d_ym = ((y == 0 ? Ly() - 1 : y - 1) - y) * W();
        d_yp = ((y == Ly() - 1 ? 0 : y + 1) - y) * W();
        const int nv = g.Lh - 8 * q;                       // sites in this word
        const int nv_last = g.Lh - 8 * (W() - 1);          // sites in the row's last word
        vmask = nv >= 8 ? 0xFFFFFFFFu : ((1u << (4 * nv)) - 1u);
        sh_next = 4 * ((nv >= 8 ? 8 : nv) - 1);
        m_next = (1u << sh_next) - 1u;
        sh_prev = q == 0 ? 4 * (nv_last - 1) : 28;
    }

    // Glue mask: nibbles of word q (row parity p) whose site has x < lg.
    __device__ __forceinline__ uint32_t glue_mask(int lg, int p) const
    {
        int nj = ((lg - p + 1) >> 1) - 8 * q;   // # of sites 2h + p < lg in this word
        nj = nj < 0 ? 0 : (nj > 8 ? 8 : nj);
        return nj == 8 ? 0xFFFFFFFFu : ((1u << (4 * nj)) - 1u);
    }

    // The x neighbour not at the same h: h-1 for p = 0, h+1 for p = 1.  Word w
    // of the other colour oth is word q of the row; the row's other words are
    // w + d_qm / w + d_qp.
    __device__ __forceinline__ uint32_t xshift(const uint32_t* oth, int w, int p,
                                               uint32_t nx0) const
    {
        const uint32_t nb = ld(oth, w + (p ? d_qp : d_qm), 6);
        if (FAST) return p ? __funnelshift_r(nx0, nb, 4) : __funnelshift_l(nb, nx0, 4);
        // ragged rows: the row's last word holds fewer than eight sites
        return p ? (((nx0 >> 4) & m_next) | ((nb & 0xFu) << sh_next))
                 : ((nx0 << 4) | ((nb >> sh_prev) & 0xFu));
    }

    // Bulk row, 2 <= t < L_t, all links full beta.  up: offset of the t+1 row
    // (rowW, or -(L_t - 1) rowW at t = L_t - 1); c0: Philox block of the word's
    // first four sites.
    __device__ __forceinline__ void bulk_item(uint32_t* own_b, const uint32_t* oth, int w, int up,
                                              int p, uint32_t c0, uint32_t sweep, uint32_t c3) const
    {
        const uint4 ua = philox_r0(c0, sweep, hi1, lo1, c3, K);
        const uint4 ub = philox_r0(c0 + 1u, sweep, hi1, lo1, c3, K);
        bulk_update(own_b, oth, w, up, p, ua, ub);
    }

    // The same update with the word's two Philox blocks (ua, ub) supplied.
    __device__ __forceinline__ void bulk_update(uint32_t* own_b, const uint32_t* oth, int w, int up,
                                                int p, const uint4& ua, const uint4& ub) const
    {
        const uint32_t own = ld(own_b, w, 1);
        const uint32_t ntm = ld(oth, w - rowW(), 10);
        const uint32_t ntp = ld(oth, w + up, 11);
        const uint32_t nx0 = ld(oth, w, 5);
        const uint32_t nx1 = xshift(oth, w, p, nx0);
        uint32_t dsum = (own ^ ntm) + (own ^ ntp) + (own ^ nx0) + (own ^ nx1);
        if (D == 3) dsum += (own ^ ld(oth, w + d_ym, 7)) + (own ^ ld(oth, w + d_yp, 8));
        uint32_t flip = accept8<D>(dsum, ua, ub, tab);
        if (!FAST) flip &= vmask;
        st(own_b, w, own ^ flip, 9);
    }

    // Site jl of a cut-row word that switches during the protocol: couplings
    // beta (1 - lambda) to its own replica (self_w), beta lambda to the next
    // one (glue_w), tested against step k's table; replaces its flip bit.
    // record: add its share of the work increment dE_k.
    __device__ __forceinline__ void switched_site(uint32_t& flip, int jl, uint32_t own,
                                                  uint32_t self_w, uint32_t glue_w, uint32_t dsum,
                                                  const uint4& ua, const uint4& ub, int k,
                                                  const TeamJob& J, int w_self, int w_glue,
                                                  bool record, int& dE) const
    {
        const int sh = 4 * jl;
        const uint32_t ob = (own >> sh) & 1u;
        const int as = (int)(ob ^ ((self_w >> sh) & 1u));
        const int ag = (int)(ob ^ ((glue_w >> sh) & 1u));
        const int a_cnt = (int)((dsum >> sh) & 0xFu) - as;   // fixed links
        const int a = (2 * D - 1) - 2 * a_cnt;
        const int b = 1 - 2 * as;
        const int cg = 1 - 2 * ag;
        const int mm = a * J.den + b * w_self + cg * w_glue;
        const int ti = (((a + 2 * D - 1) >> 1) * 2 + (b > 0)) * 2 + (cg > 0);
        const bool acc = (mm <= 0) || (word8(ua, ub, jl) < __ldg(J.tcut + k * (8 * D) + ti));
        flip = (flip & ~(0xFu << sh)) | ((uint32_t)acc << sh);
        if (record) dE += b - cg;
    }

    // Row t of replica r (word w, row parity p), a row next to the cut (t = 0,
    // 1) or a bulk row, in one instruction stream: a bulk row's neighbour
    // "across" is its t+1 row with an empty glue mask, and only the switched
    // sites of a cut row (k >= 0: the protocol step, whose table they use)
    // take the per-site loop.  lg = columns glued across the cut.
    __device__ __forceinline__ void row_update(uint32_t* own_b, const uint32_t* oth, int w, int t,
                                               int r, int p, const uint4& ua, const uint4& ub,
                                               int k, int lg, const TeamJob& J, int w_self,
                                               int w_glue, bool record, int& dE) const
    {
        const int Lt = g.Lt;
        const int rw = rowW();
        const int repW = Lt * rw;
        const int n = g.nrep;
        const bool cut = t < 2;
        // the ordinary time neighbour (t - 1; t = 2 for the cut row t = 1)
        const int off_n = t == 0 ? (Lt - 1) * rw : (t == 1 ? (Lt == 2 ? -rw : rw) : -rw);
        // the row across the cut (t = 0, 1), else t + 1
        const int off_x = t == 0 ? rw : t == 1 ? -rw : (t == Lt - 1 ? -(Lt - 1) * rw : rw);
        // the glued partner across the cut: replica r+1 above it, r-1 below (mod n)
        const int off_g = !cut ? 0 : t == 0 ? (r == n - 1 ? -(n - 1) * repW : repW)
                                           : (r == 0 ? (n - 1) * repW : -repW);
        const uint32_t m = cut ? glue_mask(lg, p) : 0u;
        const uint32_t own = ld(own_b, w, 1);
        const uint32_t nrm = ld(oth, w + off_n, 2);
        const uint32_t self_w = ld(oth, w + off_x, 3);
        const uint32_t glue_w = ld(oth, w + off_x + off_g, 4);
        const uint32_t cross = (self_w & ~m) | (glue_w & m);
        const uint32_t nx0 = ld(oth, w, 5);
        const uint32_t nx1 = xshift(oth, w, p, nx0);
        uint32_t dsum = (own ^ nrm) + (own ^ cross) + (own ^ nx0) + (own ^ nx1);
        if (D == 3) dsum += (own ^ ld(oth, w + d_ym, 7)) + (own ^ ld(oth, w + d_yp, 8));
        uint32_t flip = accept8<D>(dsum, ua, ub, tab);
        // Switching sites g0 <= x < g1 during the protocol: couplings
        // beta (1 - lambda) to their own replica, beta lambda to the next one.
        // Site j of the word has x = 2 (8q + j) + p.
        const int jlo = (cut && k >= 0) ? max(((J.g0 - p + 1) >> 1) - 8 * q, 0) : 8;
        const int jhi = min(((J.g1 - p + 1) >> 1) - 8 * q, 8);
#pragma unroll 1
        for (int jl = jlo; jl < jhi; ++jl)
            switched_site(flip, jl, own, self_w, glue_w, dsum, ua, ub, k, J, w_self, w_glue,
                          record, dE);
        if (!FAST) flip &= vmask;
        st(own_b, w, own ^ flip, 9);
    }

    __device__ __forceinline__ void half_sweep(int c, uint32_t sweep, int k, int lg,
                                               const TeamJob& J, int w_self, int w_glue,
                                               bool record, int& dE) const
    {
        const int rw = rowW();
        const int Lt = g.Lt;
        const int cw = g.nrep * Lt * rw;
        uint32_t* own_b = S + c * cw;
        const uint32_t* oth = S + (1 - c) * cw;
        const uint32_t c3 = (uint32_t)c | c3base;
        const int stride = TS * rw;
        const uint32_t cstride = (uint32_t)(TS * Ly() * g.G);   // Philox blocks per TS slices
        const int pc = (c + y) & 1;
        const int wrap_up = -(Lt - 1) * rw;
        if (t0 >= Lt) return;   // a thread without sites
#pragma unroll 1
        for (int r = r0; r < g.nrep; r += RS) {
            int t = t0;
            int w = (r * Lt + t0) * rw + y * W() + q;
            uint32_t c0 = (uint32_t)(((r * Lt + t0) * Ly() + y) * g.G + 2 * q);
            // The thread's first row, cut (t0 < 2) or bulk, in one stream for
            // the whole team; with TS = 1 the team's second row (t = 1) is a
            // cut row too.  The rest are bulk rows.
            do {
                const uint4 ua = philox_r0(c0, sweep, hi1, lo1, c3, K);
                const uint4 ub = philox_r0(c0 + 1u, sweep, hi1, lo1, c3, K);
                row_update(own_b, oth, w, t, r, (pc ^ t) & 1, ua, ub, k, lg, J, w_self, w_glue,
                           record, dE);
                t += TS;
                w += stride;
                c0 += cstride;
            } while (t < 2 && t < Lt);
            if (TS & 1) {
                for (; t < Lt; t += TS, w += stride, c0 += cstride)
                    bulk_item(own_b, oth, w, t == Lt - 1 ? wrap_up : rw, (pc ^ t) & 1, c0, sweep,
                              c3);
            } else {
                // t keeps its parity: the x-shift direction is fixed for the row set.
                // Each row's update runs beside the Philox blocks of the next row
                // (they do not depend on spins), so one warp's instruction stream
                // mixes the wide multiplies with the update's logic; the blocks'
                // round-0 products M0 c0 advance by additions.
                const int p = (pc ^ t0) & 1;
                if constexpr (CLT > 0 && CTS > 0 && CLT % CTS == 0 && CLT / CTS >= 3) {
                    // L_t and the slice step fixed at compile time: the rows
                    // t0 + k CTS, k = 1 .. L_t/CTS - 1, unrolled with immediate
                    // word offsets (no loop or address arithmetic per row)
                    constexpr int NROW = CLT / CTS;
                    constexpr int STR = CTS * (D == 2 ? 1 : CLY) * CW;
                    const int up_last = t0 == CTS - 1 ? wrap_up : rw;
                    uint64_t p0 = (uint64_t)kPhiloxM0 * c0;
                    const uint64_t dp = (uint64_t)kPhiloxM0 * cstride;
                    uint4 ua = philox_p0(p0, sweep, hi1, lo1, c3, K);
                    uint4 ub = philox_p0(p0 + kPhiloxM0, sweep, hi1, lo1, c3, K);
#pragma unroll
                    for (int k = 1; k < NROW - 1; ++k) {
                        p0 += dp;
                        const uint4 na = philox_p0(p0, sweep, hi1, lo1, c3, K);
                        const uint4 nb = philox_p0(p0 + kPhiloxM0, sweep, hi1, lo1, c3, K);
                        bulk_update(own_b, oth, w + (k - 1) * STR, rw, p, ua, ub);
                        ua = na;
                        ub = nb;
                    }
                    bulk_update(own_b, oth, w + (NROW - 2) * STR, up_last, p, ua, ub);
                } else if (t < Lt) {
                    uint64_t p0 = (uint64_t)kPhiloxM0 * c0;
                    const uint64_t dp = (uint64_t)kPhiloxM0 * cstride;
                    uint4 ua = philox_p0(p0, sweep, hi1, lo1, c3, K);
                    uint4 ub = philox_p0(p0 + kPhiloxM0, sweep, hi1, lo1, c3, K);
                    for (; t < Lt - TS; t += TS, w += stride, c0 += cstride) {
                        p0 += dp;
                        const uint4 na = philox_p0(p0, sweep, hi1, lo1, c3, K);
                        const uint4 nb = philox_p0(p0 + kPhiloxM0, sweep, hi1, lo1, c3, K);
                        bulk_update(own_b, oth, w, rw, p, ua, ub);
                        ua = na;
                        ub = nb;
                    }
                    bulk_update(own_b, oth, w, t == Lt - 1 ? wrap_up : rw, p, ua, ub);
                }
            }
        }
    }

    // Threads that own one row of each colour (a team with a thread per word
    // of the lattice): the Philox blocks of half-sweep (sweep, c) of that row.
    // They depend on the sweep index and the colour only, never on spins, so
    // they can be drawn a half-sweep ahead.
    __device__ __forceinline__ void row_draw(uint32_t sweep, int c, uint4& ua, uint4& ub) const
    {
        const uint32_t c0 = (uint32_t)(((r0 * g.Lt + t0) * Ly() + y) * g.G + 2 * q);
        const uint32_t c3 = (uint32_t)c | c3base;
        ua = philox_r0(c0, sweep, hi1, lo1, c3, K);
        ub = philox_r0(c0 + 1u, sweep, hi1, lo1, c3, K);
    }

    // The half-sweep of colour c over this thread's one row, blocks supplied.
    __device__ __forceinline__ void row_half_sweep(int c, const uint4& ua, const uint4& ub, int k,
                                                   int lg, const TeamJob& J, int w_self,
                                                   int w_glue, bool record, int& dE) const
    {
        const int Lt = g.Lt;
        if (t0 >= Lt) return;   // a thread without sites
        const int rw = rowW();
        const int repW = Lt * rw;
        const int n = g.nrep;
        const int w = (r0 * Lt + t0) * rw + y * W() + q;
        row_update(S + c * n * repW, S + (1 - c) * n * repW, w, t0, r0, (c + y + t0) & 1, ua, ub,
                   k, lg, J, w_self, w_glue, record, dE);
    }

    // Loads a stored configuration (int8 +-1, natural order [r][t][y][x]) into
    // this thread's words: site j of word (c, R, q) has x = 2 (8q + j) + p.
    __device__ __forceinline__ void import_spins(const int8_t* src) const
    {
        const int rw = rowW();
        const int cw = g.nrep * g.Lt * rw;
        for (int c = 0; c < 2; ++c) {
            uint32_t* base = S + c * cw;
            for (int r = r0; r < g.nrep; r += RS) {
                int w = (r * g.Lt + t0) * rw + y * W() + q;
                for (int t = t0; t < g.Lt; t += TS, w += TS * rw) {
                    const int p = (c + t + y) & 1;
                    const long long row0 = ((long long)(r * g.Lt + t) * Ly() + y) * g.L;
                    uint32_t v = 0;
                    for (int j = 0; j < 8; ++j) {
                        const int x = 2 * (8 * q + j) + p;
                        if (x < g.L && src[row0 + x] < 0) v |= 1u << (4 * j);
                    }
                    st(base, w, v, 12);
                }
            }
        }
    }

    __device__ __forceinline__ void hot_start() const
    {
        const int rw = rowW();
        const int cw = g.nrep * g.Lt * rw;
        const uint32_t cstride = (uint32_t)(TS * Ly() * g.G);
        for (int c = 0; c < 2; ++c) {
            uint32_t* base = S + c * cw;
            const uint32_t c3 = (uint32_t)c | c3base | (1u << 30);
            for (int r = r0; r < g.nrep; r += RS) {
                int w = (r * g.Lt + t0) * rw + y * W() + q;
                uint32_t c0 = (uint32_t)(((r * g.Lt + t0) * Ly() + y) * g.G + 2 * q);
                for (int t = t0; t < g.Lt; t += TS, w += TS * rw, c0 += cstride) {
                    const uint4 ua = philox_r0(c0, 0u, hi1, lo1, c3, K);
                    const uint4 ub = philox_r0(c0 + 1u, 0u, hi1, lo1, c3, K);
                    const uint32_t v = (ua.x >> 31) | ((ua.y >> 31) << 4) | ((ua.z >> 31) << 8) |
                                       ((ua.w >> 31) << 12) | ((ub.x >> 31) << 16) |
                                       ((ub.y >> 31) << 20) | ((ub.z >> 31) << 24) |
                                       ((ub.w >> 31) << 28);
                    st(base, w, v & vmask, 12);
                }
            }
        }
    }
};

struct CtaBarrier {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct WarpBarrier {
    __device__ __forceinline__ void operator()() const { __syncwarp(); }
};

// Runs one whole trajectory with the team's threads.  Every thread sharing the
// barrier calls it with the same job (trip counts match across teams); tid < 0
// marks a thread without sites.  Returns this thread's share of sum_k dE_k
// (the caller applies the direction's sign and, in protocol 2, the factor L_y
// that makes W = (beta/N) W_int).
// sin: the stored state to start from when J.k_begin > 0 or J.start_in (else unused).
// ROW: every thread owns one row of each colour (the team has a thread per
// word); each half-sweep then draws the next one's Philox blocks beside its
// own update, so the independent chains cover the latency of the
// shared-memory loads and the barrier that a team this small (one warp per
// trajectory, few warps per SM) has no other warps to hide.
template <int D, bool FAST, int CW, int CLY, bool ROW = false, int CLT = 0, int CTS = 0, class Bar>
__device__ __forceinline__ int run_trajectory(const Geom& g, const PhiloxKeys& K, const TeamJob& J,
                                              long long traj, uint32_t* S_team,
                                              const uint32_t* tab, int tid, int nthr, Bar bar,
                                              const int8_t* sin = nullptr)
{
    const Traj<D, FAST, CW, CLY, CLT, CTS> tr(g, S_team, tab, K, (uint32_t)traj,
                                    ((uint32_t)(J.dir < 0) << 1) | ((uint32_t)J.l << 2), tid, nthr);
    int dE = 0;
    // the global sweep index: thermalisation sweeps 0 .. n_therm - 1, then
    // protocol sweep i of step k is n_therm + k n_sweep + i
    const bool resume = J.k_begin > 0 || J.start_in;
    uint32_t s = resume ? (uint32_t)J.n_therm + (uint32_t)J.k_begin * (uint32_t)J.n_sweep : 0u;
    uint4 ua, ub;   // ROW: the blocks of the coming half-sweep
    if constexpr (ROW) tr.row_draw(s, 0, ua, ub);
    auto half = [&](int c, int kk, int lg, int ws, int wg, bool rec) {
        if constexpr (ROW) {
            uint4 na, nb;
            tr.row_draw(c ? s + 1u : s, c ^ 1, na, nb);
            tr.row_half_sweep(c, ua, ub, kk, lg, J, ws, wg, rec, dE);
            ua = na;
            ub = nb;
        } else {
            tr.half_sweep(c, s, kk, lg, J, ws, wg, rec, dE);
        }
        bar();
    };
    if (resume) {
        if (tid >= 0) tr.import_spins(sin);
        bar();
    } else {
        tr.hot_start();
        bar();
        // thermalisation at the start geometry: forward lambda = 0 (x < g0
        // glued), reverse lambda = 1 (x < g1 glued)
        const int lg_therm = J.dir > 0 ? J.g0 : J.g1;
        for (int i = 0; i < J.n_therm; ++i, ++s) {
            half(0, -1, lg_therm, 0, 0, false);
            half(1, -1, lg_therm, 0, 0, false);
        }
    }
    for (int k = J.k_begin; k < J.k_end; ++k) {
        // protocol 2: only column y = k / den moves; the columns before it sit
        // at the end geometry, the ones after it at the start geometry
        const int ya = k / J.den;
        const int kp = k + 1 - ya * J.den;
        const int w_self = J.dir > 0 ? J.den - kp : kp;
        const int w_glue = J.dir > 0 ? kp : J.den - kp;
        int kk = k, lg = J.g0;
        if (J.prot == 2 && tr.y != ya) {
            kk = -1;
            lg = (tr.y < ya) == (J.dir > 0) ? J.g1 : J.g0;
        }
        for (int i = 0; i < J.n_sweep; ++i, ++s) {
            half(0, kk, lg, w_self, w_glue, i == 0);
            half(1, kk, lg, w_self, w_glue, false);
        }
    }
    return dE;
}

// Writes a team's final configuration as int8 +-1 in the order [r][t][y][x].
template <int D>
__device__ __forceinline__ void export_spins(const Geom& g, const uint32_t* S_team, int8_t* dst,
                                             int tid, int nthr)
{
    const int V = g.nrep * g.Lt * g.Ly * g.L;
    for (int i = tid; i < V; i += nthr) {
        const int x = i % g.L;
        const int R = i / g.L;                      // (r, t, y) row
        int y = 0, trow = R;
        if (D == 3) { y = R % g.Ly; trow = R / g.Ly; }
        const int t = trow % g.Lt;
        const int c = (x + y + t) & 1;
        const int h = x >> 1;
        const long long wi = (long long)(c * g.NR + R) * g.GW + (h >> 3);
        const uint32_t word = in_bounds(wi, 2LL * g.NR * g.GW, 13) ? S_team[wi] : 0u;
        dst[i] = ((word >> (4 * (h & 7))) & 1u) ? (int8_t)-1 : (int8_t)1;
    }
}

// ly: L_y of the job's lattice (the number of switched columns).
__device__ __forceinline__ TeamJob team_job(const JobDesc& J, int ly)
{
    TeamJob t;
    t.l = __ldg(&J.l);
    t.n_step = __ldg(&J.n_step);
    t.n_sweep = __ldg(&J.n_sweep);
    t.n_therm = __ldg(&J.n_therm);
    t.dir = __ldg(&J.dir);
    t.prot = __ldg(&J.prot);
    t.k_begin = __ldg(&J.k_begin);
    t.k_end = __ldg(&J.k_end);
    t.start_in = __ldg(&J.start_in);
    t.g0 = __ldg(&J.g0);
    t.g1 = __ldg(&J.g1);
    t.den = t.prot == 2 ? t.n_step / ly : t.n_step;
    t.tcut = J.tcut;
    return t;
}

// This thread's team and team-local id under a launch shape (warp teams do
// not cross warps).  team = -1: no team.
__device__ __forceinline__ void team_of(const LaunchShape& sh, int* team, int* tid)
{
    const int x = (int)threadIdx.x;
    if (!sh.warp) {
        *team = 0;
        *tid = x;
        return;
    }
    const int per_warp = 32 / sh.team_threads;
    const int lane = x & 31;
    const int sub = lane / sh.team_threads;
    if (sub >= per_warp) {
        *team = -1;
        *tid = -1;
        return;
    }
    *team = (x >> 5) * per_warp + sub;
    *tid = lane - sub * sh.team_threads;
}

}  // namespace jz
