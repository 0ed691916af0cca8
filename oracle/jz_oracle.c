/*
 * jz_oracle.c -- plain, slow CPU oracle for the Jarzynski replica-gluing method
 * of Bulgarelli & Panero, "Entanglement entropy from non-equilibrium Monte Carlo
 * simulations" (arXiv:2304.03311).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker, not the product: only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may load
 * it.  It shares no code, header, table or constant generator with the CUDA
 * library; both sides are written from the paper plus the bit-level conventions
 * listed below, each in its own code.
 *
 * What it computes (paper section 3, eq. for H/T of the replica lattice, and
 * Appendix A, eqs. A.1-A.6):
 *   - n = 2 replicas of a periodic L^(d-1) x L_t Ising lattice, H/T = -beta sum s_i s_j
 *     (section 1, eq. Ising_model);
 *   - a cut at time slice tau_c = 0: the temporal link (x, t=0) - (x, t=1) joins
 *     replica r to replica r+1 (mod n) for x < l and stays inside replica r for
 *     x > l (section 3, the "beta^(k,k)" / "beta^(k,k+1)" couplings);
 *   - the column x = l is switched: its self links carry beta (1 - lambda), its
 *     glue links beta lambda, lambda_k = k/N (section 3, linear protocol);
 *   - each trajectory: independent hot start, n_therm checkerboard Metropolis
 *     sweeps at lambda_0 (or Swendsen-Wang sweeps, therm_upd = 1: Appendix A
 *     asks only for an equilibrium start, and section 4 thermalises with
 *     cluster steps), then for k = 0..N-1: accumulate
 *     dW_k = H_{lambda_{k+1}}[phi_k] - H_{lambda_k}[phi_k] (Appendix A, eq.
 *     work_in_one_MC_step) and update with the kernel at lambda_{k+1} (the
 *     remark after eq. discretized_average_exp_work).
 *   The work is kept as the exact integer W_int = sum_k dE_k with
 *   dE_k = sum_{r,y} s^r(l,y,0) [s^r(l,y,1) - s^{r+1}(l,y,1)] so that
 *   W = (beta / N) W_int; the reverse protocol (lambda from 1 to 0, start at
 *   geometry l+1) flips the sign of dE_k.
 *   n replicas (section 2, Z_n / Z^n): the same geometry with the glue of
 *   replica r landing in replica r+1 mod n; Delta S_n = -ln<e^-W>/(n-1).
 *   Whole cut (Alba et al., section 3, eq.
 *   off-equilibrium_evolution_of_the_couplings): every column x < l switches
 *   together from n decoupled replicas to glued ones, so <e^-W> = Z_n(l)/Z^n
 *   and S_n(l) = -ln<e^-W>/(n-1).
 *   Protocol 2 (Appendix B, "protocol 2"; 3D): the L_y switched columns
 *   (x = l, y) are switched one after another, column y during the m = N/L_y
 *   steps y m .. (y+1) m - 1 with its own lambda = (k + 1 - y m)/m; columns
 *   already switched keep the end geometry, the others the start geometry.
 *   Then dE_k sums over the active column only and W_int = L_y sum_k dE_k,
 *   so again W = (beta / N) W_int.  In 2D (L_y = 1) it is protocol 1.
 *
 * Bit-level conventions (not fixed by the paper; shared only as a written
 * contract with the CUDA path, never as code):
 *   colour       c = (x + y + t) mod 2; a sweep updates colour 0 then colour 1.
 *   rows         R = (r * L_t + t) * L_y + y   (L_y = L in 3D, 1 in 2D).
 *   row sites    the sites of colour c in row R are x = 2h + p, p = (c + t + y) mod 2,
 *                h = 0 .. L/2-1; site h uses word (h mod 4) of Philox block q = h/4.
 *   Philox       Philox4x32-10, key = (lo32(seed), hi32(seed)),
 *                counter = (R * G + q, s, traj, c | dir<<1 | l<<2 | phase<<30),
 *                G = ceil((L/2)/4), s = global sweep index (thermalisation sweeps
 *                0..n_therm-1, protocol sweep i of step k: n_therm + k n_sweep + i),
 *                dir = 0 forward / 1 reverse, phase = 0 sweep / 1 hot start (s = 0).
 *   hot start    s_i = +1 if the top bit of its word is 0, else -1.
 *   acceptance   flip iff m <= 0 or u < T, u the site's 32-bit word.
 *                Bulk site: m = s_i sum_j s_j, T = floor(ldexp(exp(-x), 32))
 *                saturated at 2^32 - 1, x = 2.0*beta*(double)m.
 *                Switched site (x = l, t in {0,1}) during the protocol, step k:
 *                a = s_i sum over its 2d-1 full-beta neighbours, b = s_i s_self,
 *                c = s_i s_glue, m = a N + b w_self + c w_glue with
 *                (w_self, w_glue) = (N-k-1, k+1) forward, (k+1, N-k-1) reverse,
 *                x = (2.0*beta*(double)m)/(double)N, same T formula.
 *                During thermalisation the switched column is a bulk site,
 *                self-linked (forward) or glued (reverse).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ORACLE_MUTANT plants one known mistake for the tests that show the pins
 * catch it (0 = the correct oracle; the library is always built with 0):
 *   1 update of step k at lambda_k      2 work taken after the sweeps
 *   3 region A not glued                4 forward start geometry glued at x = l
 *   5 one spatial link dropped          6 sign of the work flipped
 *   7 Boltzmann factor exp(-beta m)
 * and, in the Swendsen-Wang update:
 *   8 bond probability e^-x instead of 1 - e^-x
 *   9 switched bonds of step k at lambda_k
 *  10 each site flips on its own draw instead of its cluster's
 *  11 bonds also between unequal spins
 *  12 glued links of region A stay inside one replica
 * and in protocol 2:
 *  13 the work of the active column not scaled by L_y */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

/* ---------------------------------------------------------------- Philox ---
 * Philox4x32 with 10 rounds, from the definition in Salmon, Moraes, Dror and
 * Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11): each round
 * multiplies counter words 0 and 2 by the two round constants, swaps the high
 * halves across and xors in the counter words 1, 3 and the round key; the key
 * is bumped by the two Weyl constants between rounds. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------ thresholds ---
 * Metropolis acceptance exp(-Delta H / T) with Delta H / T = 2 beta m (bulk) or
 * 2 beta m / N (switched site), quantised to 32 bits: P(u < T) = T / 2^32. */
static uint32_t quantise(double x)
{
    /* floor(2^32 e^-x), saturated at 2^32 - 1 (reached only when e^-x rounds
     * to 1, e.g. beta = 0) */
    double v = floor(ldexp(exp(-x), 32));
    return v >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)v;
}

/* Swendsen-Wang bond probability p = 1 - e^-x for a link of coupling K,
 * x = 2K (Swendsen and Wang, PRL 58 (1987) 86, the paper's ref. for its
 * cluster update), quantised the same way: a bond between equal spins is
 * active iff u < floor(2^32 (1 - e^-x)), saturated at 2^32 - 1. */
static uint32_t quantise_bond(double x)
{
    double v = floor(ldexp(ORACLE_MUTANT == 8 ? exp(-x) : -expm1(-x), 32));
    return v >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)v;
}

uint32_t oracle_bond_threshold(double x) { return quantise_bond(x); }

uint32_t oracle_threshold_bulk(double beta, int m)
{
    if (m <= 0) return 0xFFFFFFFFu; /* never consulted: m <= 0 always flips */
    double x = (ORACLE_MUTANT == 7 ? 1.0 : 2.0) * beta * (double)m;
    return quantise(x);
}

uint32_t oracle_threshold_cut(double beta, long long m, int n_step)
{
    if (m <= 0) return 0xFFFFFFFFu;
    double x = (2.0 * beta * (double)m) / (double)n_step;
    return quantise(x);
}

/* -------------------------------------------------------------- geometry --- */
typedef struct {
    int d, L, Lt, Ly, n;
    int l;        /* the switched column (shift mode) or the cut length (whole) */
    int g0, g1;   /* columns x < g0 are glued, g0 <= x < g1 switch, x >= g1 self */
    int dir;      /* +1 forward (l -> l+1), -1 reverse (l+1 -> l)            */
} geom_t;

static int site_of(const geom_t *g, int r, int t, int y, int x)
{
    return ((r * g->Lt + t) * g->Ly + y) * g->L + x;
}

static int wrap(int v, int n) { return ((v % n) + n) % n; }

/* Classes of a link seen from a site. */
enum { FULL = 0, SELF = 1, GLUE = 2 };

/* State of a switched column's pair of time links across the cut. */
enum { COL_SELF = 0, COL_GLUED = 1, COL_SWITCHING = 2 };

/* Lists the 2d links of site (r,t,y,x): nbr[] = partner site, cls[] = FULL for a
 * beta link, SELF / GLUE for the two switched links of the column x = l.
 * col = the state of the column (x = l, y): COL_SELF or COL_GLUED make it a bulk
 * site linked inside its replica or to the next one, COL_SWITCHING gives it both
 * links.  Returns the number of entries (2d, or 2d+1 for a switched site). */
static int links_of(const geom_t *g, int r, int t, int y, int x, int col,
                    int nbr[8], int cls[8])
{
    int k = 0;
    /* spatial x direction */
    if (ORACLE_MUTANT != 5) {
        nbr[k] = site_of(g, r, t, y, wrap(x - 1, g->L)); cls[k++] = FULL;
    }
    nbr[k] = site_of(g, r, t, y, wrap(x + 1, g->L)); cls[k++] = FULL;
    /* spatial y direction (3D only) */
    if (g->d == 3) {
        nbr[k] = site_of(g, r, t, wrap(y - 1, g->Ly), x); cls[k++] = FULL;
        nbr[k] = site_of(g, r, t, wrap(y + 1, g->Ly), x); cls[k++] = FULL;
    }
    /* temporal links: the link (t, t+1) is the cut link iff t == 0 */
    for (int side = 0; side < 2; ++side) {
        /* side 0: the link below the site (t-1, t); side 1: above (t, t+1) */
        int tn = side == 0 ? wrap(t - 1, g->Lt) : wrap(t + 1, g->Lt);
        int lower_t = side == 0 ? tn : t;      /* time of the link's lower end */
        int is_cut = (lower_t == 0);
        if (!is_cut) {
            nbr[k] = site_of(g, r, tn, y, x); cls[k++] = FULL;
            continue;
        }
        /* across the cut, the glue partner of replica r is replica r+1 above
         * the cut and replica r-1 below it */
        int rg = side == 1 ? wrap(r + 1, g->n) : wrap(r - 1, g->n);
        int self_site = site_of(g, r, tn, y, x);
        int glue_site = site_of(g, rg, tn, y, x);
        if (x < g->g0) {
            nbr[k] = ORACLE_MUTANT == 3 ? self_site : glue_site; cls[k++] = FULL;
        } else if (x >= g->g1) {
            nbr[k] = self_site; cls[k++] = FULL;
        } else if (col == COL_SELF) {
            nbr[k] = self_site; cls[k++] = FULL;
        } else if (col == COL_GLUED) {
            nbr[k] = glue_site; cls[k++] = FULL;
        } else {
            nbr[k] = self_site; cls[k++] = SELF;
            nbr[k] = glue_site; cls[k++] = GLUE;
        }
    }
    return k;
}

/* ------------------------------------------------------------ trajectory --- */
typedef struct {
    geom_t g;
    double beta;
    int n_step, n_sweep, n_therm;
    int prot;             /* 1 all columns together, 2 one column y at a time */
    int m;                /* protocol 2: steps per column, N / L_y; protocol 1: N */
    int update;           /* 0 checkerboard Metropolis, 1 Swendsen-Wang */
    int therm_update;     /* the update of the thermalisation sweeps */
    uint32_t key[2];
    uint32_t bulk_T[8];   /* indexed by m/2 for m = 2, 4, ..., 2d */
    const uint32_t *cut_T; /* [n_step][table], see cut_index() */
    uint32_t bond_full;   /* Swendsen-Wang bond threshold of a full-beta link */
    const uint32_t *bond_self, *bond_glue; /* [n_step] switched links at lambda_{k+1} */
} run_t;

/* The switched-site table of one step is indexed by a (odd, |a| <= 2d-1), b, c. */
static int cut_index(const geom_t *g, int a, int b, int c)
{
    int ia = (a + 2 * g->d - 1) / 2;
    return (ia * 2 + (b > 0)) * 2 + (c > 0);
}

static uint32_t word_for(const run_t *R, int colour, int phase, int sweep,
                         long long traj, int r, int t, int y, int x)
{
    const geom_t *g = &R->g;
    int Lh = g->L / 2;
    int G = (Lh + 3) / 4;
    int row = (r * g->Lt + t) * g->Ly + y;
    int h = x / 2;
    uint32_t ctr[4], out[4];
    ctr[0] = (uint32_t)(row * G + h / 4);
    ctr[1] = (uint32_t)sweep;
    ctr[2] = (uint32_t)traj;
    ctr[3] = (uint32_t)colour | ((uint32_t)(g->dir < 0) << 1) |
             ((uint32_t)g->l << 2) | ((uint32_t)phase << 30);
    oracle_philox4x32_10(ctr, R->key, out);
    return out[h % 4];
}

static int colour_of(int t, int y, int x) { return (x + y + t) & 1; }

/* State of the switched column (x = l, y) at protocol step k (k < 0: the start
 * geometry, lambda = 0 forward / 1 reverse). */
static int column_state(const run_t *R, int y, int k)
{
    const geom_t *g = &R->g;
    if (k < 0) return (g->dir > 0) != (ORACLE_MUTANT == 4) ? COL_SELF : COL_GLUED;
    if (R->prot != 2) return COL_SWITCHING;
    int active = k / R->m;
    if (y == active) return COL_SWITCHING;
    /* columns already switched hold the end geometry, the others the start */
    int at_end = y < active;
    return at_end == (g->dir > 0) ? COL_GLUED : COL_SELF;
}

/* Weights of the switching column at step k, in units of 1/den:
 * lambda_{k+1} = kp/den with kp the step's index inside its column's run. */
static void step_weights(const run_t *R, int k, long long *den, long long *w_self,
                         long long *w_glue)
{
    long long m = R->prot == 2 ? R->m : R->n_step;
    long long kp = (ORACLE_MUTANT == 1 ? k : k + 1) - (long long)(k / m) * m * (R->prot == 2);
    *den = m;
    *w_self = R->g.dir > 0 ? m - kp : kp;
    *w_glue = R->g.dir > 0 ? kp : m - kp;
}

/* One checkerboard sweep at protocol step k (k < 0: thermalisation). */
static void sweep(const run_t *R, int8_t *s, long long traj, int sweep_index, int k)
{
    const geom_t *g = &R->g;
    long long N = 1, w_self = 0, w_glue = 0;   /* step k updates at lambda_{k+1} */
    if (k >= 0) step_weights(R, k, &N, &w_self, &w_glue);
    for (int colour = 0; colour < 2; ++colour) {
        for (int r = 0; r < g->n; ++r)
        for (int t = 0; t < g->Lt; ++t)
        for (int y = 0; y < g->Ly; ++y)
        for (int x = 0; x < g->L; ++x) {
            if (colour_of(t, y, x) != colour) continue;
            int i = site_of(g, r, t, y, x);
            int nbr[8], cls[8];
            int nl = links_of(g, r, t, y, x, column_state(R, y, k), nbr, cls);
            int a = 0, b = 0, c = 0, special = 0;
            for (int j = 0; j < nl; ++j) {
                int prod = s[i] * s[nbr[j]];
                if (cls[j] == FULL) a += prod;
                else if (cls[j] == SELF) { b = prod; special = 1; }
                else { c = prod; special = 1; }
            }
            uint32_t u = word_for(R, colour, 0, sweep_index, traj, r, t, y, x);
            int flip;
            if (!special) {
                int m = a;
                flip = (m <= 0) || (u < R->bulk_T[m / 2]);
            } else {
                long long m = (long long)a * N + b * w_self + c * w_glue;
                const uint32_t *T = R->cut_T + (size_t)k * (size_t)(8 * g->d);
                flip = (m <= 0) || (u < T[cut_index(g, a, b, c)]);
            }
            if (flip) s[i] = (int8_t)(-s[i]);
        }
    }
}

/* ---------------------------------------------------- Swendsen-Wang update --
 * One cluster update of the replica lattice at protocol step k (k < 0:
 * thermalisation at the start geometry), the update the paper's GPU code uses
 * (section 3, GPU paragraph).  Every link with coupling K > 0 between equal
 * spins becomes a bond with probability 1 - e^{-2K}; the clusters of bonded
 * sites are flipped independently with probability 1/2.  Bit-level
 * conventions (shared with the CUDA path only as this written contract):
 *   bonds   the links leaving site i (natural index ((r L_t + t) L_y + y) L + x)
 *           towards +x, +t in the same replica, +y and +t into replica r+1 use
 *           words 0, 1, 2, 3 of Philox block (i, s, traj, dir<<1 | l<<2 | 2<<30);
 *   flips   a cluster's representative is its smallest site index; the
 *           cluster flips iff bit (root & 31) of word (root >> 5) & 3 of Philox
 *           block (root >> 7, s, traj, dir<<1 | l<<2 | 3<<30) is set (one block
 *           holds the flip bits of 128 consecutive sites). */
static int uf_find(int *parent, int a)
{
    while (parent[a] != a) a = parent[a];
    return a;
}

/* joins the clusters of a and b; the smaller root stays the root */
static void uf_union(int *parent, int a, int b)
{
    int ra = uf_find(parent, a), rb = uf_find(parent, b);
    if (ra == rb) return;
    if (ra < rb) parent[rb] = ra; else parent[ra] = rb;
}

static uint32_t philox_word(const run_t *R, uint32_t c0, uint32_t sweep, long long traj,
                            uint32_t phase, int word)
{
    const geom_t *g = &R->g;
    uint32_t ctr[4], out[4];
    ctr[0] = c0;
    ctr[1] = sweep;
    ctr[2] = (uint32_t)traj;
    ctr[3] = ((uint32_t)(g->dir < 0) << 1) | ((uint32_t)g->l << 2) | (phase << 30);
    oracle_philox4x32_10(ctr, R->key, out);
    return out[word];
}

static void sw_sweep(const run_t *R, int8_t *s, int *parent, long long traj, int sweep_index,
                     int k)
{
    const geom_t *g = &R->g;
    const int V = g->n * g->Lt * g->Ly * g->L;
    for (int i = 0; i < V; ++i) parent[i] = i;
    for (int r = 0; r < g->n; ++r)
    for (int t = 0; t < g->Lt; ++t)
    for (int y = 0; y < g->Ly; ++y)
    for (int x = 0; x < g->L; ++x) {
        int i = site_of(g, r, t, y, x);
        /* partners and thresholds of the four forward links */
        int j[4] = {-1, -1, -1, -1};
        uint32_t T[4] = {0, 0, 0, 0};
        j[0] = site_of(g, r, t, y, wrap(x + 1, g->L));
        T[0] = R->bond_full;
        if (g->d == 3) {
            j[2] = site_of(g, r, t, wrap(y + 1, g->Ly), x);
            T[2] = R->bond_full;
        }
        int tn = wrap(t + 1, g->Lt);
        if (t != 0) {
            j[1] = site_of(g, r, tn, y, x);
            T[1] = R->bond_full;
        } else {
            int self_site = site_of(g, r, tn, y, x);
            int glue_site = site_of(g, wrap(r + 1, g->n), tn, y, x);
            if (x >= g->g1) {
                j[1] = self_site; T[1] = R->bond_full;
            } else if (x < g->g0) {
                j[3] = ORACLE_MUTANT == 12 ? self_site : glue_site; T[3] = R->bond_full;
            } else if (column_state(R, y, k) == COL_SELF) {
                j[1] = self_site; T[1] = R->bond_full;
            } else if (column_state(R, y, k) == COL_GLUED) {
                j[3] = glue_site; T[3] = R->bond_full;
            } else {
                j[1] = self_site; T[1] = R->bond_self[k];
                j[3] = glue_site; T[3] = R->bond_glue[k];
            }
        }
        for (int w = 0; w < 4; ++w) {
            if (j[w] < 0 || (s[i] != s[j[w]] && ORACLE_MUTANT != 11)) continue;
            if (philox_word(R, (uint32_t)i, (uint32_t)sweep_index, traj, 2, w) < T[w])
                uf_union(parent, i, j[w]);
        }
    }
    for (int i = 0; i < V; ++i) {
        int root = ORACLE_MUTANT == 10 ? i : uf_find(parent, i);
        uint32_t word = philox_word(R, (uint32_t)(root >> 7), (uint32_t)sweep_index, traj, 3,
                                    (root >> 5) & 3);
        if ((word >> (root & 31)) & 1u)
            s[i] = (int8_t)(-s[i]);
    }
}

/* dE_k = H_{lambda_{k+1}} - H_{lambda_k} on the current configuration, in
 * units of beta / N (Appendix A, eq. work_in_one_MC_step): every column moves
 * by 1/N in protocol 1; in protocol 2 only the active column moves, by
 * 1/m = L_y/N. */
static long long work_increment(const run_t *R, const int8_t *s, int k)
{
    const geom_t *g = &R->g;
    long long e = 0;
    for (int r = 0; r < g->n; ++r)
    for (int y = 0; y < g->Ly; ++y)
    for (int x = g->g0; x < g->g1; ++x) {
        if (R->prot == 2 && y != k / R->m) continue;
        int lo = site_of(g, r, 0, y, x);
        int up_self = site_of(g, r, 1, y, x);
        int up_glue = site_of(g, wrap(r + 1, g->n), 1, y, x);
        e += (long long)s[lo] * (s[up_self] - s[up_glue]);
    }
    if (R->prot == 2 && ORACLE_MUTANT != 13) e *= g->Ly;
    return (g->dir > 0) != (ORACLE_MUTANT == 6) ? e : -e;
}

static void hot_start(const run_t *R, int8_t *s, long long traj)
{
    const geom_t *g = &R->g;
    for (int r = 0; r < g->n; ++r)
    for (int t = 0; t < g->Lt; ++t)
    for (int y = 0; y < g->Ly; ++y)
    for (int x = 0; x < g->L; ++x) {
        uint32_t u = word_for(R, colour_of(t, y, x), 1, 0, traj, r, t, y, x);
        s[site_of(g, r, t, y, x)] = (u >> 31) ? -1 : 1;
    }
}

static void update(const run_t *R, int upd, int8_t *s, int *parent, long long traj,
                   int sweep_index, int k)
{
    if (upd == 1) sw_sweep(R, s, parent, traj, sweep_index, k);
    else sweep(R, s, traj, sweep_index, k);
}

static long long run_trajectory(const run_t *R, long long traj, int8_t *s, int *parent)
{
    hot_start(R, s, traj);
    for (int i = 0; i < R->n_therm; ++i) update(R, R->therm_update, s, parent, traj, i, -1);
    long long w = 0;
    for (int k = 0; k < R->n_step; ++k) {
        if (ORACLE_MUTANT != 2) w += work_increment(R, s, k);
        for (int i = 0; i < R->n_sweep; ++i)
            update(R, R->update, s, parent, traj, R->n_therm + k * R->n_sweep + i, k);
        if (ORACLE_MUTANT == 2) w += work_increment(R, s, k);
    }
    return w;
}

/* ------------------------------------------------------------- entry point --
 * Runs trajectories traj0 .. traj0+n_traj-1 of one transformation l -> l+1
 * (dir = +1) or l+1 -> l (dir = -1).  work_out[i] = W_int of trajectory
 * traj0 + i; spins_out (nullable) receives the final configuration of each
 * trajectory as int8 +-1 in the natural order [traj][r][t][y][x].
 * upd selects the update (0 Metropolis, 1 Swendsen-Wang), prot the protocol
 * (1 all switched columns together, 2 one column at a time; n_step must then be
 * a multiple of L_y).  n_rep >= 2 is the number of replicas n.  whole = 0: the
 * transformation moves the end of region A by one column (x < l glued, column
 * l switching); whole = 1: Alba et al.'s whole-cut transformation from n
 * decoupled replicas to replicas glued along x < l (columns 0 .. l-1 switching,
 * 1 <= l <= L; section 3, eq. off-equilibrium_evolution_of_the_couplings).
 * therm_upd selects the update of the thermalisation sweeps (0 Metropolis, 1
 * Swendsen-Wang).  n_threads > 0 sets the OpenMP thread count (trajectories are
 * independent, so the result does not depend on it).  Returns 0, or -1 on bad
 * arguments. */
int oracle_run_therm(int d, int L, int Lt, double beta, int l, int n_step, int n_sweep,
                     int n_therm, int dir, int upd, int therm_upd, int prot, int n_rep,
                     int whole, uint64_t seed, long long traj0, int n_traj, int n_threads,
                     long long *work_out, int8_t *spins_out)
{
    if ((d != 2 && d != 3) || L < 2 || Lt < 2 || (L & 1) || (Lt & 1)) return -1;
    if (upd != 0 && upd != 1) return -1;
    if (therm_upd != 0 && therm_upd != 1) return -1;
    if (prot != 1 && prot != 2) return -1;
    if (n_rep < 2 || n_rep > 16 || (whole != 0 && whole != 1)) return -1;
    if (whole ? (l < 1 || l > L || prot != 1) : (l < 0 || l >= L)) return -1;
    if (n_step < 1 || n_sweep < 0 || n_therm < 0) return -1;
    if (dir != 1 && dir != -1) return -1;
    run_t R;
    memset(&R, 0, sizeof R);
    R.g.d = d; R.g.L = L; R.g.Lt = Lt; R.g.Ly = d == 3 ? L : 1; R.g.n = n_rep;
    R.g.l = l; R.g.dir = dir;
    R.g.g0 = whole ? 0 : l;
    R.g.g1 = whole ? l : l + 1;
    if (prot == 2 && n_step % R.g.Ly != 0) return -1;
    R.prot = prot;
    R.m = prot == 2 ? n_step / R.g.Ly : n_step;
    R.beta = beta; R.n_step = n_step; R.n_sweep = n_sweep; R.n_therm = n_therm;
    R.key[0] = (uint32_t)seed; R.key[1] = (uint32_t)(seed >> 32);
    for (int m = 2; m <= 2 * d; m += 2) R.bulk_T[m / 2] = oracle_threshold_bulk(beta, m);
    int per_step = 8 * d;
    uint32_t *cut = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n_step * per_step);
    if (!cut) return -1;
    for (int k = 0; k < n_step; ++k) {
        long long den, w_self, w_glue;
        step_weights(&R, k, &den, &w_self, &w_glue);
        for (int a = -(2 * d - 1); a <= 2 * d - 1; a += 2)
        for (int b = -1; b <= 1; b += 2)
        for (int c = -1; c <= 1; c += 2) {
            long long m = (long long)a * den + b * w_self + c * w_glue;
            cut[(size_t)k * per_step + cut_index(&R.g, a, b, c)] =
                oracle_threshold_cut(beta, m, (int)den);
        }
    }
    R.cut_T = cut;
    /* Swendsen-Wang bond thresholds: full links x = 2 beta, switched links at
     * step k: x = (2 beta w)/den with w = w_self or w_glue of lambda_{k+1} */
    R.update = upd;
    R.therm_update = therm_upd;
    R.bond_full = quantise_bond(2.0 * beta);
    uint32_t *bonds = (uint32_t *)malloc(sizeof(uint32_t) * 2 * (size_t)n_step);
    if (!bonds) { free(cut); return -1; }
    for (int k = 0; k < n_step; ++k) {
        long long den, w_self, w_glue;
        step_weights(&R, k, &den, &w_self, &w_glue);
        if (ORACLE_MUTANT == 9) { w_self += dir; w_glue -= dir; }   /* lambda_k */
        bonds[k] = quantise_bond((2.0 * beta * (double)w_self) / (double)den);
        bonds[n_step + k] = quantise_bond((2.0 * beta * (double)w_glue) / (double)den);
    }
    R.bond_self = bonds;
    R.bond_glue = bonds + n_step;
    int V = n_rep * L * Lt * R.g.Ly;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    int failed = 0;
#pragma omp parallel
    {
        int8_t *s = (int8_t *)malloc((size_t)V);
        int *parent = (int *)malloc(sizeof(int) * (size_t)V);
        if (!s || !parent) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int i = 0; i < n_traj; ++i) {
            if (!s || !parent) continue;
            work_out[i] = run_trajectory(&R, traj0 + i, s, parent);
            if (spins_out) memcpy(spins_out + (size_t)i * V, s, (size_t)V);
        }
        free(s);
        free(parent);
    }
    free(cut);
    free(bonds);
    return failed ? -1 : 0;
}

/* Thermalisation with the protocol's own update. */
int oracle_run_general(int d, int L, int Lt, double beta, int l, int n_step, int n_sweep,
                       int n_therm, int dir, int upd, int prot, int n_rep, int whole,
                       uint64_t seed, long long traj0, int n_traj, int n_threads,
                       long long *work_out, int8_t *spins_out)
{
    return oracle_run_therm(d, L, Lt, beta, l, n_step, n_sweep, n_therm, dir, upd, upd, prot,
                            n_rep, whole, seed, traj0, n_traj, n_threads, work_out, spins_out);
}

/* Two replicas, shift mode. */
int oracle_run_full(int d, int L, int Lt, double beta, int l, int n_step, int n_sweep,
                    int n_therm, int dir, int upd, int prot, uint64_t seed, long long traj0,
                    int n_traj, int n_threads, long long *work_out, int8_t *spins_out)
{
    return oracle_run_general(d, L, Lt, beta, l, n_step, n_sweep, n_therm, dir, upd, prot, 2, 0,
                              seed, traj0, n_traj, n_threads, work_out, spins_out);
}

/* Protocol 1 of oracle_run_full. */
int oracle_run_update(int d, int L, int Lt, double beta, int l, int n_step, int n_sweep,
                      int n_therm, int dir, int upd, uint64_t seed, long long traj0, int n_traj,
                      int n_threads, long long *work_out, int8_t *spins_out)
{
    return oracle_run_full(d, L, Lt, beta, l, n_step, n_sweep, n_therm, dir, upd, 1, seed,
                           traj0, n_traj, n_threads, work_out, spins_out);
}

/* The Metropolis form (update 0) of oracle_run_update. */
int oracle_run(int d, int L, int Lt, double beta, int l, int n_step, int n_sweep,
               int n_therm, int dir, uint64_t seed, long long traj0, int n_traj,
               int n_threads, long long *work_out, int8_t *spins_out)
{
    return oracle_run_update(d, L, Lt, beta, l, n_step, n_sweep, n_therm, dir, 0, seed, traj0,
                             n_traj, n_threads, work_out, spins_out);
}

/* Number of OpenMP threads a parallel region would use (1 without OpenMP). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
