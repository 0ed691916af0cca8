// jz_api.cu -- the C ABI (include/isingjz.h): argument checks, host FP64
// threshold tables, device buffers, launch grouping, estimator.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/isingjz.h"
#include "jz_device.cuh"

#include "jz_host.h"

static_assert(sizeof(jz_params) == 80, "jz_params layout is part of the ABI");

namespace jzh {

int ensure(ising_ctx* ctx, DevBuf& b, size_t bytes)
{
    if (bytes <= b.bytes) return ISING_OK;
    size_t want = bytes + bytes / 4;
    size_t delta = want - b.bytes;
    if (ctx->budget && ctx->used + delta > ctx->budget) {
        want = bytes;
        delta = want - b.bytes;
        if (ctx->used + delta > ctx->budget) return ISING_ERR_NOMEM;
    }
    if (b.ptr) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(b.ptr);
        ctx->used -= b.bytes;
        b.ptr = nullptr;
        b.bytes = 0;
    }
    if (cudaMalloc(&b.ptr, want) != cudaSuccess) {
        cudaGetLastError();
        return ISING_ERR_NOMEM;
    }
    b.bytes = want;
    ctx->used += want;
    return ISING_OK;
}

// 1 if p is device-accessible memory of the current device (device or
// managed allocation), 0 for host memory (pageable or pinned).
int is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int check_params(const jz_params* p)
{
    if (!p) return ISING_ERR_ARG;
    if (p->d != 2 && p->d != 3) return ISING_ERR_UNSUPPORTED;
    if (p->update != 0 && p->update != 1) return ISING_ERR_ARG;
    if (p->protocol < 0 || p->protocol > 2) return ISING_ERR_ARG;
    if (p->protocol == 2 && p->d == 3 && p->n_step % p->L != 0) return ISING_ERR_ARG;
    if (p->L < 2 || p->L_t < 2 || p->L > 4096 || p->L_t > 4096) return ISING_ERR_ARG;
    if ((p->L & 1) || (p->L_t & 1)) return ISING_ERR_ODD_EXTENT;
    if (p->n_replica != 0 && (p->n_replica < 2 || p->n_replica > 8)) return ISING_ERR_ARG;
    if (p->whole != 0 && p->whole != 1) return ISING_ERR_ARG;
    if (p->whole ? (p->l < 1 || p->l > p->L) : (p->l < 0 || p->l > p->L - 1))
        return ISING_ERR_L_RANGE;
    if (p->whole && p->protocol == 2) return ISING_ERR_ARG;
    if (p->therm_update != 0 && p->therm_update != 1) return ISING_ERR_ARG;
    if (p->n_step < 1 || p->n_sweep < 1 || p->n_therm < 0 || p->n_traj < 1)
        return ISING_ERR_ARG;
    if (p->direction != 1 && p->direction != -1) return ISING_ERR_ARG;
    if (!(p->beta >= 0.0 && p->beta <= 4.0)) return ISING_ERR_ARG;
    if (p->traj0 < 0 || p->traj0 + p->n_traj > 0x100000000LL) return ISING_ERR_ARG;
    // the global sweep index is a 32-bit counter word
    long long sweeps = (long long)p->n_therm + (long long)p->n_step * p->n_sweep;
    if (sweeps >= 0x100000000LL) return ISING_ERR_ARG;
    // m = a N + b w_self + c w_glue must fit an int: |m| <= (2d+1) N
    if ((long long)p->n_step * (2 * p->d + 1) >= 0x7FFFFFFFLL) return ISING_ERR_ARG;
    // |W_int| <= N * 2 n L_y (switching columns), accumulated in an int
    const long long ly = p->d == 3 ? p->L : 1;
    const long long cols = p->whole ? p->l : 1;
    if ((long long)p->n_step * 2 * nrep_of(*p) * ly * cols * (p->protocol == 2 ? ly : 1) >=
        0x7FFFFFFFLL)
        return ISING_ERR_ARG;
    return ISING_OK;
}

int nrep_of(const jz_params& p) { return p.n_replica == 0 ? 2 : p.n_replica; }

// Whether p thermalises with Swendsen-Wang clusters before a Metropolis
// protocol (with no thermalisation sweeps the two are the same run).
bool sw_therm(const jz_params& p) { return p.update == 0 && p.therm_update == 1 && p.n_therm > 0; }

// Switching columns of a job: [l, l+1) when the end of region A moves by one
// column, [0, l) for the whole-cut transformation.
void cut_range(const jz_params& p, int* g0, int* g1)
{
    *g0 = p.whole ? 0 : p.l;
    *g1 = p.whole ? p.l : p.l + 1;
}

jz::Geom make_geom(int d, int L, int Lt, int nrep)
{
    jz::Geom g;
    g.L = L;
    g.Lt = Lt;
    g.Ly = d == 3 ? L : 1;
    g.Lh = L / 2;
    g.G = (g.Lh + 3) / 4;
    g.GW = (g.Lh + 7) / 8;
    g.nrep = nrep;
    g.NR = nrep * Lt * g.Ly;
    return g;
}

// Threshold T = min(floor(2^32 exp(-x)), 2^32 - 1): a site whose energy cost
// m > 0 flips with probability T / 2^32.
uint32_t threshold(double x)
{
    double v = std::floor(std::ldexp(std::exp(-x), 32));
    return v >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)v;
}

jz::PhiloxKeys key_schedule(uint64_t seed)
{
    jz::PhiloxKeys K;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int i = 0; i < 10; ++i) {
        K.k0[i] = k0;
        K.k1[i] = k1;
        k0 += jz::kPhiloxW0;
        k1 += jz::kPhiloxW1;
    }
    return K;
}

// Host tables of one job: bulk thresholds by anti-aligned count a (m = 2D - 2a,
// x = 2 beta m) and, per step k, the switched-site thresholds indexed by the
// fixed-link sum a' (odd, |a'| <= 2D-1) and the self / glue bond products b, c
// (m = a' den + b w_self + c w_glue, x = (2 beta m) / den, den = N in protocol 1
// and N / L_y in protocol 2).
void build_tables_into(const jz_params& p, uint32_t tb[4], uint32_t* tcut)
{
    const int D = p.d;
    for (int a = 0; a < 4; ++a) {
        int m = 2 * D - 2 * a;
        tb[a] = (a < D) ? threshold(2.0 * p.beta * (double)m) : 0xFFFFFFFFu;
    }
    const int per = 8 * D;
    for (long long k = 0; k < p.n_step; ++k) {
        long long N, ws, wg;
        step_weights(p, k, &N, &ws, &wg);
        for (int ia = 0; ia < 2 * D; ++ia) {
            const long long a = 2 * ia - (2 * D - 1);
            for (int ib = 0; ib < 2; ++ib)
                for (int ic = 0; ic < 2; ++ic) {
                    const long long m = a * N + (ib ? ws : -ws) + (ic ? wg : -wg);
                    uint32_t T = 0xFFFFFFFFu;
                    if (m > 0) T = threshold((2.0 * p.beta * (double)m) / (double)N);
                    tcut[(size_t)k * per + (ia * 2 + ib) * 2 + ic] = T;
                }
        }
    }
}

void build_tables(const jz_params& p, uint32_t tb[4], std::vector<uint32_t>& tcut, size_t off)
{
    build_tables_into(p, tb, tcut.data() + off);
}

// Couplings of the switching column at protocol step k, in units of 1/den:
// lambda_{k+1} = kp/den.  Protocol 1: den = N, kp = k+1.  Protocol 2: den =
// m = N/L_y and kp = k+1 - y m counts the steps of the active column y = k/m.
void step_weights(const jz_params& p, long long k, long long* den, long long* w_self,
                  long long* w_glue)
{
    const long long ly = p.d == 3 ? p.L : 1;
    const long long m = p.protocol == 2 ? p.n_step / ly : p.n_step;
    const long long kp = k + 1 - (k / m) * m;
    *den = m;
    *w_self = p.direction > 0 ? m - kp : kp;
    *w_glue = p.direction > 0 ? kp : m - kp;
}

// Swendsen-Wang bond threshold of a link with x = 2K: a bond between equal
// spins is active iff u < min(floor(2^32 (1 - e^{-x})), 2^32 - 1), i.e. with
// probability 1 - e^{-x} to 2^-32 (Swendsen and Wang, PRL 58 (1987) 86).
uint32_t bond_threshold(double x)
{
    double v = std::floor(std::ldexp(-std::expm1(-x), 32));
    return v >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)v;
}

// Swendsen-Wang tables of one job: tb[0] the full link (x = 2 beta); per step
// k the switching column's self and glued links at lambda_{k+1}:
// x = (2 beta w) / den with w = w_self, w_glue.
void build_bond_tables_into(const jz_params& p, uint32_t tb[4], uint32_t* tcut)
{
    tb[0] = bond_threshold(2.0 * p.beta);
    tb[1] = tb[2] = tb[3] = 0;
    for (long long k = 0; k < p.n_step; ++k) {
        long long den, ws, wg;
        step_weights(p, k, &den, &ws, &wg);
        tcut[2 * k] = bond_threshold((2.0 * p.beta * (double)ws) / (double)den);
        tcut[2 * k + 1] = bond_threshold((2.0 * p.beta * (double)wg) / (double)den);
    }
}

void build_bond_tables(const jz_params& p, uint32_t tb[4], std::vector<uint32_t>& tcut,
                       size_t off)
{
    build_bond_tables_into(p, tb, tcut.data() + off);
}

// Whether a Swendsen-Wang trajectory of lattice g fits one CTA's shared memory.
bool sw_fits(const jz::Geom& g)
{
    return jz::sw_smem_bytes(g) <= jz::kMaxSmemPerCta;
}

// Launch shape for lattices g in CTAs of cta_threads (0: the base layout
// that default_shape starts from, and the layout of lattices in HBM).  With
// col = GW * L_y words per time slice, each thread owns one word column of
// every TS-th slice.  col <= 32: warp teams of col * TS threads, TS =
// min(32 / col, L_t), as many per CTA as fit (default CTA 128 threads).
// Wider slices, and narrow ones whose lattice leaves room for fewer than four
// warp teams: the CTA is one team of col * TS threads, TS <= L_t (default
// about 256 threads, at most 512).  Teams per CTA stay <= 64 and within the
// per-CTA shared memory.
jz::LaunchShape shape_for(const jz::Geom& g, int cta_threads)
{
    jz::LaunchShape s{};
    const int col = g.GW * g.Ly;
    const size_t lat = jz::traj_smem_bytes(g);
    // narrow slices whose lattices are so large that fewer than four warp
    // teams fit a CTA's shared memory (or none: lattices in HBM) run as one
    // CTA team instead, so the SM still has several warps per lattice
    const size_t fit = jz::kMaxSmemPerCta / lat;
    const bool big = col <= 32 && 32 % col == 0 && fit < 4 && g.Lt * col > 32;
    if (col <= 32 && !big) {
        int ts = 32 / col;
        if (ts > g.Lt) ts = g.Lt;
        // a whole time column per thread slot leaves room in the warp: split
        // the replicas over more slots (more warps per trajectory, the same
        // lanes in use), rs a power of two dividing n
        int rs = 1;
        if (ts == g.Lt && 32 % (col * ts) == 0)
            for (int r = 2; col * ts * r <= 32 && r <= g.nrep; r *= 2)
                if (g.nrep % r == 0) rs = r;
        s.team_threads = col * ts * rs;
        s.warp = 1;
        const int per_warp = 32 / s.team_threads;
        int warps = (cta_threads > 0 ? cta_threads : 128) / 32;
        if (warps < 1) warps = 1;
        while (warps > 1 && ((size_t)warps * per_warp * lat > jz::kMaxSmemPerCta ||
                             warps * per_warp > jz::kMaxTeamsHost))
            --warps;
        s.teams = warps * per_warp;
        s.cta_threads = warps * 32;
    } else {
        // lattices in HBM wait on L2 and take the widest team by default
        // (3D L = 48, L_t = 4L: 432 threads 9.3e11, 144 threads 6.7e11)
        const bool in_hbm = lat > jz::kMaxSmemPerCta;
        int ts = (cta_threads > 0 ? cta_threads : (in_hbm ? 512 : 256)) / col;
        if (ts < 1) ts = 1;
        if (cta_threads == 0 && !in_hbm && ts > 1 && (ts & 1)) ts -= 1;
        if (ts > g.Lt) ts = g.Lt;
        while (ts > 1 && col * ts > 512) --ts;
        s.team_threads = col * ts;
        s.teams = 1;
        s.cta_threads = s.team_threads;
        s.warp = 0;
    }
    return s;
}

// The relative rate of a launch of shape sh over n_traj trajectories of g
// (n_traj <= 0: enough to fill every SM), fitted to rates measured on GB300
// for every layout of 2D L = 34 .. 256 and 3D L = 8 .. 48 (L_t = L) at 256,
// 2048 and 8192 trajectories:
//   min(active warps per SM, kSatWarps) x (fraction of lanes owning a word)
//   x R / (R + kBarrierRows) for one team per CTA,
// where active warps are the resident ones (CUDA occupancy of the kernel
// that runs g) or fewer when the trajectories do not fill the SMs, and R is
// a thread's rows per half-sweep: a CTA team drains at its barrier, a warp
// team's __syncwarp costs next to nothing.  Negative when sh cannot launch.
constexpr double kSatWarps = 16.0;     // the integer pipes are saturated from here on
constexpr double kBarrierRows = 1.5;   // a CTA barrier costs about 1.5 rows of work
double shape_score(int d, const jz::Geom& g, const jz::LaunchShape& sh, long long n_traj,
                   int n_sm)
{
    if (sh.cta_threads <= 0 || sh.cta_threads > 512 || sh.teams < 1) return -1.0;
    if ((size_t)sh.teams * jz::traj_smem_bytes(g) > jz::kMaxSmemPerCta) return -1.0;
    int ctas = 0;
    if (jz::traj_occupancy(d, g, sh, &ctas) != cudaSuccess) {
        cudaGetLastError();
        return -1.0;
    }
    if (ctas < 1) return -1.0;
    const int wc = (sh.cta_threads + 31) / 32;
    double warps = (double)ctas * wc;
    if (n_traj > 0) {
        const long long n_cta = (n_traj + sh.teams - 1) / sh.teams;
        warps = std::min(warps, (double)n_cta * wc / n_sm);
    }
    const double lanes = (double)sh.teams * sh.team_threads / (32.0 * wc);
    double sc = std::min(warps, kSatWarps) * lanes;
    if (!sh.warp) {
        const int ts = std::max(1, std::min(sh.team_threads / (g.GW * g.Ly), g.Lt));
        const double rows = (double)g.nrep * g.Lt / ts;
        sc *= rows / (rows + kBarrierRows);
    }
    return sc;
}

// The shape a lattice in shared memory runs with when no CTA size is fixed.
// Candidates: the warp-team layouts of shape_for for CTAs of 32 ... 512
// threads, and one team per CTA for every slice step TS (col * TS <= 512).
// shape_for(g, 0) is kept unless another candidate scores kKeepMargin more
// (shape_score).  On the measured layouts this picks within about 2 % of the
// fastest one on average and runs 1.39x the rate of shape_for(g, 0): narrow
// slices of large lattices (2D L ~ 130 .. 240 with L_t = L), whose warp
// teams each hold a whole lattice of shared memory and leave an SM four
// warps, gain 1.4 - 1.9x as CTA teams; small jobs, whose trajectories fill
// more SMs when each has more threads, 2 - 3x.  Lattices in HBM keep
// shape_for(g, 0).
constexpr double kKeepMargin = 1.05;
jz::LaunchShape default_shape(int d, const jz::Geom& g, long long n_traj)
{
    const jz::LaunchShape base = shape_for(g, 0);
    if (jz::traj_smem_bytes(g) > jz::kMaxSmemPerCta) return base;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        n_sm < 1) {
        cudaGetLastError();
        return base;
    }
    const double s0 = shape_score(d, g, base, n_traj, n_sm);
    jz::LaunchShape best = base;
    double best_s = s0 * kKeepMargin;
    auto consider = [&](const jz::LaunchShape& sh) {
        const double sc = shape_score(d, g, sh, n_traj, n_sm);
        if (sc > best_s) {
            best_s = sc;
            best = sh;
        }
    };
    const int col = g.GW * g.Ly;
    if (col <= 32)
        for (int t = 32; t <= 512; t *= 2) consider(shape_for(g, t));
    // one team per CTA: for w = 1 .. 16 warps the largest slice step that
    // fits them, and the even step below it; a CTA team has at least a warp
    // of threads (its first eight fill the shared threshold table)
    int last = 0;
    for (int w = 1; w <= 16; ++w) {
        const int top = std::min(32 * w / col, g.Lt);
        for (int ts = top; ts >= 1 && ts >= top - 1; --ts) {
            if (ts == last || col * ts < 32) continue;
            jz::LaunchShape sh{};
            sh.team_threads = col * ts;
            sh.teams = 1;
            sh.cta_threads = col * ts;
            sh.warp = 0;
            consider(sh);
        }
        last = top;
    }
    return best;
}

// Whether one time slice of words fits a CTA of 512 threads (any lattice
// satisfying this runs, with its lattice in HBM if not in shared memory).
bool threads_fit(const jz::Geom& g) { return g.GW * g.Ly <= 512; }

// Whether g runs with its lattice in shared memory: one team's lattice fits a
// CTA's shared memory and one time slice of words fits 512 threads.
bool shape_fits(const jz::Geom& g)
{
    return jz::traj_smem_bytes(g) <= jz::kMaxSmemPerCta && threads_fit(g);
}

// A CTA size is admissible: a multiple of 32 for warp teams, col * TS with
// TS <= L_t for CTA teams; at most 512 threads.
bool threads_ok(const jz::Geom& g, int threads)
{
    const int col = g.GW * g.Ly;
    if (threads <= 0 || threads > 512) return false;
    if (col <= 32) return threads % 32 == 0;
    return threads % col == 0 && threads / col <= g.Lt;
}

// The context's launch shape for this lattice: the tuned / fixed CTA size,
// else the default for a launch of n_traj trajectories.
jz::LaunchShape ctx_shape(ising_ctx* ctx, int d, const jz::Geom& g, long long n_traj)
{
    const auto key = std::make_tuple(d, g.L, g.Lt, g.nrep, n_traj);
    {
        std::lock_guard<std::mutex> lk(ctx->shapes_mu);
        auto it = ctx->threads.find(std::make_tuple(d, g.L, g.Lt));
        const int t = (it != ctx->threads.end() && threads_ok(g, it->second)) ? it->second : 0;
        if (t) return shape_for(g, t);
        auto c = ctx->default_shapes.find(key);
        if (c != ctx->default_shapes.end()) return c->second;
    }
    // scored without the lock (occupancy queries); a concurrent caller may
    // score the same key, with the same result
    const jz::LaunchShape sh = default_shape(d, g, n_traj);
    std::lock_guard<std::mutex> lk(ctx->shapes_mu);
    if (ctx->default_shapes.size() >= 4096) ctx->default_shapes.clear();
    ctx->default_shapes[key] = sh;
    return sh;
}

int cuda_err(cudaError_t e)
{
    if (e == cudaSuccess) return ISING_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? ISING_ERR_NOMEM : ISING_ERR_CUDA;
}

// Runs jobs[idx[0..]] (equal d, L, L_t, seed) in one launch.
int run_group(ising_ctx* ctx, const jz_params* jobs, const std::vector<int>& idx,
              int64_t* const* outs, int8_t* const* spins, bool outs_on_device,
              bool spins_on_device, const Segment* seg)
{
    const jz_params& p0 = jobs[idx[0]];
    const jz::Geom g = make_geom(p0.d, p0.L, p0.L_t, nrep_of(p0));
    const bool sw = p0.update == 1;   // Swendsen-Wang: one trajectory per CTA
    if (!sw && !threads_fit(g)) return ISING_ERR_UNSUPPORTED;
    // lattices beyond shared memory run from HBM, one slice per CTA
    const bool in_hbm = sw ? !sw_fits(g) : !shape_fits(g);
    // Swendsen-Wang thermalisation before a Metropolis protocol run from k = 0:
    // thermalisation-only sw_kernel launches leave every trajectory's spins in
    // ctx->therm, from which the Metropolis protocol starts.  A Swendsen-Wang
    // state beyond shared memory is thermalised from HBM slices, one resident
    // wave of trajectories (a chunk) per launch, so its HBM state stays one
    // wave whatever the trajectory count.
    const bool hybrid = sw_therm(p0) && (!seg || seg->k_begin == 0);
    const bool therm_hbm = hybrid && !sw_fits(g);
    const long long chunk = therm_hbm ? jz::sw_hbm_wave(p0.d) : 0;
    // HBM thermalisation launches: descriptors [first, first + n_desc) of the
    // job table (pieces of consecutive jobs, CTAs numbered within the wave)
    struct ThermWave {
        size_t first, n_desc;
        long long n_cta;
    };
    std::vector<ThermWave> therm_waves;
    long long n_traj_launch = 0;
    for (int j : idx) n_traj_launch += jobs[j].n_traj;
    jz::LaunchShape sh = sw ? shape_for(g, 0) : ctx_shape(ctx, p0.d, g, n_traj_launch);
    if (sw) sh.teams = 1;
    const int n_jobs = (int)idx.size();
    const int per = sw ? 2 : 8 * p0.d;
    const int V = g.nrep * p0.L_t * g.Ly * p0.L;

    size_t n_tcut = 0;
    long long n_cta = 0, n_traj_all = 0, n_spin_traj = 0;
    for (int j : idx) {
        n_tcut += (size_t)jobs[j].n_step * per;
        n_traj_all += jobs[j].n_traj;
        n_cta += (jobs[j].n_traj + sh.teams - 1) / sh.teams;
        if (spins && spins[j]) n_spin_traj += jobs[j].n_traj;
    }
    if (n_cta > 0x7FFFFFFFLL) return ISING_ERR_ARG;
    int rc;
    if ((rc = ensure(ctx, ctx->tcut, n_tcut * sizeof(uint32_t)))) return rc;
    if ((rc = ensure(ctx, ctx->jobs, (size_t)n_jobs * sizeof(jz::JobDesc)))) return rc;
    if (!outs_on_device && (rc = ensure(ctx, ctx->work, (size_t)n_traj_all * sizeof(long long))))
        return rc;
    if (n_spin_traj && !spins_on_device &&
        (rc = ensure(ctx, ctx->spins, (size_t)n_spin_traj * V)))
        return rc;
    size_t n_therm_desc = 0;   // thermalisation launches' job descriptors
    if (hybrid) {
        // HBM: the trajectories of all jobs, in order, cut into waves of
        // `chunk`; a job contributes one descriptor per wave it reaches
        long long fill = 0;
        for (int j : idx) {
            if (!therm_hbm) {
                ++n_therm_desc;
                continue;
            }
            for (long long off = 0; off < jobs[j].n_traj;) {
                const long long take = std::min(chunk - fill, jobs[j].n_traj - off);
                ++n_therm_desc;
                off += take;
                fill = (fill + take) % chunk;
            }
        }
        if ((rc = ensure(ctx, ctx->therm, (size_t)n_traj_all * V))) return rc;
        if ((rc = ensure(ctx, ctx->jobs, (n_jobs + n_therm_desc) * sizeof(jz::JobDesc))))
            return rc;
    }
    // one HBM lattice buffer serves the thermalisation chunks and then, on the
    // same stream, the protocol: sized for both before either launches
    size_t hbm_bytes = 0;
    if (in_hbm)
        hbm_bytes = sw ? (size_t)n_cta * jz::sw_smem_bytes(g)
                       : (size_t)n_cta * sh.teams * 2 * g.NR * g.GW * sizeof(uint32_t);
    if (therm_hbm) hbm_bytes = std::max(hbm_bytes, (size_t)chunk * jz::sw_smem_bytes(g));
    if (hbm_bytes && (rc = ensure(ctx, ctx->lattice, hbm_bytes))) return rc;

    const Range nv_group("jz run group");
    nvtxRangePushA("jz tables");   // host FP64 threshold tables (popped after the loop)
    ctx->h_tcut.assign(n_tcut, 0);
    ctx->h_jobs.assign(n_jobs, jz::JobDesc{});
    size_t off = 0;
    long long cta = 0, traj_off = 0, spin_off = 0;
    uint32_t* d_tcut = (uint32_t*)ctx->tcut.ptr;
    for (int i = 0; i < n_jobs; ++i) {
        const jz_params& p = jobs[idx[i]];
        jz::JobDesc& J = ctx->h_jobs[i];
        J.l = p.l;
        J.n_step = p.n_step;
        J.n_sweep = p.n_sweep;
        J.n_therm = p.n_therm;
        J.dir = p.direction;
        J.prot = p.protocol == 2 ? 2 : 1;
        cut_range(p, &J.g0, &J.g1);
        J.k_begin = seg ? seg->k_begin : 0;
        J.k_end = seg ? seg->k_end : p.n_step;
        J.spins_in = seg ? seg->spins_in : nullptr;
        J.w_in = seg ? seg->w_in : nullptr;
        J.start_in = 0;
        if (hybrid) {
            J.spins_in = (const int8_t*)ctx->therm.ptr + traj_off * (long long)V;
            J.start_in = 1;
        }
        J.n_traj = p.n_traj;
        J.traj0 = p.traj0;
        J.cta0 = cta;
        if (sw) build_bond_tables(p, J.tb, ctx->h_tcut, off);
        else build_tables(p, J.tb, ctx->h_tcut, off);
        J.tcut = d_tcut + off;
        J.w_out = outs_on_device ? (long long*)outs[idx[i]] : (long long*)ctx->work.ptr + traj_off;
        J.spins_out = nullptr;
        if (spins && spins[idx[i]]) {
            J.spins_out = spins_on_device ? spins[idx[i]]
                                          : (int8_t*)ctx->spins.ptr + spin_off * (long long)V;
            spin_off += p.n_traj;
        }
        off += (size_t)p.n_step * per;
        cta += (p.n_traj + sh.teams - 1) / sh.teams;
        traj_off += p.n_traj;
    }
    if (hybrid) {
        // the thermalisation jobs: Swendsen-Wang bulk bond threshold at the
        // start geometry, no protocol steps (k_end = 0, so no step table is
        // read), final spins into ctx->therm; their W_int (zero) lands in the
        // outputs that the protocol launch then overwrites
        ctx->h_jobs.resize(n_jobs + n_therm_desc);
        therm_waves.clear();
        std::vector<uint32_t> bt;
        long long sw_cta = 0;   // HBM: CTAs filled in the current wave
        size_t t = n_jobs;
        for (int i = 0; i < n_jobs; ++i) {
            const jz_params& p = jobs[idx[i]];
            jz::JobDesc T = ctx->h_jobs[i];
            bt.assign((size_t)2 * p.n_step, 0u);
            build_bond_tables(p, T.tb, bt, 0);
            T.k_begin = 0;
            T.k_end = 0;
            T.start_in = 0;
            T.spins_in = nullptr;
            T.w_in = nullptr;
            int8_t* so = (int8_t*)ctx->h_jobs[i].spins_in;   // this job's slice of ctx->therm
            for (long long off = 0; off < p.n_traj;) {
                const long long take =
                    therm_hbm ? std::min(chunk - sw_cta, (long long)p.n_traj - off) : p.n_traj;
                jz::JobDesc C = T;
                C.n_traj = (int)take;
                C.traj0 = T.traj0 + off;
                C.w_out = T.w_out + off;
                C.spins_out = so + off * (long long)V;
                C.cta0 = sw_cta;
                if (therm_hbm && sw_cta == 0) therm_waves.push_back({t, 0, 0});
                if (therm_hbm) {
                    ++therm_waves.back().n_desc;
                    therm_waves.back().n_cta += take;
                }
                ctx->h_jobs[t++] = C;
                sw_cta += take;
                if (therm_hbm && sw_cta == chunk) sw_cta = 0;   // the wave is full
                off += take;
            }
        }
    }
    nvtxRangePop();
    cudaStream_t st = ctx->stream;
    if ((rc = cuda_err(cudaMemcpyAsync(ctx->tcut.ptr, ctx->h_tcut.data(),
                                       n_tcut * sizeof(uint32_t), cudaMemcpyHostToDevice, st))))
        return rc;
    if ((rc = cuda_err(cudaMemcpyAsync(ctx->jobs.ptr, ctx->h_jobs.data(),
                                       ctx->h_jobs.size() * sizeof(jz::JobDesc),
                                       cudaMemcpyHostToDevice, st))))
        return rc;
    const jz::PhiloxKeys K = key_schedule(p0.seed);
    if (ctx->k_open) {
        if ((rc = cuda_err(cudaEventRecord(ctx->ev_k0, st)))) return rc;
        ctx->k_open = false;
    }
    if (hybrid && !therm_hbm &&
        (rc = cuda_err(jz::launch_sw(p0.d, g, K, (const jz::JobDesc*)ctx->jobs.ptr + n_jobs,
                                     n_jobs, n_traj_all, st, nullptr))))
        return rc;
    for (const ThermWave& w : therm_waves)
        if ((rc = cuda_err(jz::launch_sw(p0.d, g, K, (const jz::JobDesc*)ctx->jobs.ptr + w.first,
                                         (int)w.n_desc, w.n_cta, st,
                                         (uint32_t*)ctx->lattice.ptr))))
            return rc;
    if (sw) {
        uint32_t* gS = nullptr;
        if (in_hbm) gS = (uint32_t*)ctx->lattice.ptr;
        if ((rc = cuda_err(jz::launch_sw(p0.d, g, K, (const jz::JobDesc*)ctx->jobs.ptr, n_jobs,
                                         n_cta, st, gS))))
            return rc;
    } else {
        uint32_t* gS = nullptr;
        if (in_hbm) gS = (uint32_t*)ctx->lattice.ptr;
        if ((rc = cuda_err(jz::launch_traj(p0.d, g, K, (const jz::JobDesc*)ctx->jobs.ptr,
                                           n_jobs, n_cta, sh, st, gS))))
            return rc;
    }
    if ((rc = cuda_err(cudaEventRecord(ctx->ev_k1, st)))) return rc;
    ctx->k_timed = true;
    if (!outs_on_device || (n_spin_traj && !spins_on_device)) {
        long long c = 0, so = 0;
        for (int i = 0; i < n_jobs; ++i) {
            const jz_params& p = jobs[idx[i]];
            if (!outs_on_device &&
                (rc = cuda_err(cudaMemcpyAsync(outs[idx[i]], (long long*)ctx->work.ptr + c,
                                               p.n_traj * sizeof(long long),
                                               cudaMemcpyDeviceToHost, st))))
                return rc;
            if (spins && spins[idx[i]] && !spins_on_device) {
                if ((rc = cuda_err(cudaMemcpyAsync(spins[idx[i]],
                                                   (int8_t*)ctx->spins.ptr + so * (long long)V,
                                                   (size_t)p.n_traj * V, cudaMemcpyDeviceToHost,
                                                   st))))
                    return rc;
                so += p.n_traj;
            }
            c += p.n_traj;
        }
        if ((rc = cuda_err(cudaStreamSynchronize(st)))) return rc;
    }
    return ISING_OK;
}

int run_jobs(ising_ctx* ctx, const jz_params* jobs, int n_jobs, int64_t* const* outs,
             int8_t* const* spins)
{
    if (!ctx || !jobs || !outs || n_jobs < 1) return ISING_ERR_ARG;
    if (ctx->cancel.load()) return ISING_ERR_CANCELLED;
    ctx->k_open = true;   // a new run call: its first launch opens the timed span
    ctx->k_timed = false;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ISING_ERR_CUDA;
    for (int j = 0; j < n_jobs; ++j) {
        int rc = check_params(&jobs[j]);
        if (rc) return rc;
        if (!outs[j]) return ISING_ERR_ARG;
    }
    const bool outs_dev = is_device_ptr(outs[0]);
    for (int j = 1; j < n_jobs; ++j)
        if (is_device_ptr(outs[j]) != (int)outs_dev) return ISING_ERR_ARG;
    bool spins_dev = false;
    bool first = true;
    if (spins)
        for (int j = 0; j < n_jobs; ++j) {
            if (!spins[j]) continue;
            bool dv = is_device_ptr(spins[j]);
            if (first) { spins_dev = dv; first = false; }
            else if (dv != spins_dev) return ISING_ERR_ARG;
        }
    // one launch per (d, L, L_t, seed, update, n, thermalising update), jobs
    // kept in call order within a group
    using Key = std::tuple<int, int, int, uint64_t, int, int, int>;
    std::map<Key, std::vector<int>> groups;
    std::vector<Key> order;
    for (int j = 0; j < n_jobs; ++j) {
        auto key = std::make_tuple(jobs[j].d, jobs[j].L, jobs[j].L_t, jobs[j].seed,
                                   jobs[j].update, nrep_of(jobs[j]), (int)sw_therm(jobs[j]));
        auto it = groups.find(key);
        if (it == groups.end()) {
            order.push_back(key);
            groups[key] = {j};
        } else {
            it->second.push_back(j);
        }
    }
    for (auto& key : order) {
        auto& idx = groups[key];
        // keep the per-launch job table within bounds
        for (size_t s = 0; s < idx.size(); s += jz::kMaxJobsPerLaunch) {
            if (ctx->cancel.load()) return ISING_ERR_CANCELLED;
            std::vector<int> part(idx.begin() + s,
                                  idx.begin() + std::min(idx.size(), s + jz::kMaxJobsPerLaunch));
            int rc = run_group(ctx, jobs, part, outs, spins, outs_dev, spins_dev, nullptr);
            if (rc) return rc;
        }
    }
    return ISING_OK;
}

}  // namespace jzh

using namespace jzh;

extern "C" {

int jz_params_default(jz_params* p)
{
    if (!p) return ISING_ERR_ARG;
    std::memset(p, 0, sizeof *p);
    p->n_therm = 1000;
    p->n_sweep = 1;
    p->direction = 1;
    p->protocol = 1;
    p->n_replica = 2;
    return ISING_OK;
}

int ising_replica_init(ising_ctx** out, int device, size_t hbm_budget_bytes, void* cuda_stream)
{
    if (!out) return ISING_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) {
        cudaGetLastError();
        return ISING_ERR_CUDA;
    }
    if (device < 0 || device >= n) return ISING_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return ISING_ERR_CUDA;
    ising_ctx* ctx = new (std::nothrow) ising_ctx();
    if (!ctx) return ISING_ERR_NOMEM;
    ctx->device = device;
    ctx->budget = hbm_budget_bytes;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) ctx->gpu_name = prop.name;
    else cudaGetLastError();
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return ISING_ERR_CUDA;
        }
        ctx->own_stream = true;
    }
    if (cudaEventCreate(&ctx->ev_k0) != cudaSuccess || cudaEventCreate(&ctx->ev_k1) != cudaSuccess) {
        if (ctx->ev_k0) cudaEventDestroy(ctx->ev_k0);
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        delete ctx;
        return ISING_ERR_CUDA;
    }
    *out = ctx;
    return ISING_OK;
}

void ising_replica_free(ising_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (DevBuf* b : {&ctx->tcut, &ctx->jobs, &ctx->work, &ctx->spins, &ctx->est_in,
                      &ctx->est_out, &ctx->lattice})
        if (b->ptr) cudaFree(b->ptr);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    cudaEventDestroy(ctx->ev_k0);
    cudaEventDestroy(ctx->ev_k1);
    delete ctx;
}

int ising_last_launch_ms(ising_ctx* ctx, float* ms)
{
    if (!ctx || !ms || !ctx->k_timed) return ISING_ERR_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ISING_ERR_CUDA;
    int rc = cuda_err(cudaEventSynchronize(ctx->ev_k1));
    if (rc) return rc;
    return cuda_err(cudaEventElapsedTime(ms, ctx->ev_k0, ctx->ev_k1));
}

int ising_sync(ising_ctx* ctx)
{
    if (!ctx) return ISING_ERR_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ISING_ERR_CUDA;
    return cuda_err(cudaStreamSynchronize(ctx->stream));
}

int jarzynski_run_ex(ising_ctx* ctx, const jz_params* p, int64_t* work_int_out,
                     int8_t* spins_out)
{
    if (!p || !work_int_out) return ISING_ERR_ARG;
    int64_t* outs[1] = {work_int_out};
    int8_t* sp[1] = {spins_out};
    return run_jobs(ctx, p, 1, outs, spins_out ? sp : nullptr);
}

int jarzynski_run(ising_ctx* ctx, int d, int L, int L_t, double beta, int l, int n_step,
                  int n_sweep, int n_traj, uint64_t seed, int64_t* work_int_out)
{
    jz_params p;
    jz_params_default(&p);
    p.d = d;
    p.L = L;
    p.L_t = L_t;
    p.beta = beta;
    p.l = l;
    p.n_step = n_step;
    p.n_sweep = n_sweep;
    p.n_traj = n_traj;
    p.seed = seed;
    return jarzynski_run_ex(ctx, &p, work_int_out, nullptr);
}

int ising_set_threads(ising_ctx* ctx, int d, int L, int L_t, int threads)
{
    if (!ctx || (d != 2 && d != 3) || L < 2 || L_t < 2 || (L & 1) || (L_t & 1))
        return ISING_ERR_ARG;
    const auto key = std::make_tuple(d, L, L_t);
    if (threads != 0 && !threads_ok(make_geom(d, L, L_t, 2), threads)) return ISING_ERR_ARG;
    std::lock_guard<std::mutex> lk(ctx->shapes_mu);
    if (threads == 0) ctx->threads.erase(key);
    else ctx->threads[key] = threads;
    return ISING_OK;
}

int ising_launch_shape(ising_ctx* ctx, const jz_params* p, int* shape)
{
    if (!ctx || !p || !shape) return ISING_ERR_ARG;
    int rc = check_params(p);
    if (rc) return rc;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ISING_ERR_CUDA;
    const jz::Geom g = make_geom(p->d, p->L, p->L_t, nrep_of(*p));
    if (p->update == 1) {
        const int t = jz::sw_cta_threads(p->d);
        const int v[5] = {t, 1, t, 0, sw_fits(g) ? 0 : 1};
        std::memcpy(shape, v, sizeof v);
        return ISING_OK;
    }
    if (!threads_fit(g)) return ISING_ERR_UNSUPPORTED;
    const jz::LaunchShape sh = ctx_shape(ctx, p->d, g, p->n_traj);
    const int v[5] = {sh.team_threads, sh.teams, sh.cta_threads, sh.warp, shape_fits(g) ? 0 : 1};
    std::memcpy(shape, v, sizeof v);
    return ISING_OK;
}

int ising_autotune(ising_ctx* ctx, const jz_params* p, int* threads)
{
    if (!ctx || !p) return ISING_ERR_ARG;
    if (ctx->cancel.load()) return ISING_ERR_CANCELLED;
    const Range nv("jz autotune");
    int rc = check_params(p);
    if (rc) return rc;
    if (p->update == 1) {   // Swendsen-Wang: a fixed CTA per trajectory, nothing to tune
        if (threads) *threads = jz::sw_cta_threads(p->d);
        return ISING_OK;
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ISING_ERR_CUDA;
    const jz::Geom g = make_geom(p->d, p->L, p->L_t, nrep_of(*p));
    if (!shape_fits(g)) return ISING_ERR_UNSUPPORTED;
    jz_params s = *p;
    s.n_therm = 16;
    s.n_step = 16;
    s.n_sweep = 1;
    s.therm_update = 0;   // the launch shape is the protocol kernel's
    s.n_traj = p->n_traj < 4864 ? p->n_traj : 4864;
    s.traj0 = 0;
    if ((rc = ensure(ctx, ctx->est_in, (size_t)s.n_traj * sizeof(long long)))) return rc;
    int64_t* out = (int64_t*)ctx->est_in.ptr;
    // explicit CTA sizes, then 0: the default shape for the sample's
    // trajectory count, when it is none of theirs
    std::vector<int> cands;
    const int col = g.GW * g.Ly;
    if (col <= 32) {
        for (int t = 32; t <= 512; t *= 2) cands.push_back(t);
    } else {
        for (int ts = 1; ts <= g.Lt && col * ts <= 512; ts *= 2) cands.push_back(col * ts);
        const int def = shape_for(g, 0).cta_threads;
        if (std::find(cands.begin(), cands.end(), def) == cands.end()) cands.push_back(def);
    }
    {
        const jz::LaunchShape d0 = default_shape(p->d, g, s.n_traj);
        bool listed = false;
        for (int t : cands) {
            const jz::LaunchShape e = shape_for(g, t);
            listed = listed || (e.team_threads == d0.team_threads && e.teams == d0.teams &&
                                e.cta_threads == d0.cta_threads && e.warp == d0.warp);
        }
        if (!listed) cands.push_back(0);
    }
    const auto key = std::make_tuple(p->d, p->L, p->L_t);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return ISING_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return ISING_ERR_CUDA;
    }
    int best = shape_for(g, 0).cta_threads;
    float best_ms = 1e30f;
    int64_t* outs[1] = {out};
    for (int t : cands) {
        {
            std::lock_guard<std::mutex> lk(ctx->shapes_mu);
            if (t) ctx->threads[key] = t;
            else ctx->threads.erase(key);
        }
        if ((rc = run_jobs(ctx, &s, 1, outs, nullptr))) break;           // warm-up
        cudaEventRecord(e0, ctx->stream);
        if ((rc = run_jobs(ctx, &s, 1, outs, nullptr))) break;
        cudaEventRecord(e1, ctx->stream);
        if ((rc = cuda_err(cudaEventSynchronize(e1)))) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        std::lock_guard<std::mutex> lk(ctx->shapes_mu);
        if (best) ctx->threads[key] = best;
        else ctx->threads.erase(key);
    }
    if (rc) return rc;
    if (threads) *threads = best;
    return ISING_OK;
}

int jarzynski_run_batch(ising_ctx* ctx, const jz_params* jobs, int n_jobs,
                        int64_t* const* work_outs)
{
    return run_jobs(ctx, jobs, n_jobs, work_outs, nullptr);
}

int jarzynski_run_segment(ising_ctx* ctx, const jz_params* p, int k_begin, int k_end,
                          int64_t* work_io, int8_t* spins_io)
{
    if (!ctx || !p || !work_io || !spins_io) return ISING_ERR_ARG;
    if (ctx->cancel.load()) return ISING_ERR_CANCELLED;
    ctx->k_open = true;
    ctx->k_timed = false;
    int rc = check_params(p);
    if (rc) return rc;
    if (k_begin < 0 || k_end <= k_begin || k_end > p->n_step) return ISING_ERR_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ISING_ERR_CUDA;
    if (!is_device_ptr(work_io) || !is_device_ptr(spins_io)) return ISING_ERR_ARG;
    const Segment seg{k_begin, k_end, spins_io, (const long long*)work_io};
    int64_t* outs[1] = {work_io};
    int8_t* sp[1] = {spins_io};
    return run_group(ctx, p, std::vector<int>{0}, outs, sp, true, true, &seg);
}

int jarzynski_run_plain(ising_ctx* ctx, const jz_params* p, int64_t* work_int_out,
                        int8_t* spins_out)
{
    if (!ctx || !p || !work_int_out) return ISING_ERR_ARG;
    if (ctx->cancel.load()) return ISING_ERR_CANCELLED;
    int rc = check_params(p);
    if (rc) return rc;
    if (p->update != 0 || (p->protocol == 2 && p->d == 3) || nrep_of(*p) != 2 || p->whole ||
        sw_therm(*p))
        return ISING_ERR_UNSUPPORTED;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ISING_ERR_CUDA;
    const jz::Geom g = make_geom(p->d, p->L, p->L_t, 2);
    const int V = 2 * p->L_t * g.Ly * p->L;
    const bool w_dev = is_device_ptr(work_int_out);
    const bool s_dev = spins_out && is_device_ptr(spins_out);
    const size_t n_tcut = (size_t)p->n_step * 8 * p->d;
    if ((rc = ensure(ctx, ctx->tcut, n_tcut * sizeof(uint32_t)))) return rc;
    if (!w_dev && (rc = ensure(ctx, ctx->work, (size_t)p->n_traj * sizeof(long long)))) return rc;
    if (!s_dev && (rc = ensure(ctx, ctx->spins, (size_t)(spins_out ? p->n_traj : 1) * V)))
        return rc;
    ctx->h_tcut.assign(n_tcut, 0);
    uint32_t tb[4];
    build_tables(*p, tb, ctx->h_tcut, 0);
    cudaStream_t st = ctx->stream;
    if ((rc = cuda_err(cudaMemcpyAsync(ctx->tcut.ptr, ctx->h_tcut.data(), n_tcut * sizeof(uint32_t),
                                       cudaMemcpyHostToDevice, st))))
        return rc;
    const jz::PhiloxKeys K = key_schedule(p->seed);
    long long* w = w_dev ? (long long*)work_int_out : (long long*)ctx->work.ptr;
    for (int i = 0; i < p->n_traj; ++i) {
        if (ctx->cancel.load()) return ISING_ERR_CANCELLED;
        int8_t* s = s_dev ? spins_out + (size_t)i * V
                          : (int8_t*)ctx->spins.ptr + (spins_out ? (size_t)i * V : 0);
        if ((rc = cuda_err(jz::plain_trajectory(p->d, g, K, p->l, p->direction, p->n_step,
                                                p->n_sweep, p->n_therm,
                                                (uint32_t)(p->traj0 + i), tb,
                                                (const uint32_t*)ctx->tcut.ptr, s, w + i, st))))
            return rc;
    }
    if (!w_dev &&
        (rc = cuda_err(cudaMemcpyAsync(work_int_out, w, (size_t)p->n_traj * sizeof(long long),
                                       cudaMemcpyDeviceToHost, st))))
        return rc;
    if (spins_out && !s_dev &&
        (rc = cuda_err(cudaMemcpyAsync(spins_out, ctx->spins.ptr, (size_t)p->n_traj * V,
                                       cudaMemcpyDeviceToHost, st))))
        return rc;
    if (!w_dev || (spins_out && !s_dev)) return cuda_err(cudaStreamSynchronize(st));
    return ISING_OK;
}

int estimator_reduce(ising_ctx* ctx, const int64_t* work_int, int n_traj, double beta,
                     int n_step, int direction, int n_jack_bins, double* log_ratio,
                     double* delta_S2, double* delta_S2_err)
{
    if (!ctx || !work_int || n_traj < 1 || n_step < 1 || !log_ratio || !delta_S2 ||
        !delta_S2_err)
        return ISING_ERR_ARG;
    if (direction != 1 && direction != -1) return ISING_ERR_ARG;
    if (n_jack_bins < 1 || n_jack_bins > jz::kMaxJackBlocksHost) return ISING_ERR_ARG;
    if (!(beta >= 0.0 && std::isfinite(beta))) return ISING_ERR_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ISING_ERR_CUDA;
    const Range nv("jz estimator");
    int rc;
    const long long* src = (const long long*)work_int;
    cudaStream_t st = ctx->stream;
    if (!is_device_ptr(work_int)) {
        if ((rc = ensure(ctx, ctx->est_in, (size_t)n_traj * sizeof(long long)))) return rc;
        if ((rc = cuda_err(cudaMemcpyAsync(ctx->est_in.ptr, work_int,
                                           (size_t)n_traj * sizeof(long long),
                                           cudaMemcpyHostToDevice, st))))
            return rc;
        src = (const long long*)ctx->est_in.ptr;
    }
    if ((rc = ensure(ctx, ctx->est_out, 4 * sizeof(double)))) return rc;
    const int B = n_jack_bins < n_traj ? n_jack_bins : n_traj;
    if ((rc = cuda_err(jz::launch_estimator(src, n_traj, beta / (double)n_step, direction, B,
                                            (double*)ctx->est_out.ptr, st))))
        return rc;
    double h[3];
    if ((rc = cuda_err(cudaMemcpyAsync(h, ctx->est_out.ptr, 3 * sizeof(double),
                                       cudaMemcpyDeviceToHost, st))))
        return rc;
    if ((rc = cuda_err(cudaStreamSynchronize(st)))) return rc;
    *log_ratio = h[0];
    *delta_S2 = h[1];
    *delta_S2_err = h[2];
    return ISING_OK;
}

int ising_probe(int device, int kind, double* rate)
{
    if (!rate || kind < 0 || kind > 3) return ISING_ERR_ARG;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) {
        cudaGetLastError();
        return ISING_ERR_CUDA;
    }
    if (device < 0 || device >= n) return ISING_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return ISING_ERR_CUDA;
    const double r = jz::run_probe(kind, device);
    if (r < 0) {
        cudaGetLastError();
        return ISING_ERR_CUDA;
    }
    *rate = r;
    return ISING_OK;
}

const char* ising_strerror(int code)
{
    switch (code) {
    case ISING_OK: return "ok";
    case ISING_ERR_ARG: return "invalid argument";
    case ISING_ERR_ODD_EXTENT: return "L and L_t must be even";
    case ISING_ERR_L_RANGE: return "l must satisfy 0 <= l <= L-1";
    case ISING_ERR_NOMEM: return "device memory or HBM budget exhausted";
    case ISING_ERR_CUDA: return "CUDA runtime error";
    case ISING_ERR_TIMEOUT: return "bounded device wait gave up";
    case ISING_ERR_UNSUPPORTED: return "unsupported dimension or lattice too large";
    case ISING_ERR_NOT_FOUND: return "unknown job id";
    case ISING_ERR_PENDING: return "job not finished";
    case ISING_ERR_SCRATCH_LIMIT:
        return "protocol too long for the fixed scratch of jarzynski_run_noalloc";
    case ISING_ERR_CANCELLED: return "cancelled";
    default: return "unknown error";
    }
}

}  // extern "C"

// ------------------------------------------------------ no-allocation path --
// jarzynski_run_noalloc: the trajectory kernel with its scratch (job
// descriptor + switched-site thresholds) in one fixed device array instead of
// context buffers, for callers that cannot allocate device memory.
namespace {
constexpr size_t kNoAllocScratchBytes = (size_t)1 << 20;   // 1 MiB per device
constexpr size_t kNoAllocJobBytes = 256;                   // descriptor slot
constexpr size_t kNoAllocMaxThresholds =
    (kNoAllocScratchBytes - kNoAllocJobBytes) / sizeof(uint32_t);   // 262080 words
constexpr size_t kNoAllocWords = kNoAllocScratchBytes / sizeof(uint32_t);
static_assert(sizeof(jz::JobDesc) <= kNoAllocJobBytes, "descriptor slot too small");

// The scratch contents travel to the device as kernel arguments, in chunks of
// kStageWords words (31.7 KB of parameters per launch), so the call reads no
// host memory after it returns and needs no pinned staging buffer.
constexpr int kStageWords = 7936;
struct StageChunk {
    uint32_t w[kStageWords];
};
}  // namespace

// Held by every GPU that loads the library, until exit.  Host code sees only a
// host-side stand-in under this name; the device address comes from
// cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Copies n words of the argument chunk to dst (one launch per chunk).
__global__ void __launch_bounds__(256) noalloc_stage_kernel(uint32_t* __restrict__ dst, int n,
                                                            const StageChunk c)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        dst[i] = c.w[i];
}

namespace {
std::mutex g_noalloc_mutex;   // guards the host image below
// host image of the scratch (descriptor slot, then the thresholds), static so
// that calls never allocate
uint32_t g_noalloc_host[kNoAllocWords];
StageChunk g_noalloc_chunk;

// Device address of the scratch array on the current device.  Looked up on
// every call: after a device reset the module reloads at a new address.
int noalloc_scratch_address(void** out)
{
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return ISING_ERR_CUDA;
    }
    *out = p;
    return ISING_OK;
}
}  // namespace

extern "C" int ising_bounds_status(unsigned int* sites, unsigned int* index, int clear)
{
#ifdef JZ_BOUNDS_CHECK
    if (!sites || !index) return ISING_ERR_ARG;
    unsigned int a[2], b[2], c[2];
    int rc;
    if ((rc = cuda_err(jz::bounds_status_traj(a, clear != 0))) ||
        (rc = cuda_err(jz::bounds_status_batch(b, clear != 0))) ||
        (rc = cuda_err(jz::bounds_status_sw(c, clear != 0))))
        return rc;
    *sites = a[0] | b[0] | c[0];
    *index = a[0] ? a[1] : b[0] ? b[1] : c[1];
    return ISING_OK;
#else
    (void)sites;
    (void)index;
    (void)clear;
    return ISING_ERR_UNSUPPORTED;
#endif
}

extern "C" int ising_binary_version(int device, int* version)
{
    if (!version) return ISING_ERR_ARG;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) {
        cudaGetLastError();
        return ISING_ERR_CUDA;
    }
    if (device < 0 || device >= n) return ISING_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return ISING_ERR_CUDA;
    cudaFuncAttributes a;
    const int rc = cuda_err(cudaFuncGetAttributes(&a, noalloc_stage_kernel));
    if (rc) return rc;
    *version = a.binaryVersion;
    return ISING_OK;
}

extern "C" int jarzynski_run_noalloc(const jz_params* p, int64_t* work_int_out, void* cuda_stream)
{
    if (!p || !work_int_out) return ISING_ERR_ARG;
    int rc = check_params(p);
    if (rc) return rc;
    if (sw_therm(*p)) return ISING_ERR_UNSUPPORTED;
    const bool sw = p->update == 1;   // Swendsen-Wang: one trajectory per CTA
    const size_t n_tcut = (size_t)p->n_step * (sw ? 2 : 8 * (size_t)p->d);
    if (n_tcut > kNoAllocMaxThresholds) return ISING_ERR_SCRATCH_LIMIT;
    const jz::Geom g = make_geom(p->d, p->L, p->L_t, nrep_of(*p));
    if (sw ? !sw_fits(g) : !shape_fits(g)) return ISING_ERR_UNSUPPORTED;
    if (!is_device_ptr(work_int_out)) return ISING_ERR_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    void* base = nullptr;
    if ((rc = noalloc_scratch_address(&base))) return rc;
    uint32_t* d_words = (uint32_t*)base;
    uint32_t* d_tcut = d_words + kNoAllocJobBytes / sizeof(uint32_t);

    jz::JobDesc J{};
    J.l = p->l;
    J.n_step = p->n_step;
    J.n_sweep = p->n_sweep;
    J.n_therm = p->n_therm;
    J.dir = p->direction;
    J.prot = p->protocol == 2 ? 2 : 1;
    cut_range(*p, &J.g0, &J.g1);
    J.k_begin = 0;
    J.k_end = p->n_step;
    J.n_traj = p->n_traj;
    J.traj0 = p->traj0;
    J.cta0 = 0;
    // the thresholds go to the host image behind the descriptor slot
    uint32_t* h_tcut = g_noalloc_host + kNoAllocJobBytes / sizeof(uint32_t);
    if (sw) build_bond_tables_into(*p, J.tb, h_tcut);
    else build_tables_into(*p, J.tb, h_tcut);
    J.tcut = d_tcut;
    J.w_out = (long long*)work_int_out;
    J.spins_out = nullptr;
    std::memset(g_noalloc_host, 0, kNoAllocJobBytes);
    std::memcpy(g_noalloc_host, &J, sizeof J);
    // stage descriptor + thresholds, one launch per chunk of kernel arguments
    const size_t total = kNoAllocJobBytes / sizeof(uint32_t) + n_tcut;
    for (size_t off = 0; off < total; off += kStageWords) {
        const int cnt = (int)std::min<size_t>(kStageWords, total - off);
        std::memcpy(g_noalloc_chunk.w, g_noalloc_host + off, (size_t)cnt * sizeof(uint32_t));
        noalloc_stage_kernel<<<(cnt + 255) / 256, 256, 0, st>>>(d_words + off, cnt,
                                                               g_noalloc_chunk);
        if ((rc = cuda_err(cudaGetLastError()))) return rc;
    }
    const jz::PhiloxKeys K = key_schedule(p->seed);
    if (sw) return cuda_err(jz::launch_sw(p->d, g, K, (const jz::JobDesc*)base, 1, p->n_traj, st));
    const jz::LaunchShape sh = default_shape(p->d, g, p->n_traj);
    return cuda_err(jz::launch_traj(p->d, g, K, (const jz::JobDesc*)base, 1,
                                    (p->n_traj + sh.teams - 1) / sh.teams, sh, st));
}

// --------------------------------------------------- persistent batch plans --
namespace jz {
cudaError_t persistent_prepare(size_t smem, int threads, int* blocks_per_sm);
cudaError_t launch_persistent(const BatchJob* jobs, const int2* items, int n_items,
                              unsigned int* counter, const PhiloxKeys& K, int grid, int threads,
                              size_t smem, cudaStream_t st);
cudaError_t launch_estimator_batch(const EstJob* jobs, int n_jobs, double* out, cudaStream_t st);
}  // namespace jz

// A job's layout inside the plan's CTAs of cta threads: the warp teams of
// shape_for, or one team of the whole CTA when that keeps more of the CTA's
// lanes busy (shape_score's barrier term).  A large lattice leaves most warps
// of a warp-team CTA idle -- 2D L = 128 fits seven 32 KB lattices in a
// 384-thread CTA -- and its shared memory would then set every CTA's, one
// CTA per SM; as one team it holds one lattice.
jz::LaunchShape plan_shape(const jz::Geom& g, int cta)
{
    const jz::LaunchShape w = shape_for(g, cta);
    const int col = g.GW * g.Ly;
    const int ts = std::min(cta / col, g.Lt);
    if (ts < 1 || col * ts < 32) return w;
    auto busy = [&](const jz::LaunchShape& sh) {
        double b = (double)sh.teams * sh.team_threads / cta;
        if (!sh.warp) {
            const double rows = (double)g.nrep * g.Lt / std::min(sh.team_threads / col, g.Lt);
            b *= rows / (rows + kBarrierRows);
        }
        return b;
    };
    jz::LaunchShape c{};
    c.team_threads = col * ts;
    c.teams = 1;
    c.cta_threads = col * ts;
    c.warp = 0;
    return busy(c) > kKeepMargin * busy(w) ? c : w;
}

struct jz_plan {
    ising_ctx* ctx = nullptr;
    int n_jobs = 0, n_items = 0, threads = 0, grid = 0;
    size_t smem = 0;
    jz::PhiloxKeys K{};
    DevBuf jobs, items, tcut, counter, est_jobs;
    double* est_out = nullptr;
    // Swendsen-Wang jobs: one launch per lattice shape after the persistent
    // kernel (one CTA per trajectory, no work items)
    struct SwGroup {
        jz::Geom g{};
        int d = 0, n_jobs = 0;
        long long n_cta = 0;
        bool hbm = false;   // thermalisation from HBM slices, in waves
        long long wave = 0, fill = 0;   // hbm: trajectories per wave, CTAs in the open one
        struct Wave {
            int first, n_desc;
            long long n_cta;
        };
        std::vector<Wave> waves;        // hbm: descriptor ranges launched together
        DevBuf jobs;
        std::vector<jz::JobDesc> h_jobs;
        std::vector<size_t> toff;
    };
    std::vector<SwGroup> sw;
    DevBuf sw_tcut;
    // therm_update = 1: thermalisation-only Swendsen-Wang launches (one per
    // lattice shape) ahead of the persistent kernel, their spins in therm_spins
    std::vector<SwGroup> therm;
    DevBuf therm_spins;
    DevBuf therm_lattice;   // HBM slices of one thermalisation wave (the largest one)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

void plan_release(jz_plan* pl)
{
    if (!pl) return;
    ising_ctx* ctx = pl->ctx;
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    std::vector<DevBuf*> bufs = {&pl->jobs, &pl->items, &pl->tcut, &pl->counter, &pl->est_jobs,
                                 &pl->sw_tcut};
    for (auto& G : pl->sw) bufs.push_back(&G.jobs);
    for (auto& G : pl->therm) bufs.push_back(&G.jobs);
    bufs.push_back(&pl->therm_spins);
    bufs.push_back(&pl->therm_lattice);
    for (DevBuf* b : bufs)
        if (b->ptr) {
            cudaFree(b->ptr);
            ctx->used -= b->bytes;
        }
    delete pl;
}

// Builds (not captures) a plan for a fixed CTA size.
int plan_build(ising_ctx* ctx, const jz_params* jobs, int n_jobs, int64_t* const* work_outs,
               double* est_out, int cta, jz_plan** out)
{
    jz_plan* pl = new (std::nothrow) jz_plan();
    if (!pl) return ISING_ERR_NOMEM;
    pl->ctx = ctx;
    pl->n_jobs = n_jobs;
    pl->threads = cta;
    pl->est_out = est_out;
    pl->K = key_schedule(jobs[0].seed);
    std::vector<jz::BatchJob> bj(n_jobs);
    std::vector<uint32_t> tcut;
    std::vector<size_t> toff(n_jobs);
    std::vector<std::pair<double, int2>> items;
    std::vector<uint32_t> sw_tcut;
    size_t smem = 0;
    // therm_update = 1 jobs: byte offset of each job's spins in therm_spins
    std::vector<long long> therm_off(n_jobs, -1);
    size_t therm_bytes = 0;
    size_t therm_lattice_bytes = 0;
    auto group_of = [](std::vector<jz_plan::SwGroup>& gs, int d, const jz::Geom& g) {
        size_t gi = 0;
        while (gi < gs.size() && !(gs[gi].d == d && gs[gi].g.L == g.L && gs[gi].g.Lt == g.Lt &&
                                   gs[gi].g.nrep == g.nrep))
            ++gi;
        if (gi == gs.size()) {
            gs.emplace_back();
            gs.back().g = g;
            gs.back().d = d;
            gs.back().hbm = !sw_fits(g);
            if (gs.back().hbm) gs.back().wave = jz::sw_hbm_wave(d);
        }
        return gi;
    };
    for (int j = 0; j < n_jobs; ++j) {
        const jz_params& p = jobs[j];
        if (p.update == 1) {   // Swendsen-Wang: grouped by lattice shape
            const jz::Geom g = make_geom(p.d, p.L, p.L_t, nrep_of(p));
            if (!sw_fits(g)) {
                plan_release(pl);
                return ISING_ERR_UNSUPPORTED;
            }
            jz_plan::SwGroup& G = pl->sw[group_of(pl->sw, p.d, g)];
            jz::JobDesc J{};
            J.l = p.l;
            J.n_step = p.n_step;
            J.n_sweep = p.n_sweep;
            J.n_therm = p.n_therm;
            J.dir = p.direction;
            J.prot = p.protocol == 2 ? 2 : 1;
            cut_range(p, &J.g0, &J.g1);
            J.k_begin = 0;
            J.k_end = p.n_step;
            J.n_traj = p.n_traj;
            J.traj0 = p.traj0;
            J.cta0 = G.n_cta;
            const size_t off = sw_tcut.size();
            sw_tcut.resize(off + (size_t)p.n_step * 2);
            build_bond_tables(p, J.tb, sw_tcut, off);
            J.w_out = (long long*)work_outs[j];
            J.spins_out = nullptr;
            G.h_jobs.push_back(J);
            G.toff.push_back(off);
            G.n_cta += p.n_traj;
            ++G.n_jobs;
            continue;
        }
        jz::BatchJob& B = bj[j];
        B.g = make_geom(p.d, p.L, p.L_t, nrep_of(p));
        B.D = p.d;
        B.fast = (B.g.Lh % 8) == 0;   // rows of whole 8-site words
        B.sh = plan_shape(B.g, cta);
        B.lattice_words = 2 * B.g.NR * B.g.GW;
        if (!shape_fits(B.g) || B.sh.team_threads > cta || (B.sh.warp && B.sh.cta_threads > cta)) {
            plan_release(pl);
            return ISING_ERR_UNSUPPORTED;
        }
        const size_t sm = (size_t)B.sh.teams * B.lattice_words * 4;
        if (sm > jz::kMaxSmemPerCta) {
            plan_release(pl);
            return ISING_ERR_UNSUPPORTED;
        }
        smem = std::max(smem, sm);
        toff[j] = tcut.size();
        tcut.resize(tcut.size() + (size_t)p.n_step * 8 * p.d);
        jz::JobDesc& J = B.J;
        J.l = p.l;
        J.n_step = p.n_step;
        J.n_sweep = p.n_sweep;
        J.n_therm = p.n_therm;
        J.dir = p.direction;
        J.prot = p.protocol == 2 ? 2 : 1;
        cut_range(p, &J.g0, &J.g1);
        J.k_begin = 0;
        J.k_end = p.n_step;
        J.n_traj = p.n_traj;
        J.traj0 = p.traj0;
        J.cta0 = 0;
        build_tables(p, J.tb, tcut, toff[j]);
        J.w_out = (long long*)work_outs[j];
        J.spins_out = nullptr;
        if (sw_therm(p)) {
            // its Swendsen-Wang thermalisation: no protocol steps, spins into
            // its slice of therm_spins, from which the persistent kernel
            // starts; a state beyond shared memory runs from HBM slices in
            // launches of one resident wave of trajectories
            jz_plan::SwGroup& G = pl->therm[group_of(pl->therm, p.d, B.g)];
            jz::JobDesc T = J;
            std::vector<uint32_t> bt((size_t)2 * p.n_step);
            build_bond_tables(p, T.tb, bt, 0);
            T.k_end = 0;
            if (G.hbm)
                therm_lattice_bytes = std::max(therm_lattice_bytes,
                                               (size_t)G.wave * jz::sw_smem_bytes(B.g));
            // pieces of this job's trajectories; in HBM they fill waves of
            // G.wave CTAs shared with the group's other jobs
            for (long long off = 0; off < p.n_traj;) {
                const long long take =
                    G.hbm ? std::min(G.wave - G.fill, (long long)p.n_traj - off) : p.n_traj;
                jz::JobDesc C = T;
                C.n_traj = (int)take;
                C.traj0 = T.traj0 + off;
                C.w_out = T.w_out + off;
                C.cta0 = G.hbm ? G.fill : G.n_cta;
                if (G.hbm && G.fill == 0) G.waves.push_back({G.n_jobs, 0, 0});
                if (G.hbm) {
                    ++G.waves.back().n_desc;
                    G.waves.back().n_cta += take;
                    G.fill = (G.fill + take) % G.wave;
                }
                G.h_jobs.push_back(C);
                G.toff.push_back(((size_t)j << 32) | (size_t)off);   // job, first trajectory
                G.n_cta += take;
                ++G.n_jobs;
                off += take;
            }
            therm_off[j] = (long long)therm_bytes;
            therm_bytes += (size_t)p.n_traj * (size_t)(B.g.nrep * p.L_t * B.g.Ly * p.L);
            J.start_in = 1;
        }
        const double per_traj = (double)(B.g.nrep * p.L_t * B.g.Ly * p.L) *
                                ((double)p.n_therm + (double)p.n_step * p.n_sweep);
        for (int lo = 0; lo < p.n_traj; lo += B.sh.teams) {
            const int cnt = std::min(B.sh.teams, p.n_traj - lo);
            items.push_back({per_traj * cnt, make_int2(j, lo)});
        }
    }
    // largest items first
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<double, int2>& a, const std::pair<double, int2>& b) {
                         return a.first > b.first;
                     });
    pl->n_items = (int)items.size();
    pl->smem = smem;
    int rc;
    if ((rc = ensure(ctx, pl->tcut, tcut.size() * sizeof(uint32_t))) ||
        (rc = ensure(ctx, pl->jobs, bj.size() * sizeof(jz::BatchJob))) ||
        (rc = ensure(ctx, pl->items, items.size() * sizeof(int2))) ||
        (rc = ensure(ctx, pl->counter, sizeof(unsigned int))) ||
        (rc = ensure(ctx, pl->est_jobs, (size_t)n_jobs * sizeof(jz::EstJob)))) {
        plan_release(pl);
        return rc;
    }
    uint32_t* d_tcut = (uint32_t*)pl->tcut.ptr;
    for (int j = 0; j < n_jobs; ++j) bj[j].J.tcut = d_tcut + toff[j];
    if (!pl->therm.empty()) {
        if ((rc = ensure(ctx, pl->therm_spins, therm_bytes))) {
            plan_release(pl);
            return rc;
        }
        if (therm_lattice_bytes && (rc = ensure(ctx, pl->therm_lattice, therm_lattice_bytes))) {
            plan_release(pl);
            return rc;
        }
        int8_t* base = (int8_t*)pl->therm_spins.ptr;
        for (int j = 0; j < n_jobs; ++j)
            if (therm_off[j] >= 0) bj[j].J.spins_in = base + therm_off[j];
        for (auto& G : pl->therm) {
            for (size_t i = 0; i < G.h_jobs.size(); ++i) {
                const size_t j = G.toff[i] >> 32, off = G.toff[i] & 0xFFFFFFFFu;
                const long long V = (long long)G.g.nrep * G.g.Lt * G.g.Ly * G.g.L;
                G.h_jobs[i].tcut = bj[j].J.tcut;   // not read: no protocol steps
                G.h_jobs[i].spins_out = base + therm_off[j] + (long long)off * V;
            }
            if ((rc = ensure(ctx, G.jobs, G.h_jobs.size() * sizeof(jz::JobDesc)))) {
                plan_release(pl);
                return rc;
            }
        }
    }
    if (!pl->sw.empty()) {
        if ((rc = ensure(ctx, pl->sw_tcut, sw_tcut.size() * sizeof(uint32_t)))) {
            plan_release(pl);
            return rc;
        }
        for (auto& G : pl->sw) {
            for (size_t i = 0; i < G.h_jobs.size(); ++i)
                G.h_jobs[i].tcut = (uint32_t*)pl->sw_tcut.ptr + G.toff[i];
            if ((rc = ensure(ctx, G.jobs, G.h_jobs.size() * sizeof(jz::JobDesc)))) {
                plan_release(pl);
                return rc;
            }
        }
    }
    std::vector<int2> it(items.size());
    for (size_t i = 0; i < items.size(); ++i) it[i] = items[i].second;
    std::vector<jz::EstJob> ej(n_jobs);
    for (int j = 0; j < n_jobs; ++j) {
        ej[j].w = (const long long*)work_outs[j];
        ej[j].n = jobs[j].n_traj;
        ej[j].direction = jobs[j].direction;
        ej[j].n_blocks = std::min(32, jobs[j].n_traj);
        ej[j].scale = jobs[j].beta / (double)jobs[j].n_step;
    }
    cudaStream_t st = ctx->stream;
    // host -> device copies of the tables (empty ones skipped)
    std::vector<std::tuple<void*, const void*, size_t>> copies = {
        {pl->tcut.ptr, tcut.data(), tcut.size() * sizeof(uint32_t)},
        {pl->jobs.ptr, bj.data(), bj.size() * sizeof(jz::BatchJob)},
        {pl->items.ptr, it.data(), it.size() * sizeof(int2)},
        {pl->est_jobs.ptr, ej.data(), ej.size() * sizeof(jz::EstJob)},
        {pl->sw_tcut.ptr, sw_tcut.data(), sw_tcut.size() * sizeof(uint32_t)}};
    for (auto& G : pl->sw)
        copies.emplace_back(G.jobs.ptr, G.h_jobs.data(), G.h_jobs.size() * sizeof(jz::JobDesc));
    for (auto& G : pl->therm)
        copies.emplace_back(G.jobs.ptr, G.h_jobs.data(), G.h_jobs.size() * sizeof(jz::JobDesc));
    for (const auto& c : copies) {
        if (std::get<2>(c) == 0) continue;
        if ((rc = cuda_err(cudaMemcpyAsync(std::get<0>(c), std::get<1>(c), std::get<2>(c),
                                           cudaMemcpyHostToDevice, st)))) {
            plan_release(pl);
            return rc;
        }
    }
    if ((rc = cuda_err(cudaStreamSynchronize(st)))) {
        plan_release(pl);
        return rc;
    }
    int per_sm = 0;
    cudaDeviceProp prop;
    if ((rc = cuda_err(jz::persistent_prepare(smem, cta, &per_sm))) ||
        (rc = cuda_err(cudaGetDeviceProperties(&prop, ctx->device)))) {
        plan_release(pl);
        return rc;
    }
    if (per_sm < 1 && pl->n_items > 0) {
        plan_release(pl);
        return ISING_ERR_UNSUPPORTED;
    }
    pl->grid = std::min(per_sm * prop.multiProcessorCount, pl->n_items);
    *out = pl;
    return ISING_OK;
}

// Enqueues the plan's work directly (no graph): counter reset, kernel, estimator.
int plan_enqueue(jz_plan* pl)
{
    cudaStream_t st = pl->ctx->stream;
    int rc;
    for (const auto& G : pl->therm) {
        if (!G.hbm) {
            if ((rc = cuda_err(jz::launch_sw(G.d, G.g, pl->K, (const jz::JobDesc*)G.jobs.ptr,
                                             G.n_jobs, G.n_cta, st))))
                return rc;
            continue;
        }
        for (const auto& w : G.waves)
            if ((rc = cuda_err(jz::launch_sw(G.d, G.g, pl->K,
                                             (const jz::JobDesc*)G.jobs.ptr + w.first, w.n_desc,
                                             w.n_cta, st, (uint32_t*)pl->therm_lattice.ptr))))
                return rc;
    }
    if (pl->n_items > 0) {
        if ((rc = cuda_err(cudaMemsetAsync(pl->counter.ptr, 0, sizeof(unsigned int), st))))
            return rc;
        if ((rc = cuda_err(jz::launch_persistent((const jz::BatchJob*)pl->jobs.ptr,
                                                 (const int2*)pl->items.ptr, pl->n_items,
                                                 (unsigned int*)pl->counter.ptr, pl->K, pl->grid,
                                                 pl->threads, pl->smem, st))))
            return rc;
    }
    for (const auto& G : pl->sw)
        if ((rc = cuda_err(jz::launch_sw(G.d, G.g, pl->K, (const jz::JobDesc*)G.jobs.ptr,
                                         G.n_jobs, G.n_cta, st))))
            return rc;
    if (pl->est_out)
        return cuda_err(jz::launch_estimator_batch((const jz::EstJob*)pl->est_jobs.ptr, pl->n_jobs,
                                                   pl->est_out, st));
    return ISING_OK;
}

int plan_capture(jz_plan* pl)
{
    cudaStream_t st = pl->ctx->stream;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return ISING_ERR_CUDA;
    }
    const int rc = plan_enqueue(pl);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (rc || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc ? rc : ISING_ERR_CUDA;
    }
    pl->graph = graph;
    if (cudaGraphInstantiate(&pl->exec, graph, 0) != cudaSuccess) {
        cudaGetLastError();
        pl->exec = nullptr;
        return ISING_ERR_CUDA;
    }
    return ISING_OK;
}

}  // namespace

extern "C" {

int jz_plan_create(ising_ctx* ctx, const jz_params* jobs, int n_jobs, int64_t* const* work_outs,
                   double* est_out, int cta_threads, jz_plan** out)
{
    if (!ctx || !jobs || n_jobs < 1 || !work_outs || !out) return ISING_ERR_ARG;
    *out = nullptr;
    if (cta_threads != 0 && (cta_threads < 32 || cta_threads > 512 || cta_threads % 32))
        return ISING_ERR_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ISING_ERR_CUDA;
    for (int j = 0; j < n_jobs; ++j) {
        const int rc = check_params(&jobs[j]);
        if (rc) return rc;
        if (jobs[j].seed != jobs[0].seed || !work_outs[j] || !is_device_ptr(work_outs[j]))
            return ISING_ERR_ARG;
    }
    if (est_out && !is_device_ptr(est_out)) return ISING_ERR_ARG;
    int rc;
    int cta = cta_threads;
    bool any_metropolis = false;
    for (int j = 0; j < n_jobs; ++j) any_metropolis |= jobs[j].update == 0;
    if (cta == 0 && !any_metropolis) cta = 256;   // nothing runs in the persistent kernel
    if (cta == 0) {
        // autotune on a reduced copy: 1/16 of the trajectories, 8 + 8 sweeps
        std::vector<jz_params> small(jobs, jobs + n_jobs);
        for (auto& p : small) {
            p.n_traj = std::max(1, p.n_traj / 16);
            p.n_therm = 8;
            p.n_step = 8;
            p.n_sweep = 1;
        }
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
            return ISING_ERR_CUDA;
        float best_ms = 1e30f;
        for (int cand : {256, 288, 384, 512}) {
            jz_plan* pl = nullptr;
            if (plan_build(ctx, small.data(), n_jobs, work_outs, nullptr, cand, &pl)) continue;
            float ms = 1e30f;
            if (!plan_enqueue(pl)) {
                cudaEventRecord(e0, ctx->stream);
                if (!plan_enqueue(pl)) {
                    cudaEventRecord(e1, ctx->stream);
                    if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
                }
            }
            cudaStreamSynchronize(ctx->stream);
            cudaGetLastError();
            plan_release(pl);
            if (ms < best_ms) {
                best_ms = ms;
                cta = cand;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (cta == 0) return ISING_ERR_UNSUPPORTED;
    }
    jz_plan* pl = nullptr;
    if ((rc = plan_build(ctx, jobs, n_jobs, work_outs, est_out, cta, &pl))) return rc;
    if ((rc = plan_capture(pl))) {
        plan_release(pl);
        return rc;
    }
    *out = pl;
    return ISING_OK;
}

int jz_plan_launch(jz_plan* plan)
{
    if (!plan || !plan->exec) return ISING_ERR_ARG;
    if (cudaSetDevice(plan->ctx->device) != cudaSuccess) return ISING_ERR_CUDA;
    return cuda_err(cudaGraphLaunch(plan->exec, plan->ctx->stream));
}

int jz_plan_info(const jz_plan* plan, int* cta_threads, int* grid, int* n_items)
{
    if (!plan) return ISING_ERR_ARG;
    if (cta_threads) *cta_threads = plan->threads;
    if (grid) *grid = plan->grid;
    if (n_items) *n_items = plan->n_items;
    return ISING_OK;
}

void jz_plan_free(jz_plan* plan)
{
    if (!plan) return;
    cudaSetDevice(plan->ctx->device);
    cudaStreamSynchronize(plan->ctx->stream);
    plan_release(plan);
}

}  // extern "C"
