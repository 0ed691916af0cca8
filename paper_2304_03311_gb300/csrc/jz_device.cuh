// jz_device.cuh -- device-side building blocks of the replica-gluing kernels.
//
// Spin storage in shared memory (one trajectory per team of threads):
//   S[c][R][q]  uint32 words, c = colour, R = (r L_t + t) L_y + y the row,
//               q < GW = ceil((L/2)/8) the word within the row.  Nibble j of
//               word q holds the colour-c site h = 8q + j of row R, x = 2h + p
//               with p = (c + t + y) mod 2; 0 for spin +1 and 1 for -1.
// With this layout the four (2D) or six (3D) neighbours of the eight sites of
// one word are, in the other colour: the same word of rows t-1, t+1 (and
// y-1, y+1), the same word of the same row (one x neighbour), and that word
// shifted by one nibble (the other x neighbour).  Two Philox4x32-10 blocks
// give the eight acceptance words of one spin word.
#pragma once
#include <cstdint>

namespace jz {

constexpr int kMaxJobsPerLaunch = 4096;

// Bounds-checked builds (compiled with -DJZ_BOUNDS_CHECK: the debug library).
// Every lattice access of the trajectory kernels and every label / spin-bit
// access of the Swendsen-Wang kernel checks its index against its array; an
// index outside it sets bit `site` of this translation unit's status word
// (entry 0; entry 1 keeps one offending index) and the access is skipped.
// Release builds compile each check to nothing.
#ifdef JZ_BOUNDS_CHECK
static __device__ unsigned int jz_bounds_status[2];
__device__ __forceinline__ bool in_bounds(long long i, long long n, int site)
{
    if (i >= 0 && i < n) return true;
    atomicOr(&jz_bounds_status[0], 1u << site);
    jz_bounds_status[1] = (unsigned int)i;
    return false;
}
#else
__device__ __forceinline__ bool in_bounds(long long, long long, int) { return true; }
#endif

// Philox4x32-10 round constants and Weyl key increments (Salmon, Moraes, Dror
// and Shaw, SC'11).
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// Key schedule of one launch: k0[i], k1[i] for rounds i = 0..9.  Passed by
// value as a kernel parameter, so every round key is a constant-bank operand.
struct PhiloxKeys {
    uint32_t k0[10];
    uint32_t k1[10];
};

// Lattice shape of one launch (all jobs of a launch share it).
struct Geom {
    int L, Lt, Ly;      // spatial extent, time extent, L in 3D / 1 in 2D
    int Lh;             // L / 2 sites of one colour per row
    int G;              // Philox blocks per row, ceil(Lh / 4) (the random-stream layout)
    int GW;             // shared-memory words per row, ceil(Lh / 8) (8 sites per word)
    int nrep;           // replicas n
    int NR;             // rows per colour, n * Lt * Ly
};

// How one launch maps trajectories onto threads: a team of team_threads runs
// one trajectory; a CTA of cta_threads holds `teams` teams.  warp: every team
// lies inside one warp and synchronises with __syncwarp (no cross-warp
// barrier); otherwise the CTA is one team and uses __syncthreads.
struct LaunchShape {
    int team_threads;
    int teams;
    int cta_threads;
    int warp;
};

// Per-job (one transformation) parameters, device copy.
struct JobDesc {
    int l;              // switched column
    int n_step, n_sweep, n_therm;
    int dir;            // +1 forward, -1 reverse
    int n_traj;
    int prot;           // 1: every switched column together; 2: one column y at a time
    int g0, g1;         // columns x < g0 glued, g0 <= x < g1 switching, x >= g1 self
    int k_begin, k_end; // protocol steps run: [k_begin, k_end); 0 starts from the hot start
    int start_in;       // 1: step k_begin = 0 starts from spins_in (thermalised elsewhere)
    const int8_t* spins_in;     // k_begin > 0 or start_in: [n_traj][V] state after step k_begin - 1
    const long long* w_in;      // k_begin > 0: [n_traj] W_int of steps 0 .. k_begin - 1
    long long traj0;    // global index of the job's first trajectory
    long long cta0;     // first CTA of the job in the launch grid
    uint32_t tb[4];     // bulk thresholds by anti-aligned neighbour count a:
                        // tb[a] = T(m = 2D - 2a), a < D
    const uint32_t* tcut;   // [n_step][8D] switched-site thresholds
    long long* w_out;       // [n_traj] W_int
    int8_t* spins_out;      // [n_traj][V] final spins (+-1) or nullptr
};

// One job of a persistent batch launch.
struct BatchJob {
    JobDesc J;            // thresholds, outputs, trajectory range
    Geom g;
    int D, fast;
    LaunchShape sh;       // team size, teams per CTA (= trajectories per work item), barrier
    int lattice_words;    // 2 * NR * GW spin words per team
};

// One job of the batched estimator.
struct EstJob {
    const long long* w;   // n work values W_int
    int n;
    int direction;
    int n_blocks;         // jackknife blocks, <= 64 and <= n
    double scale;         // beta / N
};

// One Philox4x32-10 block.
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        const PhiloxKeys& K)
{
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint64_t p0 = (uint64_t)kPhiloxM0 * c0;
        const uint64_t p1 = (uint64_t)kPhiloxM1 * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ K.k0[i];
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ K.k1[i];
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
    }
    return make_uint4(c0, c1, c2, c3);
}

// One block with round 0's two products supplied: p0 = M0 * c0 and
// (hi1, lo1) = M1 * c2.  Counter word 2 is the trajectory index, fixed for a
// whole trajectory, and successive blocks of a thread step c0 by a constant,
// so callers form p0 by 64-bit additions instead of a wide multiply.
__device__ __forceinline__ uint4 philox_p0(uint64_t p0, uint32_t c1, uint32_t hi1, uint32_t lo1,
                                           uint32_t c3, const PhiloxKeys& K)
{
    uint32_t c0 = hi1 ^ c1 ^ K.k0[0];
    uint32_t c2 = (uint32_t)(p0 >> 32) ^ c3 ^ K.k1[0];
    c1 = lo1;
    c3 = (uint32_t)p0;
#pragma unroll
    for (int i = 1; i < 10; ++i) {
        const uint64_t q0 = (uint64_t)kPhiloxM0 * c0;
        const uint64_t q1 = (uint64_t)kPhiloxM1 * c2;
        const uint32_t n0 = (uint32_t)(q1 >> 32) ^ c1 ^ K.k0[i];
        const uint32_t n2 = (uint32_t)(q0 >> 32) ^ c3 ^ K.k1[i];
        c1 = (uint32_t)q1;
        c3 = (uint32_t)q0;
        c0 = n0;
        c2 = n2;
    }
    return make_uint4(c0, c1, c2, c3);
}

// The same block with only round 0's product M1 * c2 supplied (hi1, lo1).
__device__ __forceinline__ uint4 philox_r0(uint32_t c0, uint32_t c1, uint32_t hi1, uint32_t lo1,
                                           uint32_t c3, const PhiloxKeys& K)
{
    return philox_p0((uint64_t)kPhiloxM0 * c0, c1, hi1, lo1, c3, K);
}

// The last stage of the FP64 estimator of one job (Appendix A, eq.
// Jarzynski_theorem; blocked jackknife), given each jackknife block's maximum
// m_b of -W_i and shifted sum s_b = sum_i e^{-W_i - m_b} (rows lo[b] ..
// lo[b+1] - 1).  Thread b < B forms the estimate without block b, thread B
// the full one, both as max-shifted log-sum-exps over the blocks; thread 0
// then writes out[0] = ln <e^-W>, out[1] = Delta S, out[2] = the jackknife
// error.  Every thread of the CTA calls it (it holds a barrier).
__device__ __forceinline__ void estimator_finish(const double* s_max, const double* s_sum,
                                                 const int* s_lo, int B, int n, int direction,
                                                 double* s_theta, double* out)
{
    const int t = (int)threadIdx.x;
    if (t == B || (t < B && B >= 2)) {
        const int skip = t < B ? t : -1;
        const int count = t < B ? n - (s_lo[t + 1] - s_lo[t]) : n;
        double M = -INFINITY;
        for (int b = 0; b < B; ++b) if (b != skip) M = fmax(M, s_max[b]);
        double tot = 0.0;
        for (int b = 0; b < B; ++b) if (b != skip) tot += s_sum[b] * exp(s_max[b] - M);
        s_theta[t] = M + log(tot) - log((double)count);
    }
    __syncthreads();
    if (t != 0) return;
    const double sign = direction > 0 ? -1.0 : 1.0;
    const double full = s_theta[B];
    double err = 0.0;
    if (B >= 2) {
        double mean = 0.0;
        for (int b = 0; b < B; ++b) mean += sign * s_theta[b];
        mean /= B;
        double ss = 0.0;
        for (int b = 0; b < B; ++b) {
            const double d = sign * s_theta[b] - mean;
            ss += d * d;
        }
        err = sqrt((double)(B - 1) / B * ss);
    }
    out[0] = full;
    out[1] = sign * full;
    out[2] = err;
}

__device__ __forceinline__ uint32_t word_of(const uint4& u, int j)
{
    return j == 0 ? u.x : j == 1 ? u.y : j == 2 ? u.z : u.w;
}

}  // namespace jz
