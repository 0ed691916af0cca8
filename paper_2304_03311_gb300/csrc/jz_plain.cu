// jz_plain.cu -- the plain GPU form of the method, kept as the comparison
// baseline: one trajectory per launch, one launch per half-sweep (plus one per
// protocol step for the work increment), spins as int8 +-1 in global memory in
// the natural order [r][t][y][x], one thread per Philox block of four
// same-colour sites.  It follows the same random-stream and acceptance
// conventions as the fused kernel, so its results are bit-identical; only the
// execution strategy differs.
#include <cuda_runtime.h>

#include <cstdint>

#include "jz_device.cuh"

namespace jz {

struct PlainArgs {
    Geom g;
    int D;
    uint32_t traj, c3base;
    int l, lg, k, n_step, w_self, w_glue;
    uint32_t sweep;
    uint32_t tb0, tb1, tb2;
    const uint32_t* tcut;
};

__device__ __forceinline__ int nat(const Geom& g, int r, int t, int y, int x)
{
    return ((r * g.Lt + t) * g.Ly + y) * g.L + x;
}

__global__ void plain_hot_start(int8_t* s, const PlainArgs A, const PhiloxKeys K)
{
    const Geom& g = A.g;
    const int items = g.NR * g.G;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= 2 * items) return;
    const int c = gid / items, idx = gid - c * items;
    const int R = idx / g.G, q = idx - R * g.G;
    const int y = R % g.Ly, tr = R / g.Ly, t = tr % g.Lt;
    const int p = (c + t + y) & 1;
    const uint4 u = philox((uint32_t)idx, 0u, A.traj, (uint32_t)c | A.c3base | (1u << 30), K);
    for (int j = 0; j < 4; ++j) {
        const int h = 4 * q + j;
        if (h >= g.Lh) break;
        s[R * g.L + 2 * h + p] = (word_of(u, j) >> 31) ? (int8_t)-1 : (int8_t)1;
    }
}

__global__ void plain_half_sweep(int8_t* s, const PlainArgs A, const PhiloxKeys K, int c)
{
    const Geom& g = A.g;
    const int items = g.NR * g.G;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= items) return;
    const int R = idx / g.G, q = idx - R * g.G;
    const int y = R % g.Ly, tr = R / g.Ly, t = tr % g.Lt, r = tr / g.Lt;
    const int p = (c + t + y) & 1;
    const uint4 u = philox((uint32_t)idx, A.sweep, A.traj, (uint32_t)c | A.c3base, K);
    for (int j = 0; j < 4; ++j) {
        const int h = 4 * q + j;
        if (h >= g.Lh) break;
        const int x = 2 * h + p;
        const int i = nat(g, r, t, y, x);
        const int si = s[i];
        int a = si * (s[nat(g, r, t, y, (x + 1) % g.L)] + s[nat(g, r, t, y, (x + g.L - 1) % g.L)]);
        if (A.D == 3)
            a += si * (s[nat(g, r, t, (y + 1) % g.Ly, x)] + s[nat(g, r, t, (y + g.Ly - 1) % g.Ly, x)]);
        // temporal links; the link (t, t+1) is cut iff t == 0
        int b = 0, cc = 0;
        bool special = false;
        for (int side = 0; side < 2; ++side) {
            const int tn = side ? (t + 1) % g.Lt : (t + g.Lt - 1) % g.Lt;
            const bool cut = (side ? t : tn) == 0;
            if (!cut) {
                a += si * s[nat(g, r, tn, y, x)];
                continue;
            }
            const int rg = side ? (r + 1) & 1 : (r + 1) & 1;   // n = 2: r+1 = r-1
            const int self_v = s[nat(g, r, tn, y, x)], glue_v = s[nat(g, rg, tn, y, x)];
            if (A.k >= 0 && x == A.l) {
                b = si * self_v;
                cc = si * glue_v;
                special = true;
            } else {
                a += si * (x < A.lg ? glue_v : self_v);
            }
        }
        bool flip;
        const uint32_t uw = word_of(u, j);
        if (!special) {
            const int m = a;
            const uint32_t T = m == 2 * A.D ? A.tb0 : m == 2 * A.D - 2 ? A.tb1 : A.tb2;
            flip = m <= 0 || uw < T;
        } else {
            const int m = a * A.n_step + b * A.w_self + cc * A.w_glue;
            const int ti = (((a + 2 * A.D - 1) >> 1) * 2 + (b > 0)) * 2 + (cc > 0);
            flip = m <= 0 || uw < A.tcut[A.k * 8 * A.D + ti];
        }
        if (flip) s[i] = (int8_t)-si;
    }
}

__global__ void plain_work(const int8_t* s, const Geom g, int l, int dir, long long* w)
{
    int e = 0;
    for (int i = threadIdx.x; i < 2 * g.Ly; i += blockDim.x) {
        const int r = i / g.Ly, y = i % g.Ly;
        e += s[nat(g, r, 0, y, l)] *
             (s[nat(g, r, 1, y, l)] - s[nat(g, (r + 1) & 1, 1, y, l)]);
    }
    e = __reduce_add_sync(0xFFFFFFFFu, e);
    if (threadIdx.x == 0 && e != 0) atomicAdd((unsigned long long*)w, (unsigned long long)(long long)(dir * e));
}

// Runs one trajectory: hot start, thermalisation, protocol; w (device, one
// int64, zeroed here) receives W_int; the spins stay in `s` (natural order).
cudaError_t plain_trajectory(int D, const Geom& g, const PhiloxKeys& K, int l, int dir,
                             int n_step, int n_sweep, int n_therm, uint32_t traj,
                             const uint32_t tb[4], const uint32_t* tcut, int8_t* s,
                             long long* w, cudaStream_t st)
{
    PlainArgs A;
    A.g = g;
    A.D = D;
    A.traj = traj;
    A.c3base = ((uint32_t)(dir < 0) << 1) | ((uint32_t)l << 2);
    A.l = l;
    A.lg = dir > 0 ? l : l + 1;
    A.k = -1;
    A.n_step = n_step;
    A.w_self = A.w_glue = 0;
    A.tb0 = tb[0];
    A.tb1 = tb[1];
    A.tb2 = tb[2];
    A.tcut = tcut;
    const int items = g.NR * g.G;
    const int T = 128;
    cudaMemsetAsync(w, 0, sizeof(long long), st);
    plain_hot_start<<<(2 * items + T - 1) / T, T, 0, st>>>(s, A, K);
    uint32_t sweep = 0;
    for (int i = 0; i < n_therm; ++i, ++sweep) {
        A.sweep = sweep;
        plain_half_sweep<<<(items + T - 1) / T, T, 0, st>>>(s, A, K, 0);
        plain_half_sweep<<<(items + T - 1) / T, T, 0, st>>>(s, A, K, 1);
    }
    A.lg = l;
    for (int k = 0; k < n_step; ++k) {
        plain_work<<<1, 32, 0, st>>>(s, g, l, dir, w);
        A.k = k;
        A.w_self = dir > 0 ? n_step - (k + 1) : k + 1;
        A.w_glue = dir > 0 ? k + 1 : n_step - (k + 1);
        for (int i = 0; i < n_sweep; ++i, ++sweep) {
            A.sweep = sweep;
            plain_half_sweep<<<(items + T - 1) / T, T, 0, st>>>(s, A, K, 0);
            plain_half_sweep<<<(items + T - 1) / T, T, 0, st>>>(s, A, K, 1);
        }
    }
    return cudaGetLastError();
}

}  // namespace jz
