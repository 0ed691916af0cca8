// jz_host.h -- host-side internals shared by the C-ABI translation units:
// the context, device-buffer bookkeeping, argument checks, FP64 threshold
// tables, launch-shape choice and the kernel launchers.  Not part of the ABI.
#pragma once
#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/isingjz.h"
#include "jz_device.cuh"

namespace jz {
size_t traj_smem_bytes(const Geom& g);
// gS: nullptr to keep the lattices in shared memory, else an HBM buffer of
// n_cta * sh.teams * 2 * NR * GW words, one slice per CTA.
cudaError_t launch_traj(int D, const Geom& g, const PhiloxKeys& K, const JobDesc* jobs,
                        int n_jobs, long long n_cta, const LaunchShape& sh, cudaStream_t st,
                        uint32_t* gS = nullptr);
// CTAs of shape sh resident per SM for the trajectory kernel launch_traj
// runs on g with its lattices in shared memory.
cudaError_t traj_occupancy(int D, const Geom& g, const LaunchShape& sh, int* ctas_per_sm);
cudaError_t launch_estimator(const long long* w_int, int n, double scale, int direction,
                             int n_blocks, double* out, cudaStream_t st);
size_t sw_smem_bytes(const Geom& g);
// Threads of one Swendsen-Wang CTA (one trajectory) for dimension D.
int sw_cta_threads(int D);
// Trajectories one launch of the HBM Swendsen-Wang variant keeps resident on
// the device at once (its occupancy x SMs): the chunk in which lattices beyond
// shared memory are thermalised, so that their HBM state stays one wave.
long long sw_hbm_wave(int D);
// gS: nullptr to keep each trajectory's state in shared memory, else an HBM
// buffer of n_cta * sw_smem_bytes(g) bytes, one slice per CTA.
cudaError_t launch_sw(int D, const Geom& g, const PhiloxKeys& K, const JobDesc* jobs,
                      int n_jobs, long long n_cta, cudaStream_t st, uint32_t* gS = nullptr);
double run_probe(int kind, int device);
// Status words of the bounds-checked build, one per translation unit with
// kernels (zeros in release builds): [0] = check sites that saw an index
// outside their array, [1] = one such index; clear resets them.
cudaError_t bounds_status_traj(unsigned int out[2], bool clear);
cudaError_t bounds_status_batch(unsigned int out[2], bool clear);
cudaError_t bounds_status_sw(unsigned int out[2], bool clear);
cudaError_t plain_trajectory(int D, const Geom& g, const PhiloxKeys& K, int l, int dir,
                             int n_step, int n_sweep, int n_therm, uint32_t traj,
                             const uint32_t tb[4], const uint32_t* tcut, int8_t* s,
                             long long* w, cudaStream_t st);
constexpr int kMaxJackBlocksHost = 64;
constexpr size_t kMaxSmemPerCta = 227 * 1024;
constexpr int kMaxTeamsHost = 64;   // teams per CTA
}  // namespace jz

// Grow-only device buffer charged against the context's HBM budget.
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
};

struct ising_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0;   // 0 = unlimited
    size_t used = 0;
    DevBuf tcut, jobs, work, spins, est_in, est_out;
    DevBuf lattice;   // HBM lattices of shapes too large for shared memory
    DevBuf therm;     // spins after Swendsen-Wang thermalisation (therm_update = 1)
    std::vector<uint32_t> h_tcut;
    std::vector<jz::JobDesc> h_jobs;
    // Launch shapes, guarded by shapes_mu (a server's worker thread reads them
    // while the context's own thread may tune or fix them):
    std::mutex shapes_mu;
    std::map<std::tuple<int, int, int>, int> threads;   // per-shape CTA size (tuned)
    // default shapes already scored, by (d, L, L_t, n, trajectories per launch)
    std::map<std::tuple<int, int, int, int, long long>, jz::LaunchShape> default_shapes;
    // device time of the last run call's kernel launches (ising_last_launch_ms):
    // ev_k0 before its first launch, ev_k1 after its last one
    cudaEvent_t ev_k0 = nullptr, ev_k1 = nullptr;
    bool k_open = false;    // the next launch is the call's first
    bool k_timed = false;   // a run call has recorded both events
    std::atomic<int> cancel{0};   // ising_cancel: run calls refuse new work while set
    std::string gpu_name;         // device name (autotune cache key)
};

namespace jzh {
// NVTX range around a host phase (visible in Nsight timelines; a no-op
// unless a tool is attached).
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};
int ensure(ising_ctx* ctx, DevBuf& b, size_t bytes);
int is_device_ptr(const void* p);
int check_params(const jz_params* p);
int nrep_of(const jz_params& p);
void cut_range(const jz_params& p, int* g0, int* g1);
jz::Geom make_geom(int d, int L, int Lt, int nrep);
uint32_t threshold(double x);
jz::PhiloxKeys key_schedule(uint64_t seed);
void build_tables(const jz_params& p, uint32_t tb[4], std::vector<uint32_t>& tcut, size_t off);
// The same tables written to tcut[0 .. n_step * 8d) (bond tables: n_step * 2).
void build_tables_into(const jz_params& p, uint32_t tb[4], uint32_t* tcut);
void build_bond_tables_into(const jz_params& p, uint32_t tb[4], uint32_t* tcut);
uint32_t bond_threshold(double x);
void step_weights(const jz_params& p, long long k, long long* den, long long* w_self,
                  long long* w_glue);
void build_bond_tables(const jz_params& p, uint32_t tb[4], std::vector<uint32_t>& tcut,
                       size_t off);
bool sw_fits(const jz::Geom& g);
bool sw_therm(const jz_params& p);
jz::LaunchShape shape_for(const jz::Geom& g, int cta_threads);
bool shape_fits(const jz::Geom& g);
bool threads_fit(const jz::Geom& g);
bool threads_ok(const jz::Geom& g, int threads);
jz::LaunchShape default_shape(int d, const jz::Geom& g, long long n_traj);
jz::LaunchShape ctx_shape(ising_ctx* ctx, int d, const jz::Geom& g, long long n_traj);
int cuda_err(cudaError_t e);
int run_jobs(ising_ctx* ctx, const jz_params* jobs, int n_jobs, int64_t* const* outs,
             int8_t* const* spins);
// Protocol steps [k_begin, k_end) resumed from stored spins and W_int (k_begin > 0).
struct Segment {
    int k_begin, k_end;
    const int8_t* spins_in;
    const long long* w_in;
};
}  // namespace jzh
