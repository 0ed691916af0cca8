/*
 * isingjz.h -- C ABI of the GB300 (sm_103a) library for the Jarzynski
 * replica-gluing estimator of Renyi-2 entanglement entropy increments and the
 * entropic c-function (Bulgarelli & Panero, arXiv:2304.03311).
 *
 * What the library computes (one "transformation" l -> l+1):
 *   n = 2 replicas of a periodic Ising lattice of L^(d-1) x L_t sites
 *   (section 1, eq. Ising_model: H/T = -beta sum s_i s_j) are cut at the time
 *   slice tau_c = 0: for columns x < l the temporal link t = 0 -> 1 joins
 *   replica r to replica r+1, for x > l it stays in replica r (section 3, the
 *   replica H/T with couplings beta^(k,k), beta^(k,k+1)).  The column x = l is
 *   switched linearly, self coupling beta (1 - lambda_k), glue coupling
 *   beta lambda_k, lambda_k = k/N (section 3, last paragraphs of the protocol
 *   description).  Each trajectory starts from an independent hot start and
 *   n_therm checkerboard Metropolis sweeps at lambda_0, then for k = 0..N-1
 *   accumulates the integer work increment dE_k = H_{lambda_{k+1}} -
 *   H_{lambda_k} in units of beta/N (Appendix A, eq. work_in_one_MC_step) and
 *   runs n_sweep sweeps at lambda_{k+1} (Appendix A, remark after eq.
 *   discretized_average_exp_work).  <e^-W>, W = beta W_int / N, estimates
 *   Z_2(l+1)/Z_2(l) (Appendix A, eq. Jarzynski_theorem), so
 *   Delta S_2 = -ln <e^-W> (section 2, eq. definition_of_derivative_of_Renyi_entropy).
 *
 * Bit-level conventions (random stream and acceptance) are fixed so that runs
 * are reproducible and independent of batching:
 *   colour  c = (x + y + t) mod 2, colour 0 then colour 1 in each sweep;
 *   row     R = (r L_t + t) L_y + y (L_y = L in 3D, 1 in 2D); the colour-c sites
 *           of a row are x = 2h + ((c + t + y) mod 2), h < L/2; site h takes
 *           word h mod 4 of the Philox4x32-10 block q = h / 4 with
 *           counter (R ceil(L/8) + q, s, traj, c | dir<<1 | l<<2 | phase<<30),
 *           key (lo32 seed, hi32 seed); s = 0..n_therm-1 for thermalisation and
 *           n_therm + k n_sweep + i for protocol sweep i of step k; phase 1 with
 *           s = 0 is the hot start (spin -1 iff the word's top bit is set);
 *   accept  flip iff m <= 0 or word < T, T = min(floor(2^32 exp(-x)), 2^32-1),
 *           bulk: m = s_i sum_j s_j, x = 2.0*beta*m;
 *           switched site in the protocol: m = a N + b w_self + c w_glue with
 *           a the sum over its 2d-1 fixed links, b, c its self and glue bond
 *           products, (w_self, w_glue) = (N-k-1, k+1) forward and
 *           (k+1, N-k-1) reverse, x = (2.0*beta*m)/N.  Thresholds are computed
 *           on the host in IEEE double with the C library's exp.
 *
 * Memory: the caller owns every output buffer; the library owns its device
 * state.  Output pointers may be host or device memory: with device memory
 * the call only enqueues work on the context's stream (use ising_sync); with
 * host memory the call copies back and returns when the result is there.
 * Errors are returned as negative codes; nothing throws across this ABI.
 * A context must not be used from two host threads at once.
 */
#ifndef ISINGJZ_H
#define ISINGJZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------- error codes -- */
#define ISING_OK               0
#define ISING_ERR_ARG         -1  /* null pointer, non-positive count, bad beta  */
#define ISING_ERR_ODD_EXTENT  -2  /* L or L_t odd (checkerboard needs even)      */
#define ISING_ERR_L_RANGE     -3  /* l outside 0 <= l <= L-1                     */
#define ISING_ERR_NOMEM       -4  /* device allocation or HBM budget exceeded    */
#define ISING_ERR_CUDA        -5  /* a CUDA runtime call failed                  */
#define ISING_ERR_TIMEOUT     -6  /* a bounded device wait gave up               */
#define ISING_ERR_UNSUPPORTED -7  /* d not in {2,3}, lattice too large, option not served */
#define ISING_ERR_NOT_FOUND   -8  /* unknown job id                              */
#define ISING_ERR_PENDING     -9  /* job not finished yet (jz_poll)              */
#define ISING_ERR_SCRATCH_LIMIT -10 /* too large for jarzynski_run_noalloc     */
#define ISING_ERR_CANCELLED   -11 /* stopped by ising_cancel / jz_cancel          */

/* Opaque per-device context: stream, device buffers, autotune choices. */
typedef struct ising_ctx ising_ctx;

/* One transformation l -> l+1 (direction +1) or l+1 -> l (direction -1).
 *   d          lattice dimension D, 2 or 3 (section 3, "extension to higher
 *              dimensions"); time is one of the D directions
 *   L, L_t     spatial and temporal extents, both even, L >= 2, L_t >= 2
 *   update     the Monte Carlo update of every sweep (section 3):
 *              0  checkerboard Metropolis, one site at a time (the default);
 *              1  Swendsen-Wang clusters: a link of coupling K between equal
 *                 spins becomes a bond with probability 1 - e^{-2K} and every
 *                 cluster of bonded sites flips with probability 1/2.  One CTA
 *                 per trajectory; its state takes about 4.5 V (2D) or 4.6 V
 *                 (3D) bytes for the V = n L_t L^(d-1) sites, in shared memory
 *                 up to 227 KiB (V up to about 50,000), beyond that in an HBM
 *                 slice per CTA.
 *                 Served by jarzynski_run_ex, jarzynski_run_batch,
 *                 jarzynski_run_segment, jarzynski_run_noalloc, the
 *                 persistent plans and the server (jz_submit);
 *                 jarzynski_run_plain and ising_autotune's timing do not
 *                 serve it (ISING_ERR_UNSUPPORTED, resp. the fixed CTA size).
 *              Other values: ISING_ERR_ARG.
 *   beta       coupling, 0 <= beta <= 4
 *   l          width of region A before the move, 0 <= l <= L-1
 *   n_step     N >= 1 protocol steps, n_sweep >= 1 sweeps per step
 *   n_therm    thermalisation sweeps of the start ensemble (section 4 uses 1000)
 *   n_traj     trajectories, traj0 the global index of the first one (the index
 *              enters the random counter, so a range split gives the same result)
 *   seed       Philox key
 *   protocol   0 or 1: protocol 1, every switched column (x = l, y) moves
 *              together, lambda_k = k/N (section 3); 2: protocol 2 (Appendix B),
 *              the L_y columns move one after another, m = N/L_y steps each
 *              (n_step must be a multiple of L_y, else ISING_ERR_ARG); the work
 *              of the moving column is scaled by L_y so that W = (beta/N) W_int
 *              in both.  In 2D both protocols are the same computation.
 *              jarzynski_run_plain refuses protocol 2 in 3D
 *              (ISING_ERR_UNSUPPORTED).
 *   n_replica  n, the number of replicas (section 2: Tr rho_A^n = Z_n / Z^n);
 *              0 or 2 for the paper's n = 2, at most 8.  The glue of replica r
 *              lands in replica r+1 mod n.  -ln<e^-W> then estimates
 *              (n-1) Delta S_n.
 *   whole      0: the transformation moves the end of region A by one column
 *              (x < l glued, column l switching; 0 <= l <= L-1).  1: Alba et
 *              al.'s whole-cut transformation (section 3, eq.
 *              off-equilibrium_evolution_of_the_couplings): the columns x < l
 *              switch together from n decoupled replicas to glued ones
 *              (1 <= l <= L, protocol 1 only), so <e^-W> = Z_n(l)/Z^n and
 *              -ln<e^-W> = (n-1) S_n(l).  jarzynski_run_plain refuses
 *              n_replica != 2 and whole = 1 (ISING_ERR_UNSUPPORTED).
 *   therm_update  the update of the n_therm thermalisation sweeps: 0 (the
 *              default) the protocol's own `update`; 1 Swendsen-Wang clusters
 *              before a Metropolis protocol.  Jarzynski's identity needs only
 *              an equilibrium start and sweeps that keep each step's Boltzmann
 *              weight (Appendix A), and section 4 thermalises with cluster
 *              steps, which decorrelate at criticality where Metropolis sweeps
 *              do not.  The thermalisation sweeps then take the Swendsen-Wang
 *              random stream of their sweep indices 0 .. n_therm-1, the
 *              protocol sweeps the Metropolis stream of theirs, as in one run
 *              of each update.  Served by jarzynski_run_ex, jarzynski_run_batch,
 *              jarzynski_run_segment (a segment from k_begin = 0) and the
 *              server (jz_submit; the job's memory then includes n_traj V
 *              bytes of thermalised spins) and the persistent plans (the
 *              thermalisation launches ahead of the persistent kernel, in its
 *              graph).  A Swendsen-Wang state beyond shared memory is
 *              thermalised from HBM slices, in launches of one resident wave
 *              of trajectories, whose slices the server also charges to the
 *              job.  jarzynski_run_plain and jarzynski_run_noalloc return
 *              ISING_ERR_UNSUPPORTED.  Other values: ISING_ERR_ARG. */
typedef struct jz_params {
    int d, L, L_t;
    int update;
    double beta;
    int l;
    int n_step, n_sweep, n_therm;
    int n_traj;
    int direction;
    long long traj0;
    uint64_t seed;
    int protocol;
    int n_replica;
    int whole;
    int therm_update;
} jz_params;

/* Fills *p with defaults (n_therm = 1000, direction = +1, traj0 = 0, n_sweep = 1,
 * seed = 0, update = 0, protocol = 1, n_replica = 2, whole = 0, therm_update = 0)
 * and zero sizes;
 * returns ISING_OK or ISING_ERR_ARG for p == NULL. */
int jz_params_default(jz_params* p);

/* Creates a context on CUDA device `device`.
 *   hbm_budget_bytes  cap on the library's own device allocations (0 = no cap);
 *                     exceeding it returns ISING_ERR_NOMEM
 *   cuda_stream       cudaStream_t to enqueue on (NULL = the library creates one)
 * Writes the context to *out.  Errors: ISING_ERR_ARG, ISING_ERR_CUDA. */
int ising_replica_init(ising_ctx** out, int device, size_t hbm_budget_bytes,
                       void* cuda_stream);

/* Releases the context and its device memory (waits for queued work). */
void ising_replica_free(ising_ctx* ctx);

/* Blocks until all work queued on the context's stream is done.  Returns
 * ISING_OK, or the first deferred error of queued work. */
int ising_sync(ising_ctx* ctx);

/* Device time, in milliseconds, of the trajectory kernel launches of the last
 * run call on this context (jarzynski_run, _ex, _batch, _segment and the
 * autotuner's trial runs; not the plain baseline, the estimator or plans):
 * from CUDA events recorded on the context's stream just before the call's
 * first kernel launch and just after its last one, so the call's table and
 * result copies are excluded (and, for a batch of several lattice shapes,
 * the copies between its launches are included).  Waits for that launch to
 * finish.  *ms is written on success.  Errors: ISING_ERR_ARG when the last
 * run call launched no kernel (there was none yet, or it returned an error
 * before its first launch), ISING_ERR_CUDA.  This is measurement support for the section 3
 * trajectory step; the paper defines no such call. */
int ising_last_launch_ms(ising_ctx* ctx, float* ms);

/* Runs n_traj trajectories of the forward transformation l -> l+1 with
 * n_therm = 1000 and trajectory indices 0..n_traj-1 (section 3 protocol,
 * Appendix A work).  work_int_out[i] (caller-owned, n_traj int64 entries,
 * host or device memory) receives W_int of trajectory i; W = beta W_int / N.
 * Errors: ISING_ERR_ARG, ISING_ERR_ODD_EXTENT, ISING_ERR_L_RANGE,
 * ISING_ERR_UNSUPPORTED, ISING_ERR_NOMEM, ISING_ERR_CUDA. */
int jarzynski_run(ising_ctx* ctx, int d, int L, int L_t, double beta, int l,
                  int n_step, int n_sweep, int n_traj, uint64_t seed,
                  int64_t* work_int_out);

/* As jarzynski_run with every parameter of jz_params.  spins_out (nullable,
 * caller-owned, host or device) receives the final configuration of each
 * trajectory as int8 +-1 in the order [traj][r][t][y][x] (x fastest, n_traj *
 * n * L_t * L_y * L bytes).  A Metropolis replica lattice (n * L_t * L_y * L
 * / 4 bytes nibble-packed) that does not fit one CTA's 227 KiB of shared
 * memory runs from an HBM slice per CTA instead (for example the paper's 3D
 * L = 48, L_t = 4L lattice); such shapes need only L_y ceil(L/16) <= 512, and
 * the persistent plan, server, allocation-free call and autotuner refuse them
 * (ISING_ERR_UNSUPPORTED). */
int jarzynski_run_ex(ising_ctx* ctx, const jz_params* p, int64_t* work_int_out,
                     int8_t* spins_out);

/* Checkpoint / resume: runs only protocol steps k_begin .. k_end-1 of the
 * transformation p (0 <= k_begin < k_end <= n_step).  spins_io (device memory,
 * n_traj * n * L_t * L_y * L int8, order as jarzynski_run_ex's spins_out) and
 * work_io (device memory, n_traj int64) carry the state between segments: for
 * k_begin = 0 the trajectories start from the hot start and n_therm sweeps and
 * their inputs are ignored; for k_begin > 0 they hold the configuration after
 * step k_begin-1 and W_int of steps 0 .. k_begin-1.  On return (after
 * ising_sync) spins_io holds the configuration after step k_end-1 and work_io
 * W_int of steps 0 .. k_end-1.  The random counter is a function of the
 * global sweep index, so any split of [0, n_step) into segments gives the bits
 * of one jarzynski_run_ex call; the paper has no such facility.  Errors: as
 * jarzynski_run_ex, and ISING_ERR_ARG for an empty or out-of-range step range
 * or host buffers. */
int jarzynski_run_segment(ising_ctx* ctx, const jz_params* p, int k_begin, int k_end,
                          int64_t* work_io, int8_t* spins_io);

/* Cancellation and resumable runs; the paper has no counterpart.
 * ising_cancel sets the context's cancel flag (an atomic host flag; safe to
 * call from any host thread while another thread is inside a run call).
 * While it is set, every run call on the context (jarzynski_run, _ex, _batch,
 * _segment, _plain, _resumable, ising_autotune) returns ISING_ERR_CANCELLED
 * instead of enqueuing more work; work already on the device runs to its end
 * (no kernel is interrupted).  _batch and _plain test the flag between their
 * launches.  ising_cancel_reset clears it.  Errors: ISING_ERR_ARG (NULL). */
int ising_cancel(ising_ctx* ctx);
int ising_cancel_reset(ising_ctx* ctx);

/* A long transformation run as a sequence of protocol segments of
 * steps_per_segment steps (jarzynski_run_segment semantics: the random counter
 * is a function of the global sweep index, so the bits equal those of one
 * jarzynski_run_ex call), with the cancel flag tested between segments.
 *   *k_done    in: protocol steps already done (0 = start from the hot start;
 *              otherwise work_io / spins_io hold the state after step
 *              *k_done - 1); out: steps done when the call returns
 *   max_segments  0 = run to the end; > 0 = stop after that many segments
 *   work_io, spins_io  device buffers as for jarzynski_run_segment
 * At most two segments are in flight, so a cancel takes effect within about
 * two segments' time.  Returns ISING_OK when *k_done = n_step (the call has
 * synchronised the context's stream), ISING_ERR_PENDING when max_segments
 * stopped it, ISING_ERR_CANCELLED when the flag stopped it; in both of the
 * latter cases the buffers hold the consistent state after step *k_done - 1
 * and a later call (after ising_cancel_reset) resumes from there.  Errors: as
 * jarzynski_run_segment, ISING_ERR_ARG for steps_per_segment < 1 or *k_done
 * outside [0, n_step]. */
int jarzynski_run_resumable(ising_ctx* ctx, const jz_params* p, int steps_per_segment,
                            int max_segments, int* k_done, int64_t* work_io, int8_t* spins_io);

/* Runs n_jobs transformations in one device launch per lattice shape (jobs of
 * equal (d, L, L_t) share a launch; the c-function scan of section 3 is one
 * call with one job per l).  work_outs[j] is job j's caller-owned output of
 * jobs[j].n_traj entries; all of them must be host memory, or all device
 * memory.  Each job's result is bit-identical to running it alone. */
int jarzynski_run_batch(ising_ctx* ctx, const jz_params* jobs, int n_jobs,
                        int64_t* const* work_outs);

/* Uneven batches (section 3 protocol for every job; lattices of different
 * d, L, L_t and any l) as ONE persistent launch, captured with the batched
 * FP64 estimator into a CUDA graph that jz_plan_launch replays.  Swendsen-Wang
 * jobs (update = 1) join the same graph as one launch per lattice shape (one
 * CTA per trajectory) after the persistent kernel; every job's lattice must
 * fit one CTA's shared memory (ISING_ERR_UNSUPPORTED otherwise).
 *   jobs, n_jobs  the transformations; all must share one seed
 *   work_outs     n_jobs caller-owned DEVICE buffers, jobs[j].n_traj int64 each
 *   est_out       caller-owned DEVICE buffer of 3 n_jobs doubles (nullable):
 *                 per job ln <e^-W>, Delta S_2 and its jackknife error, as
 *                 estimator_reduce with 32 blocks
 *   cta_threads   CTA size of the persistent kernel (0 = autotune: each of
 *                 256, 288, 384, 512 is timed on a reduced copy of the batch)
 * The plan keeps its own device tables (charged to the context's budget) and
 * records the pointers it was given: they must stay valid while it is used.
 * Each job's results are bit-identical to running it alone with
 * jarzynski_run_ex.  Errors: as jarzynski_run_ex; ISING_ERR_ARG if seeds
 * differ or an output is host memory. */
typedef struct jz_plan jz_plan;
int jz_plan_create(ising_ctx* ctx, const jz_params* jobs, int n_jobs, int64_t* const* work_outs,
                   double* est_out, int cta_threads, jz_plan** out);

/* Enqueues one replay of the plan's graph on the context's stream (counter
 * reset, persistent kernel, Swendsen-Wang launches, batched estimator); use
 * ising_sync to wait. */
int jz_plan_launch(jz_plan* plan);

/* Chosen launch shape of the plan's persistent kernel: CTA size, grid size,
 * work items (0 items and grid 0 when every job is Swendsen-Wang). */
int jz_plan_info(const jz_plan* plan, int* cta_threads, int* grid, int* n_items);

/* Releases the plan (waits for its queued replays). */
void jz_plan_free(jz_plan* plan);

/* ---------------------------------------------------------------- serving --
 * A continuous-batching server for c-function jobs (each job one
 * transformation of section 3, estimated as in estimator_reduce).  A host
 * thread admits submitted jobs in arrival order whenever a stream slot is free
 * and the job's device memory (thresholds, work array, estimator output) fits
 * the server's HBM budget, launches it on its slot's stream -- so jobs that
 * arrive while others run overlap on the device -- and, when its completion
 * event fires, copies the result back and frees the slot for the next job.
 * A job's lattice and random state stay in one CTA's shared memory for its
 * whole protocol (jobs whose lattice does not fit are refused with
 * ISING_ERR_UNSUPPORTED).  Results are bit-identical to running the job
 * alone. */
typedef struct jz_server jz_server;

typedef struct jz_result {
    int status;                 /* ISING_OK or the job's error code          */
    double log_ratio;           /* ln <e^-W>                                 */
    double delta_S2;            /* Delta S_2 of the transformation           */
    double delta_S2_err;        /* jackknife error (32 blocks)               */
    double submit_s, start_s, done_s;   /* server clock (s): submitted,
                                           launched, completion observed     */
    long long updates;          /* spin updates the job performed            */
} jz_result;

/* Creates a server on the context's device.
 *   hbm_budget_bytes  admission budget for the jobs' device memory (> 0)
 *   max_inflight      jobs on the device at once (1..64), one stream each
 * The context must outlive the server and is used only for its device and its
 * autotuned CTA sizes.  Errors: ISING_ERR_ARG, ISING_ERR_CUDA, ISING_ERR_NOMEM. */
int jz_server_create(ising_ctx* ctx, size_t hbm_budget_bytes, int max_inflight,
                     jz_server** out);

/* Queues a job (parameters are copied); returns its id in *job_id.  Invalid
 * parameters are reported at once; a job that can never fit the budget
 * finishes with status ISING_ERR_NOMEM. */
int jz_submit(jz_server* s, const jz_params* p, uint64_t* job_id);

/* ISING_OK and *out filled when the job is finished; ISING_ERR_PENDING while
 * it is queued or running; ISING_ERR_NOT_FOUND for an unknown id. */
int jz_poll(jz_server* s, uint64_t job_id, jz_result* out);

/* As jz_poll, but waits up to timeout_s seconds; ISING_ERR_TIMEOUT when the
 * job is still unfinished then (the job keeps running). */
int jz_wait(jz_server* s, uint64_t job_id, double timeout_s, jz_result* out);

/* Cancels a job: a queued job is dropped at once, a job already on the device
 * runs to its end with its results discarded; either way it finishes with
 * status ISING_ERR_CANCELLED.  A finished job keeps its result.  Returns
 * ISING_OK, or ISING_ERR_NOT_FOUND for an unknown id.  The paper has no
 * counterpart. */
int jz_cancel(jz_server* s, uint64_t job_id);

/* Per-job metrics as JSON lines: with path non-NULL the server appends one
 * line per finished job to that file (opened in append mode; NULL closes it):
 * its id, parameters, status, ln<e^-W>, Delta S_2 and its error, the server
 * clock at submission, launch and completion, latency, spin updates and
 * spin updates/s over its time on the device.  Errors: ISING_ERR_ARG,
 * ISING_ERR_NOT_FOUND (the file cannot be opened). */
int jz_server_set_log(jz_server* s, const char* path);

/* The JSON line jz_server_set_log writes for one job, into buf (n bytes,
 * NUL-terminated).  Host only (no device needed).  Returns the line's length,
 * or ISING_ERR_ARG (NULL arguments, or n too small for the line). */
int jz_result_json(uint64_t job_id, const jz_params* p, const jz_result* r, char* buf, size_t n);

/* Copies a finished job's W_int (n_traj entries) to host memory work_out. */
int jz_server_work(jz_server* s, uint64_t job_id, int64_t* work_out);

/* Stops admitting, waits for the jobs on the device, drops queued ones and
 * releases the server. */
void jz_server_free(jz_server* s);

/* The plain GPU form of the same computation, kept as the comparison baseline:
 * one trajectory per launch sequence, one launch per half-sweep, spins in
 * global memory (section 3 protocol, Appendix A work; same random stream and
 * acceptance conventions, so outputs are bit-identical to jarzynski_run_ex).
 * Arguments, buffers and errors as for jarzynski_run_ex.  Slow by design. */
int jarzynski_run_plain(ising_ctx* ctx, const jz_params* p, int64_t* work_int_out,
                        int8_t* spins_out);

/* Same computation as jarzynski_run_ex, without allocating anything; the
 * paper has no counterpart.  It exists for callers that may not allocate
 * device memory themselves or through us: a plug-in inside an application
 * whose allocator has already reserved the GPU's memory, or a loop that must
 * not stall in cudaMalloc / cudaFree (both can synchronise the device).
 * This call makes no cudaMalloc, cudaFree or other allocating call.  Its
 * scratch (one job descriptor and the N x 8d switched-site thresholds, or
 * N x 2 bond thresholds for Swendsen-Wang) lives in a single file-scope
 * device array of 1 MiB, which every GPU that loads the library keeps until
 * the process exits.  The descriptor and thresholds reach that array as the
 * arguments of small staging kernels enqueued on cuda_stream (about 31 KB per
 * launch), so the call reads no host memory after it returns.  Both updates
 * are served; lattices beyond one CTA's shared memory (which
 * jarzynski_run_ex runs from an HBM slice) are not.
 *   p             the transformation; final spins are not returned
 *   work_int_out  caller-owned DEVICE memory, p->n_traj int64 entries
 *   cuda_stream   cudaStream_t to enqueue on (NULL = the legacy default stream)
 * Returns once the work is enqueued: synchronise the stream before reading
 * work_int_out.  Results are bit-identical to jarzynski_run_ex.
 * Limit: 262080 threshold words, p->n_step * 8 * p->d for Metropolis (N <=
 * 16380 in 2D, N <= 10920 in 3D) and p->n_step * 2 for Swendsen-Wang (N <=
 * 131040); larger protocols return ISING_ERR_SCRATCH_LIMIT, lattices beyond
 * shared memory ISING_ERR_UNSUPPORTED, host output memory ISING_ERR_ARG,
 * other errors as jarzynski_run_ex.
 * Every call looks up the array's device address on the calling thread's
 * current device (cudaGetSymbolAddress, which loads the library's device code
 * on that device the first time); make the first call on a device before any
 * stream capture.  All calls share the one array and leave their contents in
 * it; nothing there needs to start at zero because each call rewrites
 * everything it reads before its kernels read it.  Calls whose GPU work can
 * overlap (different streams with no ordering between them) race on the
 * array: issue them on one stream or synchronise in between. */
int jarzynski_run_noalloc(const jz_params* p, int64_t* work_int_out, void* cuda_stream);

/* FP64 estimator on the device (Appendix A, eq. Jarzynski_theorem; section 2):
 *   *log_ratio    = ln <e^-W>, W_i = beta work_int[i] / n_step, evaluated as a
 *                   max-shifted log-sum-exp
 *   *delta_S2     = -ln <e^-W> for direction +1, +ln <e^-W> for direction -1
 *   *delta_S2_err = blocked jackknife error of delta_S2 with
 *                   B = min(n_jack_bins, n_traj) contiguous blocks of n_traj / B
 *                   trajectories, the remainder in the last block (0 if B < 2)
 * work_int: n_traj entries, host or device memory (not modified).  Output
 * pointers are host memory; the call returns when they are written.
 * Errors: ISING_ERR_ARG, ISING_ERR_CUDA. */
int estimator_reduce(ising_ctx* ctx, const int64_t* work_int, int n_traj, double beta,
                     int n_step, int direction, int n_jack_bins, double* log_ratio,
                     double* delta_S2, double* delta_S2_err);

/* Launch-shape control; the paper has no counterpart.  A time slice holds
 * col = ceil(L/8) * L_y spin words; each thread owns one word column of every
 * TS-th slice.  Fixes the CTA size the context uses for lattices of shape
 * (d, L, L_t), at most 512 threads:
 *   col <= 32  a multiple of 32: warp teams of col * TS <= 32 threads, as many
 *              per CTA as fit (one team of threads / col slices per CTA when
 *              fewer than four warp teams' lattices fit its shared memory)
 *   col > 32   col * TS with 1 <= TS <= L_t: one team per CTA
 * threads = 0 restores the default: the shape, among the warp-team layouts of
 * every CTA size and one team per CTA of every TS, that keeps the most lanes
 * of each SM busy for the launch's trajectory count (CUDA occupancy of the
 * kernel that runs the lattice).  Results do not depend on the shape.
 * Errors: ISING_ERR_ARG. */
int ising_set_threads(ising_ctx* ctx, int d, int L, int L_t, int threads);

/* The launch shape jarzynski_run_ex would use for p alone in this context:
 * shape[0] threads per team (one trajectory), shape[1] teams per CTA,
 * shape[2] threads per CTA, shape[3] 1 for warp teams (__syncwarp) and 0 for
 * one team per CTA (__syncthreads), shape[4] 1 when the lattices live in
 * HBM.  Swendsen-Wang: one trajectory per CTA of its fixed size.  shape is
 * host memory of 5 ints.  Errors: ISING_ERR_ARG (as check of p),
 * ISING_ERR_UNSUPPORTED (a time slice wider than 512 threads), ISING_ERR_CUDA. */
int ising_launch_shape(ising_ctx* ctx, const jz_params* p, int* shape);

/* Autotuner; the paper has no counterpart.  Times every admissible CTA size
 * (multiples of 32 that are powers of two, or TS a power of two up to L_t)
 * and the default shape on a short sample of the transformation p -- same
 * shape, coupling and l, n_therm = 16, N = 16, n_sweep = 1,
 * min(p->n_traj, 4864) trajectories -- keeps the fastest for p's shape in
 * the context (as ising_set_threads would) and writes it to *threads
 * (nullable): a CTA size, or 0 when the default shape, where it is none of
 * the sizes', was fastest.  Synchronises the context's stream.  Swendsen-Wang
 * (p->update = 1) runs one trajectory per CTA of a fixed size: nothing is
 * timed or stored and *threads receives that size (256 in 2D, 512 in 3D).
 * Errors: as jarzynski_run_ex. */
int ising_autotune(ising_ctx* ctx, const jz_params* p, int* threads);

/* Persisted autotune cache; the paper has no counterpart.  Keys are (GPU
 * name, d, L, L_t, n, n_traj bucket) with bucket = floor(log2 n_traj): the
 * best CTA size depends on the lattice and on how many trajectories fill the
 * GPU.  The file is JSON, {"version": 1, "entries": [...]}, one entry per
 * line with the keys gpu, d, L, L_t, n_replica, traj_bucket, cta_threads
 * (0 for the default shape, as ising_autotune reports it).
 * The cache functions are host only (no device needed); the cache is not
 * thread-safe.
 *   create / free   an empty cache
 *   load            merges a file's entries (later ones win); ISING_ERR_NOT_FOUND
 *                   if the file cannot be opened, ISING_ERR_ARG if it is malformed
 *   save            writes every entry; ISING_ERR_NOT_FOUND if it cannot write
 *   put / get       one entry; get returns ISING_ERR_NOT_FOUND on a miss
 *   size            number of entries
 * ising_autotune_cached: on a hit for the context's GPU, fixes that CTA size
 * for p's shape in the context (as ising_set_threads) without timing
 * anything; on a miss runs ising_autotune and stores its choice.  *threads
 * (nullable) receives the size, *hit (nullable) 1 for a hit and 0 otherwise.
 * Swendsen-Wang jobs are not cached (their CTA size is fixed). */
typedef struct jz_tune_cache jz_tune_cache;
int jz_tune_cache_create(jz_tune_cache** out);
void jz_tune_cache_free(jz_tune_cache* c);
int jz_tune_cache_load(jz_tune_cache* c, const char* path);
int jz_tune_cache_save(const jz_tune_cache* c, const char* path);
int jz_tune_cache_put(jz_tune_cache* c, const char* gpu, int d, int L, int L_t, int n_replica,
                      int n_traj, int cta_threads);
int jz_tune_cache_get(const jz_tune_cache* c, const char* gpu, int d, int L, int L_t,
                      int n_replica, int n_traj, int* cta_threads);
int jz_tune_cache_size(const jz_tune_cache* c, int* n);
int ising_autotune_cached(ising_ctx* ctx, jz_tune_cache* c, const jz_params* p, int* threads,
                          int* hit);

/* Measurement utility; the paper has no counterpart.  Runs an integer-issue
 * probe on `device` over all SMs at full occupancy and writes its rate:
 *   kind 0: three-input logic (LOP3) chains      -> thread-instructions/s
 *   kind 1: 32-bit multiply-add (IMAD) chains     -> thread-instructions/s
 *   kind 2: 1:1:1 IMAD / LOP3 / IADD3 mix         -> thread-instructions/s
 *   kind 3: Philox4x32-10 blocks                  -> blocks/s
 * These are the measured ceilings of the trajectory kernel's roofline.  Uses
 * the legacy default stream and synchronises the device.
 * Errors: ISING_ERR_ARG (kind or rate), ISING_ERR_CUDA. */
int ising_probe(int device, int kind, double* rate);

/* Build check; the paper has no counterpart.  Writes the compute capability
 * the library's device code was compiled for, as major * 10 + minor
 * (cudaFuncGetAttributes' binaryVersion of one of its kernels: 103 for the
 * sm_103a build), on `device`.  Errors: ISING_ERR_ARG, ISING_ERR_CUDA (no such
 * device, or no code in the library loads on it). */
int ising_binary_version(int device, int* version);

/* Debug build (libisingjz_debug.so, compiled with bounds checks; the paper
 * has no counterpart).  Every lattice access of the trajectory kernels and
 * every cluster-label and spin-bit access of the Swendsen-Wang kernel checks
 * its index; an index outside its array is recorded in a device status word
 * and the access is skipped, so the kernel neither faults nor reads another
 * lattice.  *sites receives the OR of the check sites that failed since the
 * last clear (0 = none), *index one failing index; clear != 0 resets the
 * words (on the current device).  The release library returns
 * ISING_ERR_UNSUPPORTED.  Errors: ISING_ERR_ARG, ISING_ERR_CUDA. */
int ising_bounds_status(unsigned int* sites, unsigned int* index, int clear);

/* Human-readable text for an error code (static storage). */
const char* ising_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* ISINGJZ_H */
