/*
 * wave.h -- C ABI of libwave.so, a time-tiled 3D acoustic wave stencil for
 * NVIDIA GB300 (sm_103a).
 *
 * The library advances the damped acoustic wave equation
 *     m u_tt + d u_t = Lap u + q
 * with second-order leapfrog in time and a centred space stencil of order SO
 * (4, 8 or 16), i.e. the update printed in McCormick 2017, "Applying the
 * Polyhedral Model to Tile Loops in Devito", Fig. acoustic_devito:
 *     u[t+1] = ((dt d - 2m) u[t-1] + 4m u[t] + 2dt^2 (L_h u[t] + q)) / (dt d + 2m).
 * It runs the update either one step per pass over HBM (the plain method) or
 * T steps per pass (time tiling, Chapter "Time-Tiling": the time loop moved
 * inside the spatial tile loops, spatial loops skewed by SO/2 per step).
 *
 * Units: spacing in metres, dt in milliseconds, velocity in km/s, so
 * m = 1/v^2 is in (ms/m)^2 and v dt / h is dimensionless.
 *
 * Layout of every 3D array crossing this ABI: float32, [nx][ny][nz]
 * row-major, z fastest (the paper's u[time][x][y][z] without the time index,
 * Fig. acoustic_devito).  Grid index (i, j, k) sits at (i hx, j hy, k hz)
 * metres.  Points outside the grid are zero (a zero Dirichlet ghost layer of
 * width SO/2 that is never written, Section "Simulation").
 *
 * Pointers: "device" pointers must be CUDA device (or managed) memory on the
 * plan's device; "host" pointers are ordinary host memory.  The caller owns
 * every pointer it passes; the plan copies what it keeps (the model, tap
 * lists) and owns its wavefield buffers.  Calls are ordered on the plan's
 * stream (wave_options.stream; 0 = legacy default stream).
 *
 * Errors: every call returns a wave_status; nothing throws across the ABI.
 * On failure, wave_last_error() returns a message for the calling thread.
 * A failed call leaves the plan usable unless it returns WAVE_ERR_CUDA.
 */
#ifndef WAVE_H
#define WAVE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WAVE_OK = 0,
    WAVE_ERR_ARG = 1,     /* invalid argument (null, size, SO, range)            */
    WAVE_ERR_CFL = 2,     /* dt above the leapfrog stability limit               */
    WAVE_ERR_OOM = 3,     /* device or host allocation failed                    */
    WAVE_ERR_CUDA = 4,    /* a CUDA call failed; the plan should be destroyed    */
    WAVE_ERR_TIMEOUT = 5, /* a bounded device-side wait gave up (see wave.h top) */
    WAVE_ERR_STATE = 6    /* call out of order (e.g. no sources set)             */
} wave_status;

typedef struct wave_plan_s* wave_plan_t;

/* Tiling of one pass (a "tile schedule"):
 *   T      : time steps per pass over HBM (1 = the plain one-step method);
 *   by     : output tile extent along y (points);
 *   bz     : output tile extent along z (points, multiple of 4);
 *   xc     : extent along x of the slab one thread block streams through;
 *   unroll : the kernel variant: where the per-column queue of planes along
 *            x lives and how the pass is organised.  0 = registers, moved in
 *            a compact loop; 1 = registers, loop unrolled over the queue
 *            length; 2 = tensor memory (a ring per warp, read back with
 *            tcgen05.ld; no register queue); 4 = skewed wavefront tiling in y
 *            (T = 2, tensor memory); 5 and 6 = warp-specialised pass (a
 *            producer warp issues the TMA copies, no block-wide barrier per
 *            plane, tensor memory), 1 (5) or 2 (6) rows per thread; 7 =
 *            the warp-specialised pass with 2 rows per thread whose x
 *            queues are tensor-memory shift registers (half the tensor
 *            memory of 6, so taller tiles and more warps).
 *            Every variant computes bit-identical fields.
 * (T, by, bz, unroll) must name a compiled kernel variant (wave_tiling_check).
 * Fields T, by, bz, xc of 0 = let the library choose. */
typedef struct {
    int T, by, bz, xc, unroll;
} wave_tiling;

typedef struct {
    int sponge_width;  /* absorbing layer width in cells (default 10, 0 = none)  */
    int sponge_faces;  /* bit f set = face f absorbs, faces x-,x+,y-,y+,z-,z+;    */
                       /* default 0x2F: all but z- (z = 0 is the free surface)   */
    double vmax;       /* km/s, sets the sponge strength (default: from m)       */
    void* stream;      /* cudaStream_t for every call on the plan (default 0)    */
    wave_tiling tiling;/* forced tiling of the forward passes (0s = choose)      */
    int autotune;      /* 1 = time candidate tilings on the GPU at plan creation,*/
                       /* 0 = built-in default (the default)                     */
    int device;        /* CUDA device ordinal (default: current device)          */
} wave_options;

/* Fill *opt with the defaults listed above.  Returns WAVE_ERR_ARG on NULL. */
wave_status wave_options_default(wave_options* opt);

/* Centred second-derivative FD weights of accuracy order `so` (2..16, even) on
 * unit spacing, a[0] (centre) .. a[so/2], as exact rationals rounded to double:
 *   a_k = 2 (-1)^(k+1) (r!)^2 / (k^2 (r-k)! (r+k)!),  a_0 = -2 sum_k a_k.
 * Fig. acoustic_devito prints these for SO 8 times 2dt^2/h^2.
 * `a` is host memory of so/2 + 1 doubles.  Host only, no GPU needed. */
wave_status wave_fd_weights(int so, double* a);

/* Largest stable dt (ms) of the leapfrog update for velocity vmax (km/s):
 * 2 / (vmax sqrt(rho sum_a 1/h_a^2)), rho = |a_0| + 2 sum_k |a_k|.
 * spacing: host [3] metres.  Host only. */
wave_status wave_cfl_limit(int so, const double spacing[3], double vmax, double* dt_max);

/* Create a plan: validates the problem, builds the FD coefficients, checks
 * the CFL limit (WAVE_ERR_CFL), allocates the wavefield buffers and converts
 * the model.  The arguments are the paper's statement of the problem: the
 * grid, spacing, space order, dt and squared slowness m of the acoustic
 * example (Section "Acoustic wave equation", Fig. acoustic_devito; grid sizes
 * as in Section "Simulation Grid Size"), plus the absorbing `damp` layer of
 * the same figure (wave_options).  The plan owns its wavefields; the caller
 * keeps m.  grid: host [3] = nx, ny, nz (each >= so + 1); spacing: host [3]
 * metres; so in {4, 8, 16}; dt > 0 in ms; nt >= 0 time steps;
 * m: device [nx][ny][nz] squared slowness (copied, not kept); opt may be NULL.
 * The plan is bound to the device current at the call (or opt->device). */
wave_status wave_plan_create(wave_plan_t* out, const int grid[3], const double spacing[3], int so,
                             double dt, int nt, const float* m, const wave_options* opt);

/* Replace the model (device [nx][ny][nz], copied).  Recomputes the per-point
 * coefficients; sources and receivers stay. */
wave_status wave_set_model(wave_plan_t plan, const float* m);

/* Point sources: xyz host [nsrc][3] metres, injected through trilinear
 * weights as a term of the discrete equation (L_h u -> L_h u + sum w q);
 * wavelet device [nt][nsrc] (copied).  Update n injects row n.  nsrc = 0
 * clears the sources.  Every coordinate must be finite and inside the grid,
 * 0 <= xyz[a] <= (n_a - 1) h_a (WAVE_ERR_ARG otherwise).  The paper removes
 * its source before tiling (Section "Functional Correctness"); here it is
 * fused into every pass. */
wave_status wave_set_sources(wave_plan_t plan, int nsrc, const double* xyz, const float* wavelet);

/* Receivers: xyz host [nrec][3] metres; trace n of receiver j is the
 * trilinear interpolation of u^{n+1} (the field produced by update n).
 * nrec = 0 clears them.  Positions follow the rule of wave_set_sources (the
 * paper samples its receivers in the loop after the stencil, Section
 * "Testing environment").  A dense receiver surface (at least 4096 receivers
 * whose taps all lie in one or two adjacent z quads, e.g. a grid of
 * receivers at one depth) is recorded, when the plan's passes are one-step,
 * by a gather after every pass from the new field, with the same taps,
 * weights and summation order as the per-tap path (the traces are
 * identical). */
wave_status wave_set_receivers(wave_plan_t plan, int nrec, const double* xyz);

/* Force the tiling of the forward passes (see wave_tiling).  T = 1 selects a
 * one-step pass (one time step per pass over HBM: the plain, untiled method)
 * in the variant that `unroll` names: 0, 1 or 2 = the block-barrier pass
 * (wave_pass.cuh), 5, 6 or 7 = the warp-specialised pass (wave_lean.cuh).  All
 * one-step variants compute the same bits; the benchmark's untiled baseline is
 * the fastest of them.  Fields of 0 are chosen by the library.  Rejects a
 * schedule the tile-legality scheduler does not accept (WAVE_ERR_ARG).  A
 * one-step tiling also becomes the tiling of the plan's one-step sweeps (the
 * recompute and adjoint sweeps of wave_gradient, steps left over when nt is
 * not a multiple of T). */
wave_status wave_set_tiling(wave_plan_t plan, const wave_tiling* tiling);

/* wave_autotune with its result cached by key: the device (name and SM
 * count), the grid, the space order, T_only and the set of compiled kernel
 * variants.  A key seen before in this process applies the stored tilings
 * (the overall pick and the fastest one-step candidate, which runs the
 * one-step sweeps) without timing anything; with the environment variable
 * WAVE_AUTOTUNE_CACHE=<path> results are also appended to that text file
 * ("key T by bz xc unroll T1 by1 bz1 xc1 unroll1" per line, the last line of
 * a key wins) and looked up there, so they persist across processes.  *from_cache (may be NULL) is
 * set to 1 when the tiling came from the cache.  Errors as wave_autotune;
 * an unreadable or unwritable file only disables the file. */
wave_status wave_autotune_cached(wave_plan_t plan, int passes, int T_only, int* from_cache);

/* The tiling the forward passes use now (after defaults / autotuning). */
wave_status wave_get_tiling(wave_plan_t plan, wave_tiling* tiling);

/* The one-step tiling of the plan's one-step sweeps (the recompute and
 * adjoint sweeps of wave_gradient, steps left over when nt is not a multiple
 * of T): the built-in default, a one-step tiling given to wave_set_tiling, or
 * the fastest one-step candidate of the last autotuning (timed or cached). */
wave_status wave_get_sweep_tiling(wave_plan_t plan, wave_tiling* tiling);

/* Time candidate tilings on the GPU for this plan (T = 1..Tmax, several tile
 * shapes and slab lengths) with `passes` timed passes each, and keep the
 * fastest in point-steps per second (T = 1 may win: the paper's remark that
 * time tiling is only worthwhile when the loop is memory-bound).  T_only > 0
 * restricts the sweep to that T.  The fastest one-step candidate, whether
 * or not it wins, becomes the tiling of the plan's one-step sweeps (see
 * wave_set_tiling).  The plan's wavefields are scratch during the sweep.
 * cand / ms_per_step: host arrays of up to `cap` entries (may be
 * NULL) receiving every timed candidate and its milliseconds per time step;
 * *ncand (may be NULL) receives how many were timed. */
wave_status wave_autotune(wave_plan_t plan, int passes, int T_only, wave_tiling* cand, double* ms_per_step,
                          int cap, int* ncand);

/* Forward modelling of nt steps from u^{-1}, u^0: the update of Fig.
 * acoustic_devito applied nt times (Section "Acoustic wave equation"), run
 * T steps per pass over HBM with the plan's tiling (Chapter "Time-tiling for
 * Devito stencils", Section "Time-Tiling"); sources and receivers are the
 * loops that Section "Testing environment" lists around the stencil.
 * u_init: device [2][nx][ny][nz] = (u^{-1}, u^0), or NULL for zero fields.
 * rec_out: device [nt][nrec] traces, may be NULL when nrec = 0.
 * u_final: device [2][nx][ny][nz] receiving (u^{nt-1}, u^{nt}), may be NULL.
 * Synchronises the plan's stream at the end to report device-side timeouts
 * (WAVE_ERR_TIMEOUT). */
wave_status wave_forward(wave_plan_t plan, const float* u_init, float* rec_out, float* u_final);

/* The same as wave_forward with every array in host memory (copies inside). */
wave_status wave_forward_host(wave_plan_t plan, const float* m_host, const float* wavelet_host,
                              float* rec_host);

/* Adjoint modelling: the transpose of the linear map wavelet -> traces of
 * wave_forward (zero initial fields).  The paper has no adjoint; the map is
 * the discrete update of Fig. acoustic_devito, whose L_h is symmetric and
 * whose damping is diagonal, so its transpose is the same update run on the
 * time-reversed residual with the source and receiver loops of Section
 * "Testing environment" swapping roles (same kernels, same tiling).
 * rec_resid: device [nt][nrec] is injected at the receivers backwards in
 * time.  src_out: device [nt][nsrc] receives the adjoint field sampled at the
 * sources, or NULL.  v_final: device [2][nx][ny][nz] receives the last two
 * levels of the adjoint field in the layout of wave_forward's u_final (the
 * level before the last, then the last, which is the adjoint field at forward
 * time 0), or NULL.  Both may be NULL.  Synchronises the plan's stream. */
wave_status wave_adjoint(wave_plan_t plan, const float* rec_resid, float* src_out, float* v_final);

/* Misfit J = 1/2 sum (rec - d_obs)^2 of the plan's sources and receivers and
 * its gradient with respect to m (adjoint state).  The paper computes no
 * gradient; this is the exact gradient of the discrete update of Fig.
 * acoustic_devito, and its checkpoints trade memory for recomputation as the
 * buffered time dimension of Section "Time Dimension Buffering" trades it
 * for a bounded time tile:
 *   dJ/dm = - sum_n mu^{n+1} (u^{n+1} - 2u^n + u^{n-1}) / dt^2,
 * mu the adjoint field driven by rec - d_obs.  d_obs: device [nt][nrec];
 * grad_m: device [nx][ny][nz]; misfit: host double (may be NULL).
 * checkpoint_every = K > 0 stores (u^{n-1}, u^n) every K steps and recomputes
 * each K-step segment forward before its adjoint sweep (memory ~ (nt/K + K)
 * fields; ~ (nt/K + 2K) when the device has room for a second segment
 * buffer, and then the recompute of one segment runs on a second stream of
 * the plan while the adjoint steps through the next).  K = 0 (or K >= nt)
 * keeps every increment of one forward sweep when it fits in device memory,
 * with no recomputation.  The imaging condition is fused into the adjoint
 * passes.  The result does not depend on K.  The environment variable
 * WAVE_GRADIENT_SERIAL=1 keeps one segment buffer and one stream (the same
 * bits, less memory, slower). */
wave_status wave_gradient(wave_plan_t plan, const float* d_obs, float* grad_m, double* misfit,
                          int checkpoint_every);

/* Measurement hook.  With enable = 1 every pass kernel the plan launches is
 * bracketed by a pair of CUDA events recorded on the plan's stream, so the
 * caller can read the kernel's own device time without a profiler.
 * Counting of launched kernels is always on. */
wave_status wave_profile_enable(wave_plan_t plan, int enable);

/* Read (and with reset = 1 clear) the counters since the last reset:
 * pass_launches / pass_ms: pass kernels timed by the events above and their
 * summed duration (synchronises the plan's stream); point_steps: point
 * updates those passes performed (grid points x steps); launches: every
 * kernel of this library launched on the plan.  Any output may be NULL. */
wave_status wave_profile_read(wave_plan_t plan, int reset, long long* pass_launches, double* pass_ms,
                              double* point_steps, long long* launches);

/* Receiver sampling that allocates nothing, for callers that cannot allocate
 * device memory when they need a trace (a fixed memory pool that must not
 * grow, an allocator that owns the whole device, a real-time loop in which
 * cudaMalloc may stall).  The paper has no counterpart: this is an interface
 * of this library only.
 *
 * rec[j] = trilinear interpolation of u at xyz[j], the same taps, weights and
 * summation order as the traces of wave_forward, so sampling the field
 * wave_forward returns reproduces its last trace row.
 * grid, spacing: host [3] (cells, metres); u: device [nx][ny][nz] float32;
 * xyz: host [nrec][3] metres, each coordinate finite and inside
 * [0, (n_a - 1) h_a] (WAVE_ERR_ARG otherwise, as in wave_set_receivers);
 * rec: device [nrec] float32, written on `stream` (a cudaStream_t, NULL =
 * legacy default stream); nothing is synchronised.  The positions are
 * copied to the device on `stream`: from pageable memory the copy is done
 * before the call returns, but from pinned memory it runs later, so a pinned
 * xyz must stay valid and unchanged until the work queued on `stream` has
 * run.  At most 65536 receivers per call (WAVE_ERR_ARG beyond that).
 *
 * The tap slots live in one static device array (5.75 MiB, held by every GPU
 * that loads the library until the process exits).  Every call shares it and
 * writes every slot it reads, so no state carries over between calls, but
 * calls that overlap on the GPU (other streams, other host threads) race.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  No cudaMalloc, cudaFree or allocating library
 * routine is called. */
wave_status wave_sample_noalloc(const int grid[3], const double spacing[3], const float* u, int nrec,
                                const double* xyz, float* rec, void* stream);

/* ---- batched shots ---------------------------------------------------------
 * Many independent shots (plans with their own grid, SO, tiling, sources and
 * receivers, as the autotuner chose per shot: the per-problem tiling of
 * Section "Future Work", "Automating time-tiling in Devito") advanced
 * together.  The plans must live on one device and stay alive as long as the
 * batch. */
typedef struct wave_batch_s* wave_batch_t;

wave_status wave_batch_create(wave_batch_t* out, int nplans, const wave_plan_t* plans);

/* Autotune every plan of the batch (wave_autotune with `passes` timed passes
 * per candidate) over the tilings the persistent batched kernel runs (SO 4
 * and 8: 512-thread tiles with tensor-memory queues, T = 1, 2 or 3; x slabs
 * of one length for the whole batch, or the whole grid: 256 planes while a
 * pass level of all the shots makes at least two work items per SM, else
 * 128, 64 or 32); plans of SO 16 are tuned over every candidate. */
wave_status wave_batch_autotune(wave_batch_t batch, int passes);

/* Forward modelling of every shot from zero fields, the same results as
 * wave_forward per plan (bit-identical).  rec_out: host array of nplans
 * device pointers ([nt_i][nrec_i] each; may be NULL for shots without
 * receivers).  When every plan's tiling (and its one-step remainder passes)
 * has a shape in the persistent batched kernel, all shots run in one
 * persistent launch: a device work queue lists every (shot, pass, tile) item,
 * pass level by pass level across the shots; each thread block takes the next
 * item, waits (bounded, 2 s) until every tile of the shot's previous pass is
 * done, runs the tile and publishes it.  Otherwise every shot's own pass
 * launches run on a stream of its own.  Either way the work is captured into
 * one CUDA graph on the first call, and again when the rec_out pointers
 * change or a plan's buffers or tiling changed since.  The persistent kernel
 * reads the pass arguments from one constant-memory array per device, which
 * the graph writes before the launch: batched forwards of different batches
 * must not overlap on one device (each call synchronises `stream` before it
 * returns).  Synchronises `stream` (cudaStream_t) and reports device-side
 * timeouts (WAVE_ERR_TIMEOUT). */
wave_status wave_batch_forward(wave_batch_t batch, float* const* rec_out, void* stream);

/* How the last captured forward runs: *persistent = 1 for the persistent
 * kernel (then *items work items on *blocks thread blocks), 0 for per-shot
 * launches.  Any output may be NULL. */
wave_status wave_batch_get_mode(wave_batch_t batch, int* persistent, int* items, int* blocks);

/* Self-test of the persistent kernel's failure detection: runs the batch's
 * work queue once with shot 0's completion counter withheld (started far
 * below what its first item waits for), with dependency waits bounded by
 * limit_ms (0 < limit_ms <= 10000).  The waiting blocks give up, set the
 * queue's abort word and return; the others stop at their next item.
 * Returns WAVE_ERR_TIMEOUT when that happened (the expected outcome: the
 * device stays usable and the next wave_batch_forward recaptures and runs
 * normally), WAVE_OK if no wait gave up (a defect), WAVE_ERR_STATE if the
 * batch has no persistent work queue.  The plans' wavefields are scratch. */
wave_status wave_batch_selftest_withhold(wave_batch_t batch, double limit_ms);

/* FWI gradient of every shot (see wave_gradient), all shots' work --
 * checkpointed forward, residual, adjoint sweep, imaging -- captured in one
 * CUDA graph (one stream per shot) and replayed with a single launch; the
 * same results as wave_gradient per plan (bit-identical).
 *   d_obs          : host array of nplans device pointers, [nt_i][nrec_i];
 *   grad_m         : host array of nplans device pointers, [nx][ny][nz] each
 *                    (written);
 *   misfit         : host array of nplans doubles (written), or NULL;
 *   checkpoint_every: as in wave_gradient, for every shot.
 * Every buffer a shot needs is allocated before the capture; the graph is
 * captured again when the pointers, the segment lengths or a plan's buffers
 * change.  Synchronises `stream`.  Errors: WAVE_ERR_ARG (NULL entries),
 * WAVE_ERR_STATE (a shot without sources or receivers), WAVE_ERR_OOM,
 * WAVE_ERR_TIMEOUT, WAVE_ERR_CUDA. */
wave_status wave_batch_gradient(wave_batch_t batch, const float* const* d_obs, float* const* grad_m, double* misfit,
                                int checkpoint_every, void* stream);

wave_status wave_batch_destroy(wave_batch_t batch);

/* Destroy the plan and free its device memory.  NULL is accepted. */
wave_status wave_plan_destroy(wave_plan_t plan);

/* Message of the last failed call on this thread ("" if none). */
const char* wave_last_error(void);

/* Self-test of failure detection: launches one thread block that waits,
 * with the pass kernel's bounded-wait helper and a limit of limit_ms (0 <
 * limit_ms <= 10000), on an mbarrier phase that never completes.  Returns
 * WAVE_ERR_TIMEOUT when the wait gave up and the block returned (the
 * expected outcome: the device stays usable), WAVE_OK if the wait was
 * satisfied (a defect).  Runs on the current device; synchronises it. */
wave_status wave_selftest_timeout(double limit_ms);

/* ---- tile-legality scheduler (host only, no GPU) --------------------------
 * Chapter "Time-Tiling" / Section "Skewing Dependencies": a stencil update
 * reading u[t] at offsets +-r along an axis has the dependence distances
 * (1, +-r) on that axis; tiling through time is legal once every skewed
 * distance is lexicographically non-negative, i.e. with skew factor r per
 * skewed axis.  These calls expose the scheduler for tests and tools. */

/* Skew factor of space order so (= so/2). */
int wave_skew_factor(int so);

/* Check a tiling for a grid and SO: returns WAVE_OK if the overlapped,
 * skewed pass schedule is legal and fits the kernel's limits, else
 * WAVE_ERR_ARG with the reason in wave_last_error(). */
wave_status wave_tiling_check(const int grid[3], int so, const wave_tiling* tiling);

/* Brute-force legality of the GPU pass schedule on a tiny grid: enumerates
 * every (point, time level) every thread block computes and checks that each
 * value it reads is either a pass input or a value the same block computed
 * earlier from valid inputs, and that every output point is written exactly
 * once with a valid value.  Returns WAVE_OK or WAVE_ERR_ARG with the first
 * violation in wave_last_error(). */
wave_status wave_schedule_verify(const int grid[3], int so, const wave_tiling* tiling);

/* wave_schedule_verify with the kernel's two skew parameters overridden:
 * `lag` planes between consecutive steps along x (the kernel uses r) and
 * `halo_per_step` overlapped points per remaining step in y and z (the kernel
 * uses r).  Smaller values must be rejected; exposed for tests. */
wave_status wave_schedule_verify_custom(const int grid[3], int so, const wave_tiling* tiling, int lag,
                                        int halo_per_step);

/* Brute-force legality of the skewed wavefront variant (unroll = 4) on a
 * tiny grid, with its two inter-tile parameters overridden: the rows of
 * level n+1 that tile j takes from tile j-1 below it (`exchange_rows`, the
 * kernel exchanges 2r) and how far ahead of tile j's iteration the published
 * progress of tile j-1 must be (`wait_lead`, the kernel's wait gives 1).
 * wave_schedule_verify checks the variant with the kernel's values; smaller
 * ones must be rejected.  Returns WAVE_OK or WAVE_ERR_ARG with the first
 * violation in wave_last_error(). */
wave_status wave_schedule_verify_skew(const int grid[3], int so, const wave_tiling* tiling, int exchange_rows,
                                      int wait_lead);

/* Brute-force check of the paper's skewed time-tiled loop order in 1D+t
 * (Fig. tiled_skew_snippet / Fig. tiled_256 reduced to one space axis):
 * tiles of tt time steps x ts skewed points, skew factor `skew`, stencil
 * radius r, n points, nt steps.  Returns 1 if every point-step runs after
 * all the point-steps it reads, 0 if a dependence is violated. */
int wave_skewed_order_legal(int n, int nt, int r, int skew, int tt, int ts);

#ifdef __cplusplus
}
#endif

#endif /* WAVE_H */
