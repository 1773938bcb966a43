/*
 * fitsne_gb300.h - C ABI of the GB300 (sm_103a) FIt-SNE gradient library.
 *
 * The library computes, on one GPU, the per-iteration t-SNE gradient of
 * Linderman et al., "Efficient Algorithms for t-distributed Stochastic
 * Neighborhood Embedding" (arXiv 1712.09005):
 *
 *   dC/dy_i = 4 (alpha * A_i + F_rep,i)                      (Sec. 1.1, Sec. 1.2)
 *   A_i     = sum_j p_ij (y_i - y_j) / (1 + |y_i - y_j|^2)    (Sec. 3, sparse P)
 *   F_rep,i = sum_{l != i} (y_l - y_i) / (1 + |y_l - y_i|^2)^2 / Z   (Eq. frep)
 *
 * with F_rep and Z evaluated by the interpolation / FFT scheme of Sec. 2
 * (Algorithm 1 and its 2-D tensor version, Sec. 2.4): the points' charges are
 * spread onto p equispaced Lagrange nodes per interval of an N_int (x N_int)
 * box grid (Step 1), convolved with K1 = (1+r^2)^-1 and K2 = K1^2 through a
 * zero-padded FFT of the Toeplitz matrix (Step 2), and interpolated back
 * (Step 3); the Appendix assembles F_rep = (h_{m+1} - y(m) h_{s+2}) / Z and
 * Z = sum_i h_1(y_i) - N (the grid cannot exclude the self term, so N is
 * subtracted).
 *
 * Conventions for every entry point:
 *   - Y, dY, uY, gains are fp32, N x s, row-major (for s = 2 the pairs
 *     (y_i(1), y_i(2)) are adjacent). P is CSR with int32 row_ptr[N+1],
 *     int32 col[nnz], fp32 val[nnz]; row i holds p_ij for j != i. P should be
 *     symmetric and sum to 1 (Sec. 1.1); the library does not renormalise it.
 *   - Unless stated otherwise, pointers are DEVICE pointers owned by the
 *     caller; the library never frees them and never keeps them past the call.
 *     The plan owns all scratch memory.
 *   - Work is enqueued on the plan's stream; calls return once it is
 *     enqueued, so results are ready after the stream is synchronised.
 *   - Every function returns 0 (TSNE_OK) or a negative TSNE_ERR_* code; no
 *     exception crosses the ABI. tsne_last_error_string() describes the last
 *     failure of the calling thread. Errors detected on the device (a
 *     non-finite coordinate) are latched in the plan and reported by
 *     tsne_plan_status(), which synchronises the stream.
 *   - A plan is not thread-safe; use one plan per host thread or serialise.
 */
#ifndef FITSNE_GB300_H
#define FITSNE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TSNE_OK 0
#define TSNE_ERR_INVALID_ARG (-1) /* bad size, pointer, option or CSR structure */
#define TSNE_ERR_OOM (-2)         /* device allocation failed */
#define TSNE_ERR_NONFINITE (-3)   /* NaN or Inf met in Y (latched on the device) */
#define TSNE_ERR_TIMEOUT (-4)     /* a bounded device wait gave up */
#define TSNE_ERR_CUDA (-5)        /* a CUDA runtime call failed */
#define TSNE_ERR_CAPACITY (-6)    /* request exceeds what the plan was built for */

typedef struct tsne_plan tsne_plan;

/* Sparse affinities P (Sec. 1.1, Eq. p_ij), device CSR. */
typedef struct {
    const int32_t* row_ptr; /* [N+1], row_ptr[0] = 0, non-decreasing */
    const int32_t* col;     /* [nnz], 0 <= col < N, col != row */
    const float* val;       /* [nnz], p_ij >= 0 */
    int64_t nnz;            /* = row_ptr[N] */
} tsne_csr;

/* Plan options; zero-initialised fields take the defaults in brackets. */
typedef struct {
    int32_t n_min;     /* floor of the interval rule max(n_min, ceil(width)) [50] (Sec. 2.5) */
    int32_t n_int_max; /* cap of the rule and size of the grids [min(1000, 3000 / p) if s = 1,
                          min(400, 1200 / p) if s = 2]; p * n_int_max may not exceed 3000
                          (s = 1) or 1200 (s = 2) */
    void* stream;      /* cudaStream_t for all work; NULL = the legacy default stream */
    int32_t relabel_first; /* iteration of a run's first locality relabelling [100]; < 0: never */
    int32_t relabel_every; /* iterations between later relabellings [300] */
    int32_t force_mode;    /* work schedule of the force kernel, TSNE_FORCE_* [TSNE_FORCE_AUTO] */
    int32_t order_rounds;  /* averaging rounds of the graph order a run starts in [8], 1..64;
                              < 0: runs start in the caller's labels (see tsne_run_iters) */
} tsne_plan_opts;

/* Work schedules of the force kernel (same arithmetic, bitwise equal results):
 * GRID    a grid-stride loop over chunks of 256 rows;
 * REGION  the 32-row blocks are cut into one contiguous region per SM; an
 *         SM's warps take their own region's blocks first (so, in a
 *         relabelled run, they gather neighbours from one working set that
 *         stays in the SM's L1), then help the regions still in progress;
 * AUTO    REGION (a plan's steps and gradients; batches always use REGION
 *         over all their jobs' rows). */
#define TSNE_FORCE_AUTO 0
#define TSNE_FORCE_GRID 1
#define TSNE_FORCE_REGION 2

/* Gradient-descent schedule (Sec. 1.2 early exaggeration, Sec. 4 late
 * exaggeration). The momentum/gain update is not specified by the paper; the
 * usual t-SNE rule is used:
 *   gain <- gain + gain_inc if sign(dY) != sign(uY) else gain * gain_dec,
 *   gain <- max(gain, min_gain); uY <- mu uY - lr gain dY; Y <- Y + uY,
 * mu = momentum_early before mom_switch_iter, momentum_late from it on.
 * alpha = early_alpha for iter < early_iters, late_alpha for
 * iter >= n_iter - late_iters, 1 otherwise. */
typedef struct {
    int32_t n_iter;          /* total iterations of the run [1000] */
    int32_t early_iters;     /* [250] */
    int32_t late_iters;      /* [0] */
    int32_t mom_switch_iter; /* [250] */
    float early_alpha;       /* [12] */
    float late_alpha;        /* [1] */
    float lr;                /* [200] */
    float momentum_early;    /* [0.5] */
    float momentum_late;     /* [0.8] */
    float min_gain;          /* [0.01] */
    float gain_inc;          /* [0.2] */
    float gain_dec;          /* [0.8] */
} tsne_step_params;

/* Box and grid of the most recent gradient evaluation (read back by
 * tsne_plan_info, which synchronises the stream). */
typedef struct {
    float y_min;     /* lower corner of the box in every dimension (Sec. 2.2, 2.4) */
    float width;     /* box side; 1 when all coordinates are equal */
    float b;         /* interval width, width / n_int (FP32) */
    float delta;     /* node spacing b / p (FP32) */
    int32_t n_int;   /* intervals per dimension */
    int32_t n;       /* nodes per dimension, p * n_int */
    int32_t fft_len; /* padded FFT length per dimension (>= 2n) */
    int32_t n_chunks;/* spread work items of the last iteration */
    double Z;        /* normalisation of the last evaluation (FP64) */
    int32_t status;  /* latched device error (TSNE_OK or TSNE_ERR_NONFINITE) */
    int32_t pad;
} tsne_plan_info_t;

/* Library version string. */
const char* tsne_version(void);

/* Description of the last error returned on this host thread ("" if none). */
const char* tsne_last_error_string(void);

/* Fills *out with the defaults listed in tsne_step_params. */
void tsne_step_params_default(tsne_step_params* out);

/* alpha(iter) of the schedule (host helper, same rule as the device). */
float tsne_alpha_at(const tsne_step_params* sp, int32_t iter);

/*
 * Creates a plan for N points in s dimensions (s = 1 or 2) with p nodes per
 * interval (2 <= p <= 5; the paper recommends p = 3, Sec. 2.3).
 * n_intervals > 0 fixes N_int per dimension (1 <= n_intervals <= n_int_max);
 * 0 selects the automatic rule max(n_min, ceil(y_max - y_min)) each
 * iteration (Sec. 2.5), evaluated on the device from the FP32 bounding box.
 * Allocates all scratch for the largest grid the plan allows. N >= 2.
 * Errors: INVALID_ARG, OOM, CUDA. On success *out owns the plan.
 */
int tsne_plan_create(int64_t N, int32_t s, int32_t n_intervals, int32_t p,
                     const tsne_plan_opts* opts, tsne_plan** out);

/* Frees the plan and its scratch (synchronises its stream first). NULL is a no-op. */
int tsne_plan_destroy(tsne_plan* plan);

/*
 * Test hook: replaces the bounding box of every later evaluation by
 * [y_min, y_min + width]^s with n_int intervals (width > 0,
 * 1 <= n_int <= n_int_max); points outside are assigned to the nearest
 * edge interval. width <= 0 restores the automatic box.
 */
int tsne_plan_set_box(tsne_plan* plan, float y_min, float width, int32_t n_int);

/*
 * The interpolated gradient (Sec. 2 + Appendix, attraction of Sec. 3):
 * dY[i] = 4 (alpha A_i + F_rep,i) for all i, and Z (FP64) written to the
 * DEVICE address Z_out if it is not NULL. Y: [N x s] device, read only.
 * dY: [N x s] device, written. Y and dY must not overlap.
 */
int tsne_gradient(tsne_plan* plan, tsne_csr P, const float* Y, float alpha, float* dY,
                  double* Z_out);

/*
 * One gradient-descent iteration at index iter of the schedule sp: computes
 * the gradient with alpha(iter) and updates Y, uY and gains in place
 * (device, [N x s] each). The new Y is produced in plan scratch and copied
 * back, so the attraction of every point sees the old Y.
 */
int tsne_step(tsne_plan* plan, tsne_csr P, float* Y, float* uY, float* gains, int32_t iter,
              const tsne_step_params* sp);

/*
 * A whole run: iterations 0 .. sp->n_iter - 1 of tsne_step starting from
 * uY = 0 and gains = 1 (kept in plan scratch); Y (device) holds Y0 on entry
 * and the embedding on return. If kl_out (HOST pointer) is not NULL, the KL
 * divergence of the final embedding is computed and written (synchronises).
 */
int tsne_run(tsne_plan* plan, tsne_csr P, float* Y, const tsne_step_params* sp,
             double* kl_out);

/*
 * The same run in pieces: tsne_run_reset sets the plan's run state to uY = 0,
 * gains = 1; tsne_run_iters then performs iterations it_begin ..
 * it_begin + count - 1 of the schedule sp on Y (device, in place), keeping
 * uY and gains in the plan between calls. tsne_run equals a reset followed
 * by tsne_run_iters(0, sp->n_iter) (and the optional KL).
 *
 * Locality relabelling, so that the attraction's reads of neighbouring y_j
 * hit nearby memory (cache reuse); each builds the correspondingly
 * relabelled copy of P (plan-owned, allocated on first use: 8 bytes per
 * stored entry), rows keeping their entry order:
 *   - at iteration 0 (a run that starts at iteration 0 in the caller's
 *     labels; plan option order_rounds > 0) the points take the graph order
 *     of P: two pseudo-random coordinates per point are averaged over the
 *     point's row of P order_rounds times (z_i <- sum_j p_ij z_j / sum_j
 *     p_ij; rows without entries keep 0), and the labels follow a Hilbert
 *     curve over the result (mean +- 3 standard deviations per coordinate,
 *     1024 cells each), ties by label. Points of one cluster of the kNN
 *     graph get nearby labels before the embedding has any structure.
 *     The order is kept for later runs with the same P (same pointers and
 *     nnz); the copy of P is rebuilt at every run's start unless
 *     tsne_plan_order prepared it;
 *   - at iteration relabel_first and every relabel_every iterations after
 *     it (plan options) the points are relabelled along a Hilbert curve of
 *     the current embedding (ties by label).
 * Every relabelling is deterministic and leaves every result bitwise
 * unchanged (each row's attraction sum keeps its order; the spread, Z and
 * KL sums do not depend on the labels); Y is returned in the caller's
 * labels. P must stay the same across the tsne_run_iters calls of one run.
 */
int tsne_run_reset(tsne_plan* plan);
int tsne_run_iters(tsne_plan* plan, tsne_csr P, float* Y, const tsne_step_params* sp,
                   int32_t it_begin, int32_t count);

/*
 * Prepares the graph order of P (see tsne_run_iters) and the copy of P in
 * that order, so that later runs of this plan with the same P (same
 * pointers and nnz) start without re-reading P: the caller promises that P's
 * contents do not change until the next tsne_plan_order call (results with
 * a changed P would use the stale copy). An embedding relabelling of a run
 * replaces the copy; the next run then rebuilds it. The paper has no
 * counterpart (a cache-locality analysis of P, like a sparse library's
 * matrix preprocessing). A relabelled run of the plan that is continued
 * afterwards (tsne_run_iters) rebuilds its own copy of P first. Enqueued on
 * the plan's stream. INVALID_ARG if the plan has order_rounds < 0; OOM.
 */
int tsne_plan_order(tsne_plan* plan, tsne_csr P);

/*
 * Checkpoint and resume of a run in pieces (the paper has no counterpart):
 * between tsne_run_iters calls the state of a run is the caller's Y plus
 * the plan's uY and gains. tsne_run_state_save copies uY and gains, in the
 * caller's labels (N x s fp32 each), to HOST buffers and synchronises;
 * tsne_run_state_load installs such HOST buffers as the run state of a plan
 * of the same N and s (this one or another, e.g. in a later process), with
 * no relabelling in effect, and synchronises. Continuing with
 * tsne_run_iters(it_begin = the next iteration, same P and schedule) gives
 * the uninterrupted run's Y bit for bit (relabelling changes no result).
 * INVALID_ARG on NULL buffers; the buffers' sizes are the caller's duty.
 */
int tsne_run_state_save(tsne_plan* plan, float* uY_host, float* gains_host);
int tsne_run_state_load(tsne_plan* plan, const float* uY_host, const float* gains_host);

/*
 * KL(P || Q) = sum_ij p_ij log(p_ij / q_ij) over the stored entries of P
 * (Sec. 1.1), with Z from the interpolation scheme at Y. Squared distances,
 * logarithms and every sum in FP64 (from the FP32 coordinates and values).
 * kl_out is a HOST pointer (synchronises).
 */
int tsne_kl(tsne_plan* plan, tsne_csr P, const float* Y, double* kl_out);

/*
 * Same as tsne_run, but with HOST buffers: row_ptr/col/val (host, CSR as
 * above) and Y (host, [N x s], Y0 in, embedding out) are copied to and from
 * plan-owned device memory inside the call. The CSR is validated on the host
 * first (INVALID_ARG on a malformed matrix). Synchronises.
 */
int tsne_run_host(tsne_plan* plan, const int32_t* row_ptr, const int32_t* col,
                  const float* val, int64_t nnz, float* Y, const tsne_step_params* sp,
                  double* kl_out);

/*
 * Checks a device CSR on the device: row_ptr[0] = 0, non-decreasing,
 * row_ptr[N] = nnz, 0 <= col < N, col != row, finite val >= 0.
 * Returns TSNE_OK or INVALID_ARG (synchronises).
 */
int tsne_validate_csr(tsne_plan* plan, tsne_csr P);

/* Synchronises the plan's stream and returns the latched device status
 * (TSNE_OK, TSNE_ERR_NONFINITE) or TSNE_ERR_CUDA; clears the latch. */
int tsne_plan_status(tsne_plan* plan);

/* Box/grid/Z of the most recent evaluation (synchronises). */
int tsne_plan_info(tsne_plan* plan, tsne_plan_info_t* out);

/*
 * Copies an internal buffer of the most recent evaluation to HOST memory,
 * for tests (synchronises). Nodes are indexed g = (g_1, g_2), row-major; a
 * node's position is y_min + (g + 1/2) delta; t is a point's coordinate
 * inside its box in units of delta and j the node's index in the box.
 *   0  spread grids as FP64 [(s+1) x n^s] (accumulated exactly on the device
 *      in fixed point): w0 = sum_i L_g(y_i) and the dipole grids
 *      d_m = sum_i L_g(y_i) (t_m - j_m - 1/2) = (w_{y(m)} - y~_g(m) w0) / delta
 *   1  node values, fp32 [n^s x 4] = (0, u'_1, u'_2, v) with v = K2 * w0
 *      (= h_{s+2} at the nodes) and u'_m = K2 * d_m - G_m * w0 with
 *      G_m(o) = o_m K2(o delta), i.e. (v_{m+1} - y~(m) v) / delta; u'_2 = 0
 *      when s = 1. (Z is formed from the spectra, so K1 * w0 is not kept.)
 *   2  bucket offsets, int32 [n_int^s + 1] (points per box, exclusive scan)
 * bytes must be at least the size above; the size needed is returned in
 * *bytes_needed (may be NULL).
 */
int tsne_debug_copy(tsne_plan* plan, int32_t which, void* host_dst, size_t bytes,
                    size_t* bytes_needed);

/*
 * Phase timing (tracing). enable != 0 makes every later gradient, step or run
 * record CUDA events on the plan's stream around its four phases:
 *   0 bounding box, 1 counting sort + spread (Step 1),
 *   2 FFT convolution + Z (Step 2), 3 attraction + interpolation + update
 *   (Step 3, the force kernel).
 * tsne_plan_profile_read synchronises, writes the summed milliseconds and
 * the number of timed evaluations per phase to ms_out[4] / count_out[4]
 * (HOST arrays, either may be NULL) and clears the record. enable = 0 stops
 * recording (the record is kept until read).
 */
int tsne_plan_profile(tsne_plan* plan, int32_t enable);
int tsne_plan_profile_read(tsne_plan* plan, double* ms_out, int64_t* count_out);

/* Number of kernels this plan has launched since it was created (host-side
 * count of every kernel launch the library enqueued for it). */
int64_t tsne_plan_launch_count(const tsne_plan* plan);

/* ------------------------------------------------------------------------
 * Batched iterations of many independent embedding jobs.
 *
 * The paper's method is one embedding at a time (Algorithm 1 per
 * iteration); a batch runs the same per-iteration path (box, counting sort,
 * spread, FFT convolution + Z, attraction + Step 3 + update) for many jobs at
 * once: every phase is ONE kernel launch whose blocks share out the work
 * items of all jobs, each job keeping its own P, Y, optimizer state,
 * bounding box, N_int, node grid and FFT length (decided on the device every
 * iteration). The launch sequence of one iteration is captured once in a
 * CUDA graph and replayed, so an iteration of all jobs costs one host call.
 * Jobs join and leave between iterations: their scratch comes from the
 * stream-ordered allocator (cudaMallocAsync on the batch's stream), which
 * never synchronises the device. A job's iterations are bitwise equal to the
 * same job run alone (no kernel mixes values of different jobs; every
 * reduction has a fixed order).
 * ------------------------------------------------------------------------ */
typedef struct tsne_batch tsne_batch;

/* Batch options; tsne_batch_opts_default fills the defaults in brackets. */
typedef struct {
    int32_t n_min;     /* floor of the interval rule [50] (Sec. 2.5) */
    int32_t n_int_max; /* cap of the rule and size of every job's grids [min(1000, 3000 / p) if
                          s = 1, min(400, 1200 / p) if s = 2] */
    int32_t max_jobs;  /* job slots, 1 .. 256 [64] */
    int32_t use_graph; /* 1: replay one captured CUDA graph per iteration [1]; 0: plain launches */
    void* stream;      /* cudaStream_t for all work (not the legacy default stream);
                          NULL: the batch creates its own non-blocking stream */
} tsne_batch_opts;

/* Interval-count policies (the automatic rule of Sec. 2.5 gives r): */
#define TSNE_NINT_RULE 0 /* N_int = r */
#define TSNE_NINT_FILL 1 /* the most intervals whose nodes fit the FFT length r gets (>= r, <= n_int_max) */

/* Tuning of a batch (see tsne_batch_autotune). */
typedef struct {
    int32_t chunk;        /* points per spread work item, one warp each: 32, 64 [64], 128 or 256
                             (a box of c points gets ceil(c / chunk) warps) */
    int32_t fft_threads;  /* threads per CTA of the 2-D FFT passes: 256, 512, 1024, or 0 [0] for
                             256 (row passes) / 512 (column pass) */
    int32_t n_int_policy; /* TSNE_NINT_RULE [default] or TSNE_NINT_FILL */
    float ms_per_iter;    /* set by tsne_batch_autotune: measured time of one iteration */
} tsne_batch_tuning;

void tsne_batch_opts_default(tsne_batch_opts* out);

/* Creates an empty batch of jobs in s dimensions (1 or 2) with p nodes per
 * interval (2..5). Errors: INVALID_ARG, OOM, CUDA. */
int tsne_batch_create(int32_t s, int32_t p, const tsne_batch_opts* opts, tsne_batch** out);

/* Frees the batch and every job's scratch (synchronises its stream). NULL is a no-op. */
int tsne_batch_destroy(tsne_batch* batch);

/* Device bytes a job of N points takes in this batch (Y, two Y buffers,
 * optimizer state and grid scratch; P is the caller's and not counted), or -1. */
int64_t tsne_batch_job_bytes(const tsne_batch* batch, int64_t N);

/* Device bytes of all jobs now in the batch (sum of tsne_batch_job_bytes). */
int64_t tsne_batch_bytes_in_use(const tsne_batch* batch);

/*
 * Adds a job: N points, affinities P (device CSR as in tsne_gradient; the
 * caller keeps P alive and unchanged until the job is removed), Y0 (device,
 * [N x s], copied into the job), n_intervals (0 = the automatic rule, else a
 * fixed N_int <= n_int_max) and the schedule sp (copied; the job runs
 * iterations 0 .. sp->n_iter - 1 with uY = 0, gains = 1 at the start, exactly
 * as tsne_run). *job_id receives the job's slot (0 .. max_jobs - 1). Work is
 * enqueued on the batch's stream. Errors: INVALID_ARG, CAPACITY (no free
 * slot), OOM, CUDA.
 */
int tsne_batch_add_job(tsne_batch* batch, int64_t N, tsne_csr P, const float* Y0,
                       int32_t n_intervals, const tsne_step_params* sp, int32_t* job_id);

/* Removes a job and returns its scratch to the stream-ordered pool (after the
 * work already enqueued). Fetch its result first (tsne_batch_get_y). */
int tsne_batch_remove_job(tsne_batch* batch, int32_t job_id);

/* Enqueues count iterations of every job still inside its schedule (jobs
 * that finished skip every phase). */
int tsne_batch_iterate(tsne_batch* batch, int32_t count);

/* Synchronises the batch's stream; for every slot k writes the job's next
 * iteration index (= iterations done; -1 for a free slot) to iter_out[k] and
 * its latched device status (TSNE_OK or TSNE_ERR_NONFINITE) to status_out[k]
 * (HOST arrays of max_jobs entries; either may be NULL). */
int tsne_batch_poll(tsne_batch* batch, int32_t* iter_out, int32_t* status_out);

/* Enqueues a copy of the job's current Y to Y_out (device, [N x s]). */
int tsne_batch_get_y(tsne_batch* batch, int32_t job_id, float* Y_out);

/* KL(P || Q) of the job's current Y (as tsne_kl; Z recomputed at that Y).
 * kl_out is a HOST pointer; synchronises. */
int tsne_batch_kl(tsne_batch* batch, int32_t job_id, double* kl_out);

/* Sets or reads the tuning used from the next iteration on (every job). */
int tsne_batch_set_tuning(tsne_batch* batch, const tsne_batch_tuning* t);
int tsne_batch_get_tuning(const tsne_batch* batch, tsne_batch_tuning* out);

/*
 * Autotuner: times `iters` iterations of the batch's current jobs under
 * candidate tunings (coordinate search over chunk in {32, 64, 128, 256}, then
 * fft_threads in {256, 512, 1024} for s = 2), restoring every job's state
 * after each trial, so the jobs' results do not depend on the tuning run.
 * Neither knob changes a result bit; the interval policy, which does, is
 * left as the caller set it (TSNE_NINT_FILL changes a run's final KL by up
 * to about 1 %). Applies the fastest tuning and writes it (with its measured
 * ms_per_iter) to *out (may be NULL). Synchronises; needs at least one job.
 */
int tsne_batch_autotune(tsne_batch* batch, int32_t iters, tsne_batch_tuning* out);

/* Kernels this batch has launched (host-side count). */
int64_t tsne_batch_launch_count(const tsne_batch* batch);

/* The batch's cudaStream_t. */
void* tsne_batch_stream(const tsne_batch* batch);

/*
 * Input affinities P from data X on the GPU (Sec. 1.1, Eq. p_ij, with the
 * k exact nearest neighbours of Sec. 3 in place of all points):
 *   p_{j|i} = exp(-beta_i d_ij^2) / sum_{l in kNN(i)} exp(-beta_i d_il^2)
 *   beta_i by bisection so that exp(H(P_i)) = perplexity (natural log),
 *     stopping at |H - log perplexity| < 1e-5 or after 200 steps (the paper
 *     gives no stopping rule);
 *   p_ij = (p_{j|i} + p_{i|j}) / (2N), CSR with sorted columns, no diagonal.
 * Distances are FP32 in difference form; neighbours are ordered by
 * (distance, index); the bisection runs in FP64; values are rounded once to
 * FP32. Every step is deterministic.
 *
 * tsne_affinity_create: workspace for N points of dimension D (1..64) and k
 * neighbours (1..256, k < N, 2 N k < 2^31); all device memory (about
 * 40 N k bytes) is allocated here; work is enqueued on stream (cudaStream_t,
 * NULL = legacy default). INVALID_ARG on bad sizes, OOM. The kNN kernel is
 * chosen here: the tensor-core one (tcgen05 tiles of 128 x 128
 * approximate distances shortlist the candidates; the shortlist gets the
 * exact FP32 distances; queries whose shortlist is not provably complete
 * are recomputed by the row kernel; it needs about 1040 + 8 S bytes more
 * device memory per point, S = 2 k + 32 rounded up to 64, 128, 256 or 512,
 * plus 512 KB per SM). The environment variable FITSNE_KNN_KERNEL=tiled or
 * =rows, read at create, selects the register-tiled FP32 kernel (where its
 * shared memory (D, k) fits) or the one-candidate-per-lane one instead (all
 * three give the same lists and distances, bit for bit).
 * tsne_affinity_compute: X is DEVICE memory, N x D row-major FP32, read
 * only; 1 <= perplexity <= k. Writes into *P_out a CSR that points into the
 * workspace: valid until the next compute or destroy, owned by the
 * workspace. Synchronises the stream (the host needs nnz).
 * tsne_affinity_knn_copy: copies the last compute's neighbour lists
 * (N x k, sorted by (d^2, index)), their squared distances and p_{j|i} to
 * host buffers (any may be NULL). INVALID_ARG before the first compute.
 */
typedef struct tsne_affinity tsne_affinity;
int tsne_affinity_create(int64_t N, int32_t D, int32_t k, void* stream, tsne_affinity** out);
int tsne_affinity_destroy(tsne_affinity* aff);
int tsne_affinity_compute(tsne_affinity* aff, const float* X, double perplexity, tsne_csr* P_out);
int tsne_affinity_knn_copy(const tsne_affinity* aff, int32_t* idx_host, float* d2_host,
                           double* pcond_host);
/* Device time (CUDA events on the workspace's stream) of the last compute's
 * phases: ms_out[0] kNN, [1] bandwidths, [2] edge sort, [3] symmetrisation.
 * INVALID_ARG before the first compute. */
int tsne_affinity_phase_ms(const tsne_affinity* aff, double* ms_out);
/* Kernels the workspace has launched (host-side count). */
int64_t tsne_affinity_launch_count(const tsne_affinity* aff);
/* The kNN kernel chosen at create (*kernel_out: 0 row kernel, 1 register-
 * tiled, 2 tensor cores) and the number of queries of the last compute that
 * the tensor-core kernel left to the row kernel (*recomputed_out; 0 for the
 * other kernels). Either pointer may be NULL. INVALID_ARG on a NULL
 * workspace. */
int tsne_affinity_knn_info(const tsne_affinity* aff, int32_t* kernel_out, int64_t* recomputed_out);

/*
 * t-SNE heatmaps (Sec. 5). A 1-D embedding y of N cells is cut into n_bins
 * equal-width bins over [min y, max y]:
 *   w = (max y - min y) / n_bins,  bin(y) = floor((y - min y) * (1 / w)),
 * each operation rounded once in FP32 (round to nearest, no FMA), clamped to
 * [0, n_bins - 1]; w = 0 (or 1 / w not finite) puts every cell in bin 0.
 * Gene g becomes h_g in R^{n_bins}, h_g[b] = sum of E[i, g] over the cells i
 * of bin b, and genes are compared by |h_g - h_g'| (Euclidean); each gene
 * of interest is enriched with the m genes nearest to it (itself excluded,
 * ties by the smaller gene index), the rows of the heatmap.
 *
 * tsne_heatmap_create: workspace for n_bins (1..2^20) bins, G genes and up
 * to max_goi (1..65535) genes of interest per search (about 8 max_goi G
 * bytes of device memory, allocated here); work is enqueued on stream
 * (cudaStream_t, NULL = legacy default). INVALID_ARG on bad sizes, OOM.
 * tsne_heatmap_bin: y is DEVICE fp32 [N] (1 <= N <= 2^31 - 2); E is the
 * cells x genes expression matrix as a DEVICE CSR (int32 row_ptr[N + 1],
 * int32 gene index col[nnz] in [0, G), fp32 val[nnz]; nnz < 2^31). Writes
 * the caller's DEVICE buffers H, FP64 n_bins x G row-major (H[b * G + g] =
 * h_g[b]), and bin_count, int32 [n_bins] (cells per bin). H is summed with
 * FP64 atomics: its last bits may differ between calls. Synchronises the
 * stream; NONFINITE if y holds NaN or Inf, INVALID_ARG if a row of E is
 * malformed (row_ptr decreasing or beyond nnz) or a gene index is out of
 * range (such rows / entries are skipped, the rest is summed).
 * tsne_heatmap_nearest: for each of the n_goi (1..max_goi) gene indices in
 * goi_host (HOST memory), the m (1..min(256, G - 1)) genes nearest to it in
 * the distance above over the DEVICE matrix H of the last bin call:
 * idx_host[q * m + r] and dist_host[q * m + r] (HOST, n_goi x m, int32 and
 * FP64, in increasing distance). Synchronises the stream; INVALID_ARG on bad
 * sizes or an index outside [0, G).
 * tsne_heatmap_phase_ms: device time (CUDA events) of the last calls:
 * ms_out[0] clearing and range, [1] binning and sums, [2] distances,
 * [3] selection (0 before the first search). INVALID_ARG before a bin call.
 */
typedef struct tsne_heatmap tsne_heatmap;
int tsne_heatmap_create(int32_t n_bins, int32_t G, int32_t max_goi, void* stream, tsne_heatmap** out);
int tsne_heatmap_destroy(tsne_heatmap* hm);
int tsne_heatmap_bin(tsne_heatmap* hm, const float* y, int64_t N, tsne_csr E, double* H, int32_t* bin_count);
int tsne_heatmap_nearest(tsne_heatmap* hm, const double* H, const int32_t* goi_host, int32_t n_goi, int32_t m,
                         int32_t* idx_host, double* dist_host);
int tsne_heatmap_phase_ms(const tsne_heatmap* hm, double* ms_out);
/* Kernels the workspace has launched (host-side count). */
int64_t tsne_heatmap_launch_count(const tsne_heatmap* hm);

/*
 * KL(P || Q) without any device allocation (the paper has no counterpart;
 * this exists for callers that cannot call cudaMalloc, e.g. a process whose
 * own allocator owns all device memory, or code that must not let
 * cudaMalloc/cudaFree synchronise the device). Same sum as tsne_kl, for the
 * caller's Z (the value tsne_gradient wrote to Z_out at the same Y):
 *   KL = sum p log p + sum p log(1 + |y_i - y_j|^2) + (sum p) log Z.
 * P and Y (N x s, s = 1 or 2) are device data as in tsne_gradient; kl_out is
 * a DEVICE address that receives one double; work is enqueued on stream
 * (cudaStream_t, NULL = legacy default) and the call returns without
 * synchronising. 1 <= N <= 2^31 - 2 and 0 <= nnz <= 2^31 - 1, else
 * INVALID_ARG. Its scratch is a fixed 16,640-byte array in the library's
 * device image (per-block partial sums of at most 1,024 reduction blocks and
 * a completion counter), held by every GPU that loads the library until
 * process exit. The first call on a device looks up that array's address
 * (cudaGetSymbolAddress), so make it before any stream capture; the address
 * is kept until process exit, so do not call this entry point on a device
 * the process has reset with cudaDeviceReset (the array may move). All calls
 * share the array: calls whose work overlaps on the GPU (different streams,
 * or different host threads on one device) race; serialise them.
 * tsne_noalloc_last_error_string describes the last failure of this entry
 * point on the calling thread.
 */
int tsne_kl_noalloc(tsne_csr P, const float* Y, int64_t N, int32_t s, double Z, double* kl_out,
                    void* stream);
const char* tsne_noalloc_last_error_string(void);

#ifdef __cplusplus
}
#endif

#endif /* FITSNE_GB300_H */
