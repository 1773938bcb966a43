// Internal declarations of the GB300 FIt-SNE library: the job table every
// kernel walks, the per-iteration parameter block written on the device, the
// plan and batch objects, shared device helpers and the kernel launchers.
// Not part of the public ABI (include/fitsne_gb300.h).
//
// Every per-iteration kernel serves a whole table of independent jobs (a
// plan is a table of one job; a batch holds up to kMaxJobs). Each job owns
// its box, grid, FFT length and scratch; a kernel's blocks share out the
// work items of all jobs (the item counts may depend on each job's grid of
// the current iteration, decided on the device), so one launch per phase
// serves every job and the launch geometry never depends on a device value.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fitsne_gb300.h"

namespace fitsne {

constexpr int kWarp = 32;
constexpr int kMaxStages = 16;    // radix stages of one FFT
constexpr int kScanBlock = 2048;  // boxes per scan work item (1024 threads x 2)
constexpr int kBoxThreads = 256;  // threads of the bounding-box blocks
constexpr int kBoxBlocks = 608;   // bounding-box work items of a large job (4 per SM)
constexpr int kHistBins = 11776;  // boxes of a shared-memory histogram (46 KB: with the
                                  // job split it stays under the 48 KB default limit)
constexpr int kSortPts = 2048;    // points per work item of the sort kernels (256 threads x 8)
constexpr int kForceChunk = 256;  // rows per work item of the force kernel (8 warps x 32)
constexpr int kMaxJobs = 256;     // jobs of one table
constexpr int kMinChunk = 32;     // smallest spread work item (points)
#ifndef FITSNE_DEFAULT_CHUNK
#define FITSNE_DEFAULT_CHUNK 64
#endif
constexpr int kDefaultChunk = FITSNE_DEFAULT_CHUNK;  // points per spread work item of a plan

// One FFT length of the table: L = product of radix[0..nst), each radix in
// {2, 3, 4, 5}; tw_off locates its L twiddles exp(-2 pi i j / L).
struct FftEntry {
    int32_t L;
    int32_t nst;
    int32_t tw_off;
    int32_t radix[kMaxStages];
};

// Box, grid, schedule values and normalisation of a job's current
// iteration. Written by the bounding-box kernel (box fields, active, alpha,
// momentum, cur), the scan (n_chunks) and the last column-FFT item (Z); read
// by every later kernel of the iteration.
struct Params {
    float y_min;      // box lower corner (Sec. 2.2)
    float width;      // box side
    float b;          // interval width, width / n_int
    float inv_b;      // 1 / b (FP32, decides the interval of a point)
    float delta;      // node spacing b / p
    float inv_delta;  // p / b
    float delta2;     // delta^2 (kernel argument scale)
    float fx_scale;   // 2^fx_shift: spread values are accumulated as integers x * fx_scale
    int32_t n_int;    // intervals per dimension
    int32_t n;        // nodes per dimension = p * n_int
    int32_t L;        // FFT length per dimension (even, >= 2n)
    int32_t n_boxes;  // n_int^s
    int32_t fft_idx;  // entry of the FFT table
    int32_t n_chunks; // spread work items
    int32_t error;    // latched TSNE_ERR_NONFINITE
    int32_t fx_shift; // binary point of the fixed-point spread grids
    double Z;         // sum_i h_1(y_i) - N
    float inv_Z;      // 1 / Z in FP32
    float fx_inv;     // 2^-fx_shift
    float p_f;        // p as a float
    int32_t active;   // 0: the job is past its schedule (every later kernel skips it)
    float alpha;      // exaggeration of this iteration
    float momentum;   // momentum of this iteration (step mode)
    int32_t cur;      // ybuf[cur] holds the Y of this iteration
    int32_t pad;
};

// Per-job state advanced on the device after every step, so that a fixed
// launch sequence (or a CUDA graph of it) can be replayed iteration after
// iteration.
struct JobDyn {
    int32_t iter;   // schedule index of the next step
    int32_t cur;    // ybuf[cur] holds the current Y
    int32_t error;  // copy of the latched Params::error (for polling)
    int32_t pad;
};

enum : int32_t { kModeGradient = 0, kModeStep = 1 };

// One row of the job table (device memory). Pointers are device addresses.
struct Job {
    // affinities P (CSR; a relabelled copy during a relabelled run)
    const int32_t* row_ptr;
    const int32_t* col;
    const float* val;
    // embedding: ybuf[cur] is read; a step writes ybuf[cur ^ 1]
    float* ybuf[2];
    float* dY;      // gradient mode: output
    float* uY;      // step mode: momentum state
    float* gains;   // step mode: gains
    double* Z_out;  // optional device address receiving Z
    JobDyn* dyn;
    int64_t N;
    int32_t mode;   // kModeGradient or kModeStep
    float alpha;    // gradient mode: exaggeration
    // schedule (step mode; Sec. 1.2 early and Sec. 4 late exaggeration)
    int32_t n_iter, early_iters, late_iters, mom_switch_iter;
    float early_alpha, late_alpha, lr, momentum_early, momentum_late, min_gain, gain_inc,
        gain_dec;
    // interval rule (Sec. 2.5) and grid
    int32_t n_int_fixed, n_min, n_int_max, fx_shift;
    int32_t force_box, force_n_int;
    float force_y_min, force_width;
    int32_t chunk;                // points per spread work item
    int32_t iter_end;             // step mode: the job is active while dyn->iter < iter_end
    const int32_t* n_int_table;   // [n_int_max + 1]: N_int used for rule value r (NULL: r)
    // scratch (see JobMem)
    Params* params;
    float* box_partial;      // [2 kBoxBlocks]
    unsigned* tickets;       // [4] self-resetting completion counters
    int32_t* counts;         // [n_boxes_max] points per box (zero between iterations)
    int32_t* box_start;      // [n_boxes_max + 1]
    int32_t* cursor;         // [n_boxes_max]
    int32_t* chunk_start;    // [n_boxes_max + 1]
    int32_t* chunk_box;      // [chunk_cap]
    int32_t* block_pts;      // [scan items]
    int32_t* block_chunks;   // [scan items]
    float* sorted_y;         // [N s]
    long long* w;            // [(s+1) n_max^s] fixed point
    float2* spec;            // [4 n_max L_max] (s = 2)
    float4* hgrid;           // [n_max^s]
    double* z_partial;       // [L_max / 2 + 1]
};

// Table-wide constants of one launch (shared by every job of the table).
struct Tables {
    const FftEntry* fft;      // FFT lengths
    const float2* tw;         // twiddles
    const int32_t* fft_of_n;  // [n_max + 1] entry for n nodes per dimension
};

// Scratch of one job, carved out of one device allocation (JobMem::bytes).
struct JobLayout {
    int64_t N;
    int s, p, n_int_max;
    int n_max, L_max;
    int64_t n_boxes_max, chunk_cap, G;
    int scan_items;
};

// Per-table capacities that size the launch grids (upper bounds of each
// phase's work items over the table).
struct TableCaps {
    int s, p;
    int njobs;
    int64_t sum_N;          // points of all jobs
    int64_t sum_box_items;  // bounding-box work items of all jobs
    int64_t sum_chunk_cap;  // spread work items of all jobs (upper bound)
    int max_n;              // largest nodes per dimension of any job
    int max_L;              // largest FFT length of any job
    int max_scan_items;     // largest scan work items of any job
    int sm_count;
    int fft_threads;        // threads per CTA of the 2-D FFT passes (0: 256 rows / 512 columns)
};

JobLayout job_layout(int64_t N, int s, int p, int n_int_max, int L_max);
// Bytes of the job's scratch (including ybuf[1], uY, gains when with_state).
size_t job_scratch_bytes(const JobLayout& lay, bool with_state);
// Points the scratch fields of J (and ybuf[1], uY, gains when with_state) into base.
void job_carve(const JobLayout& lay, void* base, bool with_state, Job* J);
// Zeroes what must start at zero (parameter block, counters, box counts).
cudaError_t job_zero(const JobLayout& lay, const Job& J, cudaStream_t st);

// ----------------------------------------------------------------------------
// Host helpers shared by the plan and the batch (fitsne_abi.cu).
// ----------------------------------------------------------------------------
// Records a failure for tsne_last_error_string and returns code.
int set_error(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
void clear_error();
// Binary point of the fixed-point spread for N points.
int fixed_point_shift(int64_t N, int s, int p);
// FFT length table (every even 5-smooth L up to the first >= 2 n_max) with
// twiddles and the n -> entry map, in device memory.
struct FftSet {
    FftEntry* table = nullptr;
    float2* tw = nullptr;
    int32_t* of_n = nullptr;
    int n_fft = 0;
    int L_max = 0;
    size_t bytes = 0;
};
int fft_set_create(int n_max, cudaStream_t st, FftSet* out);
void fft_set_destroy(FftSet* f);
// Fills the schedule fields of J from sp (step mode).
void job_set_schedule(Job* J, const tsne_step_params* sp);

}  // namespace fitsne

struct tsne_plan {
    int64_t launches;       // kernels launched for this plan
    int profiling;          // record phase events
    void* prof;             // phase event record (fitsne_abi.cu)
    int64_t N;
    int s, p;
    int n_int_fixed, n_min, n_int_max;
    cudaStream_t stream;
    int n_max;              // p * n_int_max
    int sm_count;
    fitsne::JobLayout lay;
    fitsne::TableCaps caps;
    // box override (test hook)
    int force_box;
    float force_y_min, force_width;
    int force_n_int;
    int fx_shift;            // fixed-point binary point of the spread (plan constant)
    // the plan's one-row job table
    void* job_mem;           // the job's scratch (JobLayout)
    fitsne::Job host_job;    // host copy of the row (written to the device when it changes)
    fitsne::Job uploaded;    // what the device row holds
    int uploaded_valid;
    fitsne::Job* d_job;      // [1] device table
    fitsne::JobDyn* d_dyn;   // [1]
    fitsne::FftSet fft;
    fitsne::Tables tables;
    double* kl_partial;      // [kl_blocks]
    unsigned* kl_ticket;     // [1]
    double* kl_out_dev;      // [1]
    int32_t* valid_flag;     // [1]
    float* y_next;           // [N * s]
    float* uY_run;           // [N * s] (tsne_run state)
    float* gains_run;        // [N * s]
    // locality relabelling of a run (fitsne_reorder.cu)
    int relabel_first, relabel_every;  // iterations at which a run relabels (first < 0: never)
    int reordered;           // run state and rp2/col2/val2 use the relabelled order
    int32_t* perm;           // [N] new label -> caller's label
    int32_t* inv;            // [N] caller's label -> new label
    int32_t* perm_next;      // [N]
    int32_t* inv_next;       // [N]
    int32_t* row_len;        // [N]
    int32_t* cur_of;         // [N]
    int32_t* rp2;            // [N + 1] relabelled P
    int32_t* col2;           // [nnz2_cap]
    float* val2;             // [nnz2_cap]
    int64_t nnz2_cap;
    unsigned long long* sort_keys;  // [next_pow2(N)]
    int32_t* scan_bsum;      // [N / 2048 + 1]
    unsigned* relabel_ticket;  // [1]
    float* tmp_state;        // [N * s]
    float* y_cur;            // [N * s] run state Y in the relabelled order
    // graph order of a run's start (fitsne_reorder.cu), allocated on first use
    int order_rounds;        // averaging rounds of the graph order (0: runs start in the caller's labels)
    int32_t* gperm;          // [N] graph order: new label -> caller's label
    int32_t* ginv;           // [N] its inverse
    int gorder_valid;        // gperm/ginv hold the graph order of the P in gorder_key
    tsne_csr gorder_key;     // pointers and nnz of that P
    int gorder_prepared;     // tsne_plan_order: runs with that P may reuse rp2/col2/val2
    int p2_holds_gorder;     // rp2/col2/val2 hold that P in the graph order
    int p2_is_run;           // rp2/col2/val2 hold the run's P in the run's order (perm/inv)
    float* order_z;          // [4 N] two float2 coordinate buffers
    double* order_stats;     // [4 * 256 + 2] block partials, then the key window (4 floats)
    // steady-state step of a run as a CUDA graph (box with the deferred
    // advance, sort, spread, FFT, forces), replayed on gstream; built on first use
    cudaStream_t gstream;
    cudaGraphExec_t step_exec;
    int step_kernels;        // kernels of one replay
    cudaEvent_t g_in, g_out; // fences between the plan's stream and gstream
    // force kernel scheduling
    int force_mode;          // TSNE_FORCE_* (plan option)
    int n_regions;           // SM id range of the device
    unsigned* region_next;   // [n_regions + 1] block counters of the region-scheduled kernel, claimed total
    // host-buffer path (tsne_run_host), allocated on first use
    int64_t host_nnz_cap;
    int32_t* h_row_ptr;
    int32_t* h_col;
    float* h_val;
    float* h_Y;
};

namespace fitsne {

// ----------------------------------------------------------------------------
// Work sharing over the jobs of a table. split_jobs fills s_start[0..njobs]
// with the exclusive prefix of count(J) over the table (the whole block
// calls it; blockDim.x must be a multiple of 32 and at most 1024) and
// returns the total; job_of maps an item of [0, total) to its job.
// ----------------------------------------------------------------------------
__device__ __forceinline__ int warp_incl_scan(int x) {
    const int lane = threadIdx.x % 32;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

template <typename F>
__device__ __forceinline__ int split_jobs(const Job* __restrict__ jobs, int njobs, int32_t* s_start,
                                          F count) {
    if (njobs == 1) {  // a plan: one count, two barriers
        __syncthreads();   // an earlier split's total has been read by every thread
        if (threadIdx.x == 0) {
            s_start[0] = 0;
            s_start[1] = count(jobs[0]);
        }
        __syncthreads();
        return s_start[1];
    }
    __shared__ int32_t s_wsum[32];
    __shared__ int32_t s_carry;
    const int lane = threadIdx.x % 32, wid = threadIdx.x / 32, nw = blockDim.x / 32;
    if (threadIdx.x == 0) s_carry = 0;
    for (int base = 0; base < njobs; base += blockDim.x) {
        const int j = base + threadIdx.x;
        const int c = j < njobs ? count(jobs[j]) : 0;
        const int x = warp_incl_scan(c);
        __syncthreads();  // s_carry and s_wsum of the previous pass are consumed
        if (lane == 31) s_wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            const int t = lane < nw ? s_wsum[lane] : 0;
            s_wsum[lane] = warp_incl_scan(t);
        }
        __syncthreads();
        const int ex = x - c + (wid ? s_wsum[wid - 1] : 0) + s_carry;
        if (j < njobs) s_start[j] = ex;
        __syncthreads();
        if (threadIdx.x == 0) s_carry += s_wsum[nw - 1];
    }
    __syncthreads();
    if (threadIdx.x == 0) s_start[njobs] = s_carry;
    __syncthreads();
    return s_start[njobs];
}

__device__ __forceinline__ int job_of(const int32_t* s_start, int njobs, int item) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_start[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// A job takes part in the phases after the bounding box iff this holds.
__device__ __forceinline__ bool job_live(const Params& P) { return P.active && !P.error; }

// ----------------------------------------------------------------------------
// Device helpers shared by the spread and the gather (identical weights on
// both sides of the convolution).
// ----------------------------------------------------------------------------

// Interval of coordinate y: floor((y - y_min) * inv_b) in FP32 round-to-nearest
// with no contraction, clamped to [0, n_int - 1].
__device__ __forceinline__ int interval_of(float y, const Params& P) {
    float f = __fmul_rn(__fsub_rn(y, P.y_min), P.inv_b);
    if (!(f >= 0.0f)) return 0;
    if (f >= (float)P.n_int) return P.n_int - 1;
    int l = (int)floorf(f);
    return l > P.n_int - 1 ? P.n_int - 1 : l;
}

// Local coordinate t = (y - (y_min + l b)) / delta = p (y - y_min - l b) / b
// in units of the node spacing. The differences are taken exactly (two-sum
// and two-product) and the scaling is one product and one correctly rounded
// division by the FP32 interval width itself, so t carries FP32 accuracy far
// from the box corner and its rounding errors are unbiased (no rounded
// 1/delta shared by every point).
__device__ __forceinline__ float local_t(float y, int l, const Params& P) {
    float u = __fsub_rn(y, P.y_min);
    float bb = __fsub_rn(u, y);
    float u_lo = __fadd_rn(__fsub_rn(y, __fsub_rn(u, bb)), __fsub_rn(-P.y_min, bb));
    float lf = (float)l;
    float m = __fmul_rn(lf, P.b);
    float m_lo = __fmaf_rn(lf, P.b, -m);
    float d = __fadd_rn(__fsub_rn(u, m), __fsub_rn(u_lo, m_lo));
    return __fdiv_rn(__fmul_rn(d, P.p_f), P.b);
}

// Lagrange basis on nodes j + 1/2, j = 0..PP-1 (Sec. 2.1, Eq. kerinterp).
template <int PP>
__device__ __forceinline__ void lagrange(float t, float (&Lw)[PP]) {
#pragma unroll
    for (int j = 0; j < PP; ++j) {
        float num = 1.0f, den = 1.0f;
#pragma unroll
        for (int k = 0; k < PP; ++k) {
            if (k == j) continue;
            num *= t - ((float)k + 0.5f);
            den *= (float)(j - k);
        }
        Lw[j] = num * (1.0f / den);
    }
}

// ----------------------------------------------------------------------------
// Launchers (defined in the .cu files). Each enqueues one phase for the
// njobs rows of the device table jobs on stream; sm_count sizes the grids;
// caps give per-table upper bounds of the work (see TableCaps).
// ----------------------------------------------------------------------------

// ignore_schedule: every job is active with alpha from the job (KL passes);
// advance_first: stepping jobs first move to their next iteration (what
// launch_advance does), so that no advance kernel runs between two steps
cudaError_t launch_box(const Job* jobs, const TableCaps& c, const Tables& t, int ignore_schedule,
                       cudaStream_t st, int advance_first = 0);
cudaError_t launch_sort_and_spread(const Job* jobs, const TableCaps& c, cudaStream_t st);
cudaError_t launch_convolution(const Job* jobs, const TableCaps& c, const Tables& t,
                               cudaStream_t st);
cudaError_t launch_forces(const Job* jobs, const TableCaps& c, int step, cudaStream_t st);
cudaError_t launch_advance(const Job* jobs, int njobs, cudaStream_t st);
// Force/update step with SM-local scheduling of the tables' 32-row blocks
// (next: n_regions counters and the claimed total, zeroed here before the launch).
cudaError_t launch_forces_region(const Job* jobs, const TableCaps& c, int step, unsigned* next,
                                 int n_regions, cudaStream_t st);
// Writes the device's SM id range (%nsmid) to out_dev.
cudaError_t query_sm_id_count(int* out_dev, cudaStream_t st);
// Stream-ordered write of one table row (and, if dyn is not NULL, its JobDyn)
// through a kernel argument: no host staging buffer outlives the call.
cudaError_t launch_job_write(Job* dst, const Job& job, JobDyn* dyn_dst, const JobDyn* dyn,
                             cudaStream_t st);
// dst[0 .. N s) = row->ybuf[row->dyn->cur] (the job's current Y).
cudaError_t launch_copy_current(const Job* row, int64_t count, float* dst, cudaStream_t st);
cudaError_t fft_configure(int s, int L_max);  // shared-memory limits of the FFT kernels
int phase_launches(int s);  // kernels of one iteration (box .. advance)

// Relabels the run (state Y_cur, uY_cur, gains_cur in the current labels) and
// builds the relabelled P; the relabelled Y goes to Y_out, uY and gains are
// moved in place.
cudaError_t launch_relabel(tsne_plan* pl, const tsne_csr& P, const float* Y_cur, float* uY_cur,
                           float* gains_cur, float* Y_out);
// Graph order of P alone (rounds of neighbour averaging of two coordinates,
// Hilbert keys, sort): perm_out[k] = caller's label of new label k, inv_out
// its inverse. Uses pl->order_z, order_stats, sort_keys.
cudaError_t launch_graph_order(tsne_plan* pl, const tsne_csr& P, int rounds, int32_t* perm_out,
                               int32_t* inv_out);
// rp2/col2/val2 = P relabelled by (perm, inv), entries of each row in their order.
cudaError_t launch_order_copy(tsne_plan* pl, const tsne_csr& P, const int32_t* perm,
                              const int32_t* inv);
// Moves the run state to the order perm (new label -> caller's label), as
// launch_relabel does; copy_P = 0 keeps rp2/col2/val2 (they already hold P in
// that order).
cudaError_t launch_apply_order(tsne_plan* pl, const tsne_csr& P, const int32_t* perm, int copy_P,
                               const float* Y_cur, float* uY_cur, float* gains_cur, float* Y_out);
// to_caller = 1: dst[perm[k]] = src[k]; 0: dst[k] = src[perm[k]].
cudaError_t launch_to_labels(tsne_plan* pl, const float* src, int to_caller, float* dst);
// KL reduction with explicit scratch: 2 doubles per block in partial, a
// self-resetting completion counter, Z from Z_dev (device) or Z_val.
cudaError_t launch_kl_raw(const tsne_csr& P, const float* Y, int64_t N, int s,
                          const double* Z_dev, double Z_val, double* partial, unsigned* ticket,
                          double* out, int blocks, cudaStream_t stream);
cudaError_t launch_validate(const tsne_csr& P, int64_t N, int32_t* flag, int sm_count,
                            cudaStream_t st);
cudaError_t launch_fill(float* a, float v, int64_t n, int sm_count, cudaStream_t st);

// Exact kNN with the distance tiles on the tensor cores (fitsne_knn_tc.cu):
// lists and distances bit for bit those of knn_kernel; queries whose
// shortlist cannot be proved complete are listed for knn_kernel.
struct KnnTc;
bool knn_tc_supported(int D, int k);
int knn_tc_create(int64_t N, int D, int k, int sm_count, KnnTc** out);
void knn_tc_destroy(KnnTc* w);
// Enqueues the pass over X (N x D device, FP32) on st; *launches += kernels.
int knn_tc_launch(KnnTc* w, const float* X, int32_t* out_idx, float* out_d2, cudaStream_t st,
                  int64_t* launches);
// Synchronises st, then: the queries left to the row kernel (count, device
// list). TSNE_ERR_TIMEOUT if a pipeline wait of the pass gave up.
int knn_tc_leftover(KnnTc* w, cudaStream_t st, int64_t* count, const int32_t** list);

}  // namespace fitsne
