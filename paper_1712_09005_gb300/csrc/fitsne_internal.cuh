// Internal declarations of the GB300 FIt-SNE library: the per-iteration
// parameter block written on the device, the plan, shared device helpers and
// the kernel launchers. Not part of the public ABI (include/fitsne_gb300.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fitsne_gb300.h"

namespace fitsne {

constexpr int kWarp = 32;
constexpr int kChunk = 128;       // sorted points per spread work item
constexpr int kMaxStages = 16;    // radix stages of one FFT
constexpr int kScanBlock = 2048;  // boxes per scan block (1024 threads x 2)
constexpr int kBoxThreads = 256;  // threads of the bounding-box blocks
constexpr int kBoxBlocks = 304;   // 2 per SM on 152 SMs
constexpr int kHistBins = 12288;  // boxes that fit a shared-memory histogram (48 KB)
constexpr int kSortPts = 2048;    // points per block of the sort kernels (256 threads x 8)
constexpr int kForceChunk = 256;  // rows per CTA step of the force kernel (8 warps x 32)
#ifndef FITSNE_WIN_BYTES
#define FITSNE_WIN_BYTES 98304    // shared-memory window of Y per force CTA (relabelled runs)
#endif

// One FFT length of the plan's table: L = product of radix[0..nst), each
// radix in {2, 3, 4, 5}; tw_off locates its L twiddles exp(-2 pi i j / L).
struct FftEntry {
    int32_t L;
    int32_t nst;
    int32_t tw_off;
    int32_t radix[kMaxStages];
};

// Box, grid and normalisation of the current iteration. Written by the
// bounding-box kernel (box fields), the scan (n_chunks) and the last
// inverse-FFT block (Z); read by every later kernel of the iteration.
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
    int32_t pad;
};

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
    int L_max;              // largest FFT length in the table
    int64_t n_boxes_max;    // n_int_max^s
    int64_t chunk_cap;      // capacity of the chunk table
    int scan_blocks;        // ceil(n_boxes_max / kScanBlock)
    int n_fft;              // entries in the FFT table
    int32_t* fft_of_n;      // [n_max + 1] FFT table entry for n nodes per dimension
    int sm_count;
    // box override (test hook)
    int force_box;
    float force_y_min, force_width;
    int force_n_int;
    int fx_shift;            // fixed-point binary point of the spread (plan constant)
    // device memory
    fitsne::Params* params;
    float* box_partial;      // [kBoxBlocks * 2] min/max per block
    unsigned* tickets;       // [4] completion counters (self-resetting)
    int32_t* counts;         // [n_boxes_max] points per box (zero between iterations)
    int32_t* box_start;      // [n_boxes_max + 1]
    int32_t* cursor;         // [n_boxes_max] scatter cursors
    int32_t* chunk_start;    // [n_boxes_max + 1]
    int32_t* chunk_box;      // [chunk_cap]
    int32_t* block_pts;      // [scan_blocks] per-block totals then offsets
    int32_t* block_chunks;   // [scan_blocks]
    float* sorted_y;         // [N * s] coordinates grouped by box
    long long* w;            // [(s+1) * n_max^s] spread grids, fixed point 2^-fx_shift
    float2* spec;            // [4 * n_max * L_max] row spectra (s = 2)
    float4* hgrid;           // [n_max^s] node potentials
    double* z_partial;       // [L_max / 2 + 1] Parseval sums of Z per column pair
    double* kl_partial;      // [kl_blocks]
    double* kl_out_dev;      // [1]
    int32_t* valid_flag;     // [1]
    float* y_next;           // [N * s]
    float* uY_run;           // [N * s] (tsne_run state)
    float* gains_run;        // [N * s]
    fitsne::FftEntry* fft_table;
    float2* twiddles;
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
    unsigned long long* chunk_sum;  // [N / kForceChunk + 1]
    int32_t* chunk_centre;   // [N / kForceChunk + 1] window centre per 256-row chunk
    unsigned long long* sort_keys;  // [next_pow2(N)]
    int32_t* scan_bsum;      // [N / 2048 + 1]
    float* tmp_state;        // [N * s]
    float* y_cur;            // [N * s] run state Y in the relabelled order
    // host-buffer path (tsne_run_host), allocated on first use
    int64_t host_nnz_cap;
    int32_t* h_row_ptr;
    int32_t* h_col;
    float* h_val;
    float* h_Y;
};

namespace fitsne {

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
// Launchers (defined in the .cu files). All enqueue on plan->stream.
// ----------------------------------------------------------------------------
cudaError_t launch_box(tsne_plan* pl, const float* Y);
cudaError_t launch_sort_and_spread(tsne_plan* pl, const float* Y);
cudaError_t launch_convolution(tsne_plan* pl, double* Z_out);
cudaError_t launch_gradient(tsne_plan* pl, const tsne_csr& P, const float* Y, float alpha,
                            float* dY);
cudaError_t launch_step(tsne_plan* pl, const tsne_csr& P, const float* Y, float* Y_new,
                        float* uY, float* gains, float alpha, float momentum, float lr,
                        float min_gain, float gain_inc, float gain_dec);
// Relabels the run (state Y_cur, uY_cur, gains_cur in the current labels) and
// builds the relabelled P; the relabelled Y goes to Y_out, uY and gains are
// moved in place.
cudaError_t launch_relabel(tsne_plan* pl, const tsne_csr& P, const float* Y_cur, float* uY_cur,
                           float* gains_cur, float* Y_out);
// to_caller = 1: dst[perm[k]] = src[k]; 0: dst[k] = src[perm[k]].
cudaError_t launch_to_labels(tsne_plan* pl, const float* src, int to_caller, float* dst);
cudaError_t launch_kl(tsne_plan* pl, const tsne_csr& P, const float* Y);
// KL reduction with explicit scratch: 2 doubles per block in partial, a
// self-resetting completion counter, Z from Z_dev (device) or Z_val.
cudaError_t launch_kl_raw(const tsne_csr& P, const float* Y, int64_t N, int s,
                          const double* Z_dev, double Z_val, double* partial, unsigned* ticket,
                          double* out, int blocks, cudaStream_t stream);
cudaError_t launch_validate(tsne_plan* pl, const tsne_csr& P);
cudaError_t launch_fill(tsne_plan* pl, float* a, float v, int64_t n);
cudaError_t fft_configure(tsne_plan* pl);    // sets shared-memory limits
cudaError_t force_configure(tsne_plan* pl);  // shared-memory limit of the windowed force kernel

}  // namespace fitsne
