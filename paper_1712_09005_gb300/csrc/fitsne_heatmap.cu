// t-SNE heatmaps (Sec. 5): the cells' 1-D embedding is cut into n_bins
// equal-width bins over [min y, max y]; gene g becomes the vector
//   h_g[b] = sum over cells i in bin b of E[i, g]          (b = 0 .. n_bins - 1)
// and two genes are compared by the Euclidean distance |h_g - h_g'|. Each gene
// of interest is enriched with the genes nearest to it in that metric, and the
// vectors of that gene set are the rows of the heatmap.
//
//   hm_minmax_kernel    min and max of y, exact (order-preserving integer keys
//                       with atomicMin / atomicMax); flags a non-finite y
//   hm_bin_kernel       warp per cell: its bin (FP32, fixed rounding: the
//                       interval rule of the gradient's box), then
//                       H[b][g] += E[i, g] by FP64 atomics and the bin's cell
//                       count; flags a malformed row or a gene out of range
//                       (summing each bin's rows in a shared-memory copy of its
//                       row of H first, after a counting sort of the cells by
//                       bin, measured 2.3x slower at 50k cells x 25k genes)
//   hm_dist_kernel      thread per (gene of interest, gene): FP64 squared
//                       distance over the bins, in bin order
//   hm_select_kernel    block per (gene of interest, slice of 2048 genes): the
//                       slice's m smallest (distance, gene index), the gene
//                       itself excluded, by m rounds of a block arg-min
//   hm_merge_kernel     block per gene of interest: the m smallest of the
//                       slices' candidates (which hold the overall m smallest)
//
// H is summed by atomics, so its last bits may differ between calls (FP64
// rounding of a different summation order); bins, counts and every integer
// decision made from exact data are reproducible.
#include <float.h>
#include <limits.h>
#include <math.h>

#include <algorithm>

#include "fitsne_internal.cuh"

namespace fitsne {
namespace {

constexpr int kHmThreads = 256;
constexpr int kHmSlice = 2048;       // genes per first-stage selection block (8 per thread)
constexpr int kHmMaxM = 256;         // nearest genes per gene of interest
constexpr int kHmMaxBins = 1 << 20;

enum : int { kFlagNonFinite = 1, kFlagBadRow = 2, kFlagBadGene = 4 };

// Order-preserving map of FP32 onto unsigned integers (-0 sorts below +0).
__device__ __forceinline__ unsigned f2key(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key2f(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Bin width and its reciprocal from the range: width = (max - min) / n_bins
// and 1 / width, each rounded once in FP32; a zero or subnormal width (every
// y in one bin) gives inv_w = 0.
struct BinRule {
    float y_min, inv_w;
};
__device__ __forceinline__ BinRule bin_rule(const unsigned* minmax, int n_bins) {
    const float y_min = key2f(minmax[0]), y_max = key2f(minmax[1]);
    const float w = __fdiv_rn(__fsub_rn(y_max, y_min), (float)n_bins);
    float inv = 0.0f;
    if (w > 0.0f) {
        inv = __fdiv_rn(1.0f, w);
        if (!(inv <= FLT_MAX)) inv = 0.0f;
    }
    return BinRule{y_min, inv};
}
__device__ __forceinline__ int bin_of(float y, const BinRule& r, int n_bins) {
    const float t = __fmul_rn(__fsub_rn(y, r.y_min), r.inv_w);
    if (!(t >= 0.0f)) return 0;
    if (t >= (float)n_bins) return n_bins - 1;
    const int b = (int)floorf(t);
    return b < n_bins ? b : n_bins - 1;
}

__global__ void __launch_bounds__(kHmThreads)
hm_minmax_kernel(const float* __restrict__ y, int64_t N, unsigned* __restrict__ minmax,
                 int* __restrict__ flags) {
    __shared__ unsigned s_lo[kHmThreads / 32], s_hi[kHmThreads / 32];
    __shared__ int s_bad;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    unsigned lo = 0xffffffffu, hi = 0u;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = y[i];
        if (!(fabsf(v) <= FLT_MAX)) {
            bad = true;
            continue;
        }
        const unsigned k = f2key(v);
        lo = min(lo, k);
        hi = max(hi, k);
    }
    if (bad) s_bad = 1;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const int w = threadIdx.x / 32;
    if (threadIdx.x % 32 == 0) {
        s_lo[w] = lo;
        s_hi[w] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < kHmThreads / 32; ++k) {
            lo = min(lo, s_lo[k]);
            hi = max(hi, s_hi[k]);
        }
        atomicMin(&minmax[0], lo);
        atomicMax(&minmax[1], hi);
        if (s_bad) atomicOr(flags, kFlagNonFinite);
    }
}

__global__ void __launch_bounds__(kHmThreads)
hm_bin_kernel(const float* __restrict__ y, int64_t N, const int32_t* __restrict__ row_ptr,
              const int32_t* __restrict__ col, const float* __restrict__ val, int64_t nnz, int G,
              int n_bins, const unsigned* __restrict__ minmax, double* __restrict__ H,
              int32_t* __restrict__ count, int* __restrict__ flags) {
    const BinRule r = bin_rule(minmax, n_bins);
    const int lane = threadIdx.x % 32;
    const int64_t nwarp = (int64_t)gridDim.x * (blockDim.x / 32);
    int bad = 0;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; i < N; i += nwarp) {
        const float yi = y[i];
        if (!(fabsf(yi) <= FLT_MAX)) continue;  // flagged by the min/max pass
        const int b = bin_of(yi, r, n_bins);
        const int64_t beg = row_ptr[i], end = row_ptr[i + 1];
        if (beg < 0 || end < beg || end > nnz) {
            bad |= kFlagBadRow;
            continue;
        }
        if (lane == 0) atomicAdd(&count[b], 1);
        double* __restrict__ Hb = H + (int64_t)b * G;
        for (int64_t e = beg + lane; e < end; e += 32) {
            const int g = col[e];
            if ((unsigned)g >= (unsigned)G) {
                bad |= kFlagBadGene;
                continue;
            }
            atomicAdd(&Hb[g], (double)val[e]);
        }
    }
    if (bad) atomicOr(flags, bad);
}

__global__ void __launch_bounds__(kHmThreads)
hm_dist_kernel(const double* __restrict__ H, int G, int n_bins, const int32_t* __restrict__ goi,
               int n_goi, double* __restrict__ d2) {
    const int64_t total = (int64_t)n_goi * G;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(t / G), g = (int)(t - (int64_t)q * G);
        const int gq = goi[q];
        double acc = 0.0;
        for (int b = 0; b < n_bins; ++b) {
            const double d = H[(int64_t)b * G + gq] - H[(int64_t)b * G + g];
            acc += d * d;
        }
        d2[t] = acc;
    }
}

// (d, i) before (e, j): smaller distance, then smaller index
__device__ __forceinline__ bool pair_less(double d, int i, double e, int j) {
    return d < e || (d == e && i < j);
}

// Block-wide smallest (d, i) over the threads' (d, i); every thread gets it.
__device__ __forceinline__ void block_argmin(double& d, int& i, double* s_d, int* s_i) {
    const int lane = threadIdx.x % 32, w = threadIdx.x / 32;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const double od = __shfl_xor_sync(0xffffffffu, d, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (pair_less(od, oi, d, i)) {
            d = od;
            i = oi;
        }
    }
    if (lane == 0) {
        s_d[w] = d;
        s_i[w] = i;
    }
    __syncthreads();
    d = s_d[0];
    i = s_i[0];
    for (int k = 1; k < (int)(blockDim.x / 32); ++k)
        if (pair_less(s_d[k], s_i[k], d, i)) {
            d = s_d[k];
            i = s_i[k];
        }
    __syncthreads();
}

// Block (p, q): the m smallest (distance, gene) of genes [p kHmSlice,
// (p + 1) kHmSlice) for gene of interest q, held 8 per thread in registers;
// (inf, INT_MAX) marks "no more genes in the slice".
__global__ void __launch_bounds__(kHmThreads)
hm_select_kernel(const double* __restrict__ d2, int G, const int32_t* __restrict__ goi, int m, int P,
                 double* __restrict__ cand_d, int32_t* __restrict__ cand_i) {
    __shared__ double s_d[kHmThreads / 32];
    __shared__ int s_i[kHmThreads / 32];
    constexpr int K = kHmSlice / kHmThreads;
    const int p = blockIdx.x, q = blockIdx.y;
    const int gq = goi[q];
    double dv[K];
    int gv[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int g = p * kHmSlice + k * kHmThreads + threadIdx.x;
        dv[k] = INFINITY;
        gv[k] = INT_MAX;
        if (g < G && g != gq) {
            double d = d2[(int64_t)q * G + g];
            dv[k] = (d <= DBL_MAX) ? d : INFINITY;  // NaN ranks as +inf, by index
            gv[k] = g;
        }
    }
    double last_d = -INFINITY;
    int last_i = -1;
    for (int r = 0; r < m; ++r) {
        double bd = INFINITY;
        int bi = INT_MAX;
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (gv[k] != INT_MAX && pair_less(last_d, last_i, dv[k], gv[k]) && pair_less(dv[k], gv[k], bd, bi)) {
                bd = dv[k];
                bi = gv[k];
            }
        block_argmin(bd, bi, s_d, s_i);
        if (threadIdx.x == 0) {
            cand_d[((int64_t)q * P + p) * m + r] = bd;
            cand_i[((int64_t)q * P + p) * m + r] = bi;
        }
        last_d = bd;
        last_i = bi;
    }
}

__global__ void __launch_bounds__(kHmThreads)
hm_merge_kernel(const double* __restrict__ cand_d, const int32_t* __restrict__ cand_i, int P, int m,
                int32_t* __restrict__ out_idx, double* __restrict__ out_d) {
    __shared__ double s_d[kHmThreads / 32];
    __shared__ int s_i[kHmThreads / 32];
    const int q = blockIdx.x;
    const int C = P * m;
    const double* __restrict__ cd = cand_d + (int64_t)q * C;
    const int32_t* __restrict__ ci = cand_i + (int64_t)q * C;
    double last_d = -INFINITY;
    int last_i = -1;
    for (int r = 0; r < m; ++r) {
        double bd = INFINITY;
        int bi = INT_MAX;
        for (int c = threadIdx.x; c < C; c += blockDim.x) {
            const double d = cd[c];
            const int i = ci[c];
            if (i != INT_MAX && pair_less(last_d, last_i, d, i) && pair_less(d, i, bd, bi)) {
                bd = d;
                bi = i;
            }
        }
        block_argmin(bd, bi, s_d, s_i);
        if (threadIdx.x == 0) {
            out_idx[(int64_t)q * m + r] = bi;
            out_d[(int64_t)q * m + r] = sqrt(bd);
        }
        last_d = bd;
        last_i = bi;
    }
}

}  // namespace
}  // namespace fitsne

struct tsne_heatmap {
    int n_bins = 0, G = 0, max_goi = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    int slices = 0;                // first-stage selection blocks per gene of interest
    int* flags = nullptr;          // device: kFlag* bits of the last bin call
    unsigned* minmax = nullptr;    // device: order keys of min y, max y
    int32_t* goi = nullptr;        // device [max_goi]
    double* d2 = nullptr;          // device [max_goi x G]
    double* cand_d = nullptr;      // device [max_goi x slices x kHmMaxM]
    int32_t* cand_i = nullptr;
    int32_t* idx = nullptr;        // device [max_goi x kHmMaxM]
    double* dist = nullptr;        // device [max_goi x kHmMaxM]
    int64_t launches = 0;
    bool binned = false, searched = false;
    cudaEvent_t ev[6] = {};        // bin: 0..2, nearest: 3..5
};

namespace {

int hm_cuda_fail(cudaError_t e, const char* what) {
    return fitsne::set_error(TSNE_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define HCU(call, what)                                         \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return hm_cuda_fail(e_, what);   \
    } while (0)

void free_heatmap(tsne_heatmap* h) {
    if (!h) return;
    void* ps[] = {h->flags, h->minmax, h->goi, h->d2, h->cand_d, h->cand_i, h->idx, h->dist};
    for (void* p : ps)
        if (p) cudaFree(p);
    for (cudaEvent_t e : h->ev)
        if (e) cudaEventDestroy(e);
    delete h;
}

template <typename T>
int hm_alloc(T** p, size_t count, const char* what) {
    *p = nullptr;
    if (cudaMalloc((void**)p, (count ? count : 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fitsne::set_error(TSNE_ERR_OOM, "cudaMalloc of %zu bytes for %s failed", count * sizeof(T), what);
    }
    return TSNE_OK;
}

int hm_grid(int64_t items, int per_block, int sm_count) {
    const int64_t g = (items + per_block - 1) / per_block;
    const int64_t cap = 8LL * (sm_count > 0 ? sm_count : 1);
    return (int)std::max<int64_t>(1, std::min(g, cap));
}

}  // namespace

extern "C" {

int tsne_heatmap_create(int32_t n_bins, int32_t G, int32_t max_goi, void* stream, tsne_heatmap** out) {
    fitsne::clear_error();
    if (!out) return fitsne::set_error(TSNE_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_bins < 1 || n_bins > fitsne::kHmMaxBins)
        return fitsne::set_error(TSNE_ERR_INVALID_ARG, "n_bins = %d outside [1, %d]", n_bins, fitsne::kHmMaxBins);
    if (G < 1) return fitsne::set_error(TSNE_ERR_INVALID_ARG, "G = %d must be positive", G);
    if ((int64_t)n_bins * G > ((int64_t)1 << 40))
        return fitsne::set_error(TSNE_ERR_INVALID_ARG, "n_bins x G = %lld is too large", (long long)n_bins * G);
    if (max_goi < 1 || max_goi > 65535)
        return fitsne::set_error(TSNE_ERR_INVALID_ARG, "max_goi = %d outside [1, 65535]", max_goi);
    tsne_heatmap* h = new tsne_heatmap();
    h->n_bins = n_bins;
    h->G = G;
    h->max_goi = max_goi;
    h->stream = (cudaStream_t)stream;
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev);
    for (int e = 0; e < 6 && ce == cudaSuccess; ++e) ce = cudaEventCreate(&h->ev[e]);
    if (ce != cudaSuccess) {
        free_heatmap(h);
        return hm_cuda_fail(ce, "device setup");
    }
    h->slices = (G + fitsne::kHmSlice - 1) / fitsne::kHmSlice;
    const size_t nc = (size_t)max_goi * (size_t)h->slices * fitsne::kHmMaxM;
    int rc = hm_alloc(&h->flags, 1, "flags");
    if (!rc) rc = hm_alloc(&h->minmax, 2, "range");
    if (!rc) rc = hm_alloc(&h->goi, (size_t)max_goi, "genes of interest");
    if (!rc) rc = hm_alloc(&h->d2, (size_t)max_goi * (size_t)G, "distances");
    if (!rc) rc = hm_alloc(&h->cand_d, nc, "candidate distances");
    if (!rc) rc = hm_alloc(&h->cand_i, nc, "candidate genes");
    if (!rc) rc = hm_alloc(&h->idx, (size_t)max_goi * fitsne::kHmMaxM, "nearest genes");
    if (!rc) rc = hm_alloc(&h->dist, (size_t)max_goi * fitsne::kHmMaxM, "nearest distances");
    if (rc) {
        free_heatmap(h);
        return rc;
    }
    *out = h;
    return TSNE_OK;
}

int tsne_heatmap_destroy(tsne_heatmap* h) {
    fitsne::clear_error();
    if (!h) return TSNE_OK;
    cudaStreamSynchronize(h->stream);
    free_heatmap(h);
    return TSNE_OK;
}

int tsne_heatmap_bin(tsne_heatmap* h, const float* y, int64_t N, tsne_csr E, double* H, int32_t* bin_count) {
    fitsne::clear_error();
    if (!h) return fitsne::set_error(TSNE_ERR_INVALID_ARG, "heatmap object is NULL");
    if (!y || !H || !bin_count || !E.row_ptr || (E.nnz > 0 && (!E.col || !E.val)))
        return fitsne::set_error(TSNE_ERR_INVALID_ARG, "NULL pointer argument");
    if (N < 1 || N > INT32_MAX - 1) return fitsne::set_error(TSNE_ERR_INVALID_ARG, "N = %lld outside [1, 2^31 - 2]", (long long)N);
    if (E.nnz < 0 || E.nnz > INT32_MAX) return fitsne::set_error(TSNE_ERR_INVALID_ARG, "nnz = %lld outside [0, 2^31 - 1]", (long long)E.nnz);
    using namespace fitsne;
    cudaStream_t st = h->stream;
    h->binned = false;
    HCU(cudaEventRecord(h->ev[0], st), "event");
    HCU(cudaMemsetAsync(H, 0, sizeof(double) * (size_t)h->n_bins * (size_t)h->G, st), "clear H");
    HCU(cudaMemsetAsync(bin_count, 0, sizeof(int32_t) * (size_t)h->n_bins, st), "clear counts");
    HCU(cudaMemsetAsync(h->flags, 0, sizeof(int), st), "clear flags");
    HCU(cudaMemsetAsync(h->minmax, 0xff, sizeof(unsigned), st), "init min");
    HCU(cudaMemsetAsync(h->minmax + 1, 0, sizeof(unsigned), st), "init max");
    hm_minmax_kernel<<<hm_grid(N, kHmThreads, h->sm_count), kHmThreads, 0, st>>>(y, N, h->minmax, h->flags);
    HCU(cudaGetLastError(), "min/max launch");
    HCU(cudaEventRecord(h->ev[1], st), "event");
    hm_bin_kernel<<<hm_grid(32 * N, kHmThreads, 4 * h->sm_count), kHmThreads, 0, st>>>(
        y, N, E.row_ptr, E.col, E.val, E.nnz, h->G, h->n_bins, h->minmax, H, bin_count, h->flags);
    HCU(cudaGetLastError(), "bin launch");
    HCU(cudaEventRecord(h->ev[2], st), "event");
    h->launches += 2;
    int flags = 0;
    HCU(cudaMemcpyAsync(&flags, h->flags, sizeof(int), cudaMemcpyDeviceToHost, st), "read flags");
    HCU(cudaStreamSynchronize(st), "bin synchronise");
    h->binned = true;
    if (flags & kFlagNonFinite) return set_error(TSNE_ERR_NONFINITE, "non-finite coordinate in y");
    if (flags & kFlagBadRow) return set_error(TSNE_ERR_INVALID_ARG, "E.row_ptr is not a valid CSR row table");
    if (flags & kFlagBadGene) return set_error(TSNE_ERR_INVALID_ARG, "a gene index in E.col is outside [0, G)");
    return TSNE_OK;
}

int tsne_heatmap_nearest(tsne_heatmap* h, const double* H, const int32_t* goi_host, int32_t n_goi, int32_t m,
                         int32_t* idx_host, double* dist_host) {
    fitsne::clear_error();
    if (!h) return fitsne::set_error(TSNE_ERR_INVALID_ARG, "heatmap object is NULL");
    if (!H || !goi_host || !idx_host || !dist_host) return fitsne::set_error(TSNE_ERR_INVALID_ARG, "NULL pointer argument");
    if (n_goi < 1 || n_goi > h->max_goi)
        return fitsne::set_error(TSNE_ERR_INVALID_ARG, "n_goi = %d outside [1, %d]", n_goi, h->max_goi);
    if (m < 1 || m > fitsne::kHmMaxM || m > h->G - 1)
        return fitsne::set_error(TSNE_ERR_INVALID_ARG, "m = %d outside [1, min(%d, G - 1)]", m, fitsne::kHmMaxM);
    for (int q = 0; q < n_goi; ++q)
        if (goi_host[q] < 0 || goi_host[q] >= h->G)
            return fitsne::set_error(TSNE_ERR_INVALID_ARG, "gene of interest %d outside [0, %d)", goi_host[q], h->G);
    using namespace fitsne;
    cudaStream_t st = h->stream;
    h->searched = false;
    HCU(cudaEventRecord(h->ev[3], st), "event");
    HCU(cudaMemcpyAsync(h->goi, goi_host, sizeof(int32_t) * n_goi, cudaMemcpyHostToDevice, st), "upload genes");
    hm_dist_kernel<<<hm_grid((int64_t)n_goi * h->G, kHmThreads, 4 * h->sm_count), kHmThreads, 0, st>>>(
        H, h->G, h->n_bins, h->goi, n_goi, h->d2);
    HCU(cudaGetLastError(), "distance launch");
    HCU(cudaEventRecord(h->ev[4], st), "event");
    hm_select_kernel<<<dim3(h->slices, n_goi), kHmThreads, 0, st>>>(h->d2, h->G, h->goi, m, h->slices,
                                                                      h->cand_d, h->cand_i);
    hm_merge_kernel<<<n_goi, kHmThreads, 0, st>>>(h->cand_d, h->cand_i, h->slices, m, h->idx, h->dist);
    HCU(cudaGetLastError(), "selection launch");
    HCU(cudaEventRecord(h->ev[5], st), "event");
    h->launches += 3;
    HCU(cudaMemcpyAsync(idx_host, h->idx, sizeof(int32_t) * (size_t)n_goi * m, cudaMemcpyDeviceToHost, st),
        "download genes");
    HCU(cudaMemcpyAsync(dist_host, h->dist, sizeof(double) * (size_t)n_goi * m, cudaMemcpyDeviceToHost, st),
        "download distances");
    HCU(cudaStreamSynchronize(st), "nearest synchronise");
    h->searched = true;
    return TSNE_OK;
}

int tsne_heatmap_phase_ms(const tsne_heatmap* h, double* ms_out) {
    fitsne::clear_error();
    if (!h || !ms_out) return fitsne::set_error(TSNE_ERR_INVALID_ARG, "NULL argument");
    if (!h->binned) return fitsne::set_error(TSNE_ERR_INVALID_ARG, "no bin call has completed");
    float a = 0.0f, b = 0.0f, c = 0.0f, d = 0.0f;
    HCU(cudaEventElapsedTime(&a, h->ev[0], h->ev[1]), "event time");
    HCU(cudaEventElapsedTime(&b, h->ev[1], h->ev[2]), "event time");
    if (h->searched) {
        HCU(cudaEventElapsedTime(&c, h->ev[3], h->ev[4]), "event time");
        HCU(cudaEventElapsedTime(&d, h->ev[4], h->ev[5]), "event time");
    }
    ms_out[0] = a;
    ms_out[1] = b;
    ms_out[2] = c;
    ms_out[3] = d;
    return TSNE_OK;
}

int64_t tsne_heatmap_launch_count(const tsne_heatmap* h) { return h ? h->launches : 0; }

}  // extern "C"
