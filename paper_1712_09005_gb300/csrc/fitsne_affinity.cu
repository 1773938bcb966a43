// Input affinities P on the GPU (Sec. 1.1, Eq. p_ij, restricted to the k
// exact nearest neighbours as in Sec. 3):
//   p_{j|i} = exp(-beta_i |x_i - x_j|^2) / sum_{l in kNN(i)} exp(-beta_i |x_i - x_l|^2),
//   beta_i by bisection so that exp(H(P_i)) = perplexity (natural log),
//   p_ij = (p_{j|i} + p_{i|j}) / (2N), symmetric CSR with sorted columns.
//
//   knn_kernel        exact kNN, FP32 squared distances in difference form
//                     (no cancellation); candidates streamed through shared
//                     memory; each warp keeps the sorted top-k of 4 queries
//                     (ties by the smaller index, as the oracle breaks them)
//   calibrate_kernel  warp per row, FP64 bisection on beta (the oracle's rule:
//                     start 1, double / halve while a side is open, else the
//                     midpoint; stop at |H - log perplexity| < 1e-5 or 200 steps)
//   radix kernels     stable LSD sort of the kNN edges (i -> j) by j: the
//                     edges into each j, in increasing i
//   symmetrise        per row the union of its out-list (sorted by column)
//                     and in-list (sorted by source) by co-ranking, values
//                     (p_{j|i} + p_{i|j}) / 2N in FP64 rounded once to FP32
// Every step is deterministic.
#include <limits.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "fitsne_internal.cuh"

namespace fitsne {

namespace {

constexpr unsigned kFullA = 0xffffffffu;
constexpr int kKnnTile = 128;     // candidates per shared-memory tile
constexpr int kKnnQ = 8;          // queries per warp
constexpr int kKnnWarps = 8;      // warps per CTA
constexpr int kKnnDMax = 64;      // largest input dimension
constexpr int kKnnKMax = 256;     // largest k
constexpr int kRadixTile = 4096;  // items per radix-sort block
constexpr int kRadixThreads = 256;

// Shared-memory row stride in floats: a multiple of 4 (float4 reads) with an
// odd number of float4s, so 8 lanes reading 8 consecutive rows hit 8
// disjoint groups of 4 banks.
__host__ __device__ __forceinline__ int knn_stride(int D) {
    int Ds = (D + 3) / 4 * 4;
    if ((Ds / 4) % 2 == 0) Ds += 4;
    return Ds;
}

__host__ __forceinline__ size_t knn_smem_bytes(int D, int k) {
    const size_t Ds = (size_t)knn_stride(D);
    return sizeof(float) * (kKnnTile * Ds + (size_t)kKnnWarps * kKnnQ * Ds) +
           (sizeof(float) + sizeof(int)) * (size_t)kKnnWarps * kKnnQ * k;
}

// (d, idx) lexicographic order: the kNN order of the oracle (stable sort of
// distances by index).
__device__ __forceinline__ bool knn_less(float d, int i, float e, int j) {
    return d < e || (d == e && i < j);
}

// Inserts (d, i) into the sorted list (ld, li) of k entries held in shared
// memory by the warp (lane-strided), dropping the last entry.
__device__ __forceinline__ void knn_insert(float* ld, int* li, int k, float d, int i, int lane) {
    // position = entries strictly before (d, i)
    int pos = 0;
    for (int m = lane; m < k; m += 32) pos += knn_less(ld[m], li[m], d, i) ? 1 : 0;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) pos += __shfl_xor_sync(kFullA, pos, o);
    // shift [pos, k - 1) right by one (read all, then write)
    float vd[kKnnKMax / 32];
    int vi[kKnnKMax / 32];
#pragma unroll
    for (int t = 0; t < kKnnKMax / 32; ++t) {
        const int m = lane + 32 * t;
        vd[t] = (m < k) ? ld[m] : 0.0f;
        vi[t] = (m < k) ? li[m] : 0;
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < kKnnKMax / 32; ++t) {
        const int m = lane + 32 * t;
        if (m >= pos && m + 1 < k) {
            ld[m + 1] = vd[t];
            li[m + 1] = vi[t];
        }
    }
    if (lane == 0 && pos < k) {
        ld[pos] = d;
        li[pos] = i;
    }
    __syncwarp();
}

}  // namespace

// Exact k nearest neighbours of queries [q0, q0 + nq) among all N points
// (self excluded). X is N x D row-major. Output sorted by (d^2, index).
// With kList the queries are qlist[q0 .. q0 + nq) instead (the queries the
// tensor-core kNN leaves to this kernel).
template <bool kList>
__global__ void __launch_bounds__(kKnnWarps * 32)
knn_kernel(const float* __restrict__ X, int64_t N, int D, int k, int64_t q0, int64_t nq,
           int32_t* __restrict__ out_idx, float* __restrict__ out_d2, const int32_t* __restrict__ qlist) {
    extern __shared__ float sm[];
    __shared__ int64_t s_id[kKnnWarps * kKnnQ];  // query of each slot (kList), -1 past the end
    const int Ds = knn_stride(D);
    float* s_c = sm;                                     // [kKnnTile][Ds]
    float* s_q = s_c + kKnnTile * Ds;                    // [kKnnWarps * kKnnQ][Ds]
    float* s_ld = s_q + kKnnWarps * kKnnQ * Ds;          // [kKnnWarps * kKnnQ][k]
    int* s_li = reinterpret_cast<int*>(s_ld + kKnnWarps * kKnnQ * k);
    const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
    const int64_t nqb = (nq + kKnnWarps * kKnnQ - 1) / (kKnnWarps * kKnnQ);
    for (int64_t qb = blockIdx.x; qb < nqb; qb += gridDim.x) {
        const int64_t qbase = q0 + qb * kKnnWarps * kKnnQ;
        __syncthreads();
        if (kList && threadIdx.x < kKnnWarps * kKnnQ) {
            const int64_t p = qbase + threadIdx.x;
            s_id[threadIdx.x] = p < q0 + nq ? (int64_t)qlist[p] : -1;
        }
        if (kList) __syncthreads();
        for (int t = threadIdx.x; t < kKnnWarps * kKnnQ * Ds; t += blockDim.x) {
            const int q = t / Ds, d = t - q * Ds;
            const int64_t p = qbase + q;
            const int64_t gq = kList ? s_id[q] : p;
            s_q[t] = (d < D && p < q0 + nq) ? X[gq * D + d] : 0.0f;
        }
        for (int t = threadIdx.x; t < kKnnWarps * kKnnQ * k; t += blockDim.x) {
            s_ld[t] = INFINITY;
            s_li[t] = INT_MAX;
        }
        float thr[kKnnQ];
        int thi[kKnnQ];
#pragma unroll
        for (int u = 0; u < kKnnQ; ++u) { thr[u] = INFINITY; thi[u] = INT_MAX; }
        for (int64_t c0 = 0; c0 < N; c0 += kKnnTile) {
            __syncthreads();
            for (int t = threadIdx.x; t < kKnnTile * Ds; t += blockDim.x) {
                const int c = t / Ds, d = t - c * Ds;
                const int64_t gc = c0 + c;
                s_c[t] = (d < D && gc < N) ? X[gc * D + d] : 0.0f;
            }
            __syncthreads();
            for (int cc = lane; cc < kKnnTile; cc += 32) {
                const int64_t gc = c0 + cc;
                float acc[kKnnQ];
#pragma unroll
                for (int u = 0; u < kKnnQ; ++u) acc[u] = 0.0f;
                const float4* cv = reinterpret_cast<const float4*>(s_c + cc * Ds);
                for (int d4 = 0; d4 < Ds / 4; ++d4) {
                    const float4 c = cv[d4];
#pragma unroll
                    for (int u = 0; u < kKnnQ; ++u) {
                        const float4 q = reinterpret_cast<const float4*>(s_q + (wid * kKnnQ + u) * Ds)[d4];
                        const float a = q.x - c.x, b = q.y - c.y, e = q.z - c.z, f = q.w - c.w;
                        acc[u] = fmaf(a, a, acc[u]);
                        acc[u] = fmaf(b, b, acc[u]);
                        acc[u] = fmaf(e, e, acc[u]);
                        acc[u] = fmaf(f, f, acc[u]);
                    }
                }
#pragma unroll
                for (int u = 0; u < kKnnQ; ++u) {
                    // a non-finite distance ranks as +inf (by index among
                    // equals), so every list fills with valid indices
                    if (!(acc[u] <= 3.402823466e38f)) acc[u] = INFINITY;
                    const int64_t p = qbase + wid * kKnnQ + u;
                    const int64_t gq = kList ? s_id[wid * kKnnQ + u] : p;
                    const bool ok = gc < N && p < q0 + nq && gc != gq;
                    const int ci = (int)gc;
                    const bool take = ok && knn_less(acc[u], ci, thr[u], thi[u]);
                    unsigned m = __ballot_sync(kFullA, take);
                    float* ld = s_ld + (wid * kKnnQ + u) * k;
                    int* li = s_li + (wid * kKnnQ + u) * k;
                    while (m) {
                        const int src = __ffs(m) - 1;
                        m &= m - 1;
                        const float d = __shfl_sync(kFullA, acc[u], src);
                        const int i = __shfl_sync(kFullA, ci, src);
                        if (knn_less(d, i, thr[u], thi[u])) {
                            knn_insert(ld, li, k, d, i, lane);
                            thr[u] = ld[k - 1];
                            thi[u] = li[k - 1];
                        }
                    }
                }
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < kKnnWarps * kKnnQ * k; t += blockDim.x) {
            const int q = t / k, m = t - q * k;
            const int64_t p = qbase + q;
            const int64_t gq = kList ? s_id[q] : p;
            if (p < q0 + nq) {
                out_idx[gq * k + m] = s_li[t];
                out_d2[gq * k + m] = s_ld[t];
            }
        }
    }
}

// ---- register-tiled kNN over the transposed data ----
//
// Xt is D x Np (Np = N rounded up to kTileC, zero past N). A CTA owns kTileQ
// queries; 128-candidate tiles stream through a double-buffered shared
// buffer by 16-byte cp.async. Thread (ty, tx) of the 16 x 16 grid holds the
// 4 x 8 distances of queries 4 ty .. 4 ty + 3 and candidates 4 tx .. 4 tx + 3,
// 64 + 4 tx .. 64 + 4 tx + 3, accumulated over d in order (the same sums as
// knn_kernel). The tile of distances goes to shared memory; warp w then
// filters queries 8 w .. 8 w + 7 against their current k-th entry and
// inserts the survivors into the sorted lists.
constexpr int kTileQ = 64;
constexpr int kTileC = 128;
// Smallest N for which the tiled kernel is chosen by default. Its selection
// (sorted insertions between two barriers, 8 warps per SM) costs about the
// same per query at any N, while the distances cost O(N) per query, so the
// row kernel (16 warps per SM hide the insertions) wins on small N.
#ifndef FITSNE_KNN_TC_MIN_N
#define FITSNE_KNN_TC_MIN_N 0  // faster than the row kernel from N = 2,000 (0.42 against 1.52 ms) up
#endif
#ifndef FITSNE_KNN_TILED_MIN_N
#define FITSNE_KNN_TILED_MIN_N 400000
#endif
constexpr int kTiledThreads = 256;
constexpr int kDistStride = kTileC + 4;

__host__ __forceinline__ size_t knn_tiled_smem_bytes(int D, int k) {
    return sizeof(float) * ((size_t)D * kTileQ + 2 * (size_t)D * kTileC + (size_t)kTileQ * kDistStride) +
           (sizeof(float) + sizeof(int)) * (size_t)kTileQ * k;
}

__global__ void transpose_pad_kernel(const float* __restrict__ X, int64_t N, int D, int64_t Np,
                                     float* __restrict__ Xt) {
    const int64_t total = (int64_t)D * Np;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = e / Np, n = e - d * Np;
        Xt[e] = n < N ? X[n * D + d] : 0.0f;
    }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int NPEND>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(NPEND) : "memory");
}

// copies rows d = 0..D-1 of Xt[:, n0 .. n0 + W) into dst[d][0 .. W) (W floats per row)
template <int W>
__device__ __forceinline__ void load_cols(float* dst, const float* __restrict__ Xt, int64_t Np, int D,
                                          int64_t n0) {
    constexpr int V = W / 4;  // float4 per row
    for (int t = threadIdx.x; t < D * V; t += kTiledThreads) {
        const int d = t / V, v = t - d * V;
        cp_async16(dst + d * W + 4 * v, Xt + (int64_t)d * Np + n0 + 4 * v);
    }
}

__global__ void __launch_bounds__(kTiledThreads, 1)
knn_tiled_kernel(const float* __restrict__ Xt, int64_t N, int64_t Np, int D, int k,
                 int32_t* __restrict__ out_idx, float* __restrict__ out_d2) {
    extern __shared__ __align__(16) float sm_t[];
    float* s_q = sm_t;                                // [D][kTileQ]
    float* s_c = s_q + D * kTileQ;                    // [2][D][kTileC]
    float* s_d = s_c + 2 * D * kTileC;                // [kTileQ][kDistStride]
    float* s_ld = s_d + kTileQ * kDistStride;         // [kTileQ][k]
    int* s_li = reinterpret_cast<int*>(s_ld + kTileQ * k);
    const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t nqb = (N + kTileQ - 1) / kTileQ;
    const int64_t ntiles = Np / kTileC;
    for (int64_t qb = blockIdx.x; qb < nqb; qb += gridDim.x) {
        const int64_t q0 = qb * kTileQ;
        __syncthreads();  // the previous block's lists are written out
        for (int t = threadIdx.x; t < kTileQ * k; t += kTiledThreads) {
            s_ld[t] = INFINITY;
            s_li[t] = INT_MAX;
        }
        float thr[8];
        int thi[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) { thr[u] = INFINITY; thi[u] = INT_MAX; }
        load_cols<kTileQ>(s_q, Xt, Np, D, q0);
        load_cols<kTileC>(s_c, Xt, Np, D, 0);
        cp_async_commit();
        for (int64_t tile = 0; tile < ntiles; ++tile) {
            const int b = (int)(tile & 1);
            if (tile + 1 < ntiles) load_cols<kTileC>(s_c + (b ^ 1) * D * kTileC, Xt, Np, D, (tile + 1) * kTileC);
            cp_async_commit();
            cp_async_wait<1>();
            __syncthreads();
            // 4 x 8 distances of this thread
            float acc[4][8];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
            const float* cb = s_c + b * D * kTileC;
#pragma unroll 2
            for (int d = 0; d < D; ++d) {
                const float4 a = *reinterpret_cast<const float4*>(s_q + d * kTileQ + 4 * ty);
                const float4 c0 = *reinterpret_cast<const float4*>(cb + d * kTileC + 4 * tx);
                const float4 c1 = *reinterpret_cast<const float4*>(cb + d * kTileC + 64 + 4 * tx);
                const float qa[4] = {a.x, a.y, a.z, a.w};
                const float cc[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float t = qa[i] - cc[j];
                        acc[i][j] = fmaf(t, t, acc[i][j]);
                    }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float* row = s_d + (4 * ty + i) * kDistStride;
                *reinterpret_cast<float4*>(row + 4 * tx) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
                *reinterpret_cast<float4*>(row + 64 + 4 * tx) =
                    make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
            }
            __syncthreads();
            // selection: warp wid owns queries 8 wid .. 8 wid + 7
            const int64_t c_base = tile * kTileC;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int ql = 8 * wid + u;
                const int64_t gq = q0 + ql;
                const float4 v = *reinterpret_cast<const float4*>(s_d + ql * kDistStride + 4 * lane);
                const float dv[4] = {v.x, v.y, v.z, v.w};
                float* ld = s_ld + ql * k;
                int* li = s_li + ql * k;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int64_t gc = c_base + 4 * lane + t;
                    float dd = dv[t];
                    // a non-finite distance ranks as +inf (by index among equals)
                    if (!(dd <= 3.402823466e38f)) dd = INFINITY;
                    const int ci = (int)gc;
                    const bool take = gq < N && gc < N && gc != gq && knn_less(dd, ci, thr[u], thi[u]);
                    unsigned m = __ballot_sync(kFullA, take);
                    while (m) {
                        const int src = __ffs(m) - 1;
                        m &= m - 1;
                        const float d = __shfl_sync(kFullA, dd, src);
                        const int i = __shfl_sync(kFullA, ci, src);
                        if (knn_less(d, i, thr[u], thi[u])) {
                            knn_insert(ld, li, k, d, i, lane);
                            thr[u] = ld[k - 1];
                            thi[u] = li[k - 1];
                        }
                    }
                }
            }
        }
        cp_async_wait<0>();
        __syncthreads();
        for (int t = threadIdx.x; t < kTileQ * k; t += kTiledThreads) {
            const int q = t / k, m = t - q * k;
            const int64_t gq = q0 + q;
            if (gq < N) {
                out_idx[gq * k + m] = s_li[t];
                out_d2[gq * k + m] = s_ld[t];
            }
        }
    }
}

// Bisection on beta per row (warp per row), FP64, the oracle's rule; writes
// p_{j|i} (FP64) over the row's k neighbours.
//
// Each step first evaluates H in FP32 (exponentials, sums, logarithm); only
// when that value lies within 1e-5 + kCalibSlack of the target does the step
// evaluate H in FP64 as above. kCalibSlack bounds |H_fp32 - H_fp64|: the
// exponent -beta x_j carries 3 roundings (beta, x_j, the product) and expf 2
// units, so each term e_j errs by at most e_j (|t_j| 1.8e-7 + 2.4e-7) with
// t_j = beta x_j; summed over k <= 256 terms (e_0 = 1 bounds S from below)
// log S errs by at most 6.4e-5 and beta mu by 4e-5 + 5.5 x 6.4e-5; the FP32
// sums (256 terms) add 1.6e-5 each; about 5e-4 in all, and the slack keeps a
// factor 4 over it. So every decision (stop, sharpen, flatten) is the one the
// FP64 evaluation takes: the same path, the same beta, the same p_{j|i} bit
// for bit, with FP64 only in the last steps. exact_only: FP64 at every step.
constexpr double kCalibSlack = 2e-3;

__global__ void calibrate_kernel(const float* __restrict__ d2, int64_t N, int k, double target,
                                 double* __restrict__ pc, int exact_only) {
    const int lane = threadIdx.x % 32;
    const int64_t nwarp = (int64_t)gridDim.x * blockDim.x / 32;
    constexpr int V = kKnnKMax / 32;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; i < N; i += nwarp) {
        const float* row = d2 + i * k;
        const double dmin = (double)row[0];  // the list is sorted: row[0] is the smallest
        double x[V];
        float xf[V];
#pragma unroll
        for (int t = 0; t < V; ++t) {
            const int m = lane + 32 * t;
            x[t] = m < k ? (double)row[m] - dmin : 0.0;
            xf[t] = (float)x[t];
        }
        double beta = 1.0, lo = -INFINITY, hi = INFINITY;
        for (int it = 0; it < 200; ++it) {
            double H = NAN;
            if (!exact_only) {
                const float bf = (float)beta;
                float Sf = 0.0f, Wf = 0.0f;
#pragma unroll
                for (int t = 0; t < V; ++t) {
                    if (lane + 32 * t < k) {
                        const float e = expf(-bf * xf[t]);
                        Sf += e;
                        Wf += e > 0.0f ? e * xf[t] : 0.0f;
                    }
                }
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) {
                    Sf += __shfl_xor_sync(kFullA, Sf, o);
                    Wf += __shfl_xor_sync(kFullA, Wf, o);
                }
                H = (double)(logf(Sf) + bf * (Wf / Sf));
            }
            if (!(fabs(H - target) > 1e-5 + kCalibSlack)) {  // near the target (or NaN): FP64
                double S = 0.0, W = 0.0;
#pragma unroll
                for (int t = 0; t < V; ++t) {
                    if (lane + 32 * t < k) {
                        const double e = exp(-beta * x[t]);
                        S += e;
                        W += e > 0.0 ? e * x[t] : 0.0;  // x = inf: no 0 * inf
                    }
                }
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) {
                    S += __shfl_xor_sync(kFullA, S, o);
                    W += __shfl_xor_sync(kFullA, W, o);
                }
                // every lane holds the same sums: one lane takes the logarithm
                if (lane == 0) H = log(S) + beta * (W / S);
                H = __shfl_sync(kFullA, H, 0);
            }
            if (fabs(H - target) < 1e-5) break;
            if (H > target) {  // too flat: sharpen
                lo = beta;
                beta = isinf(hi) ? beta * 2.0 : (beta + hi) * 0.5;
            } else {
                hi = beta;
                beta = isinf(lo) ? beta * 0.5 : (beta + lo) * 0.5;
            }
        }
        double S = 0.0;
        double e[V];
#pragma unroll
        for (int t = 0; t < V; ++t) {
            e[t] = (lane + 32 * t < k) ? exp(-beta * x[t]) : 0.0;
            S += e[t];
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) S += __shfl_xor_sync(kFullA, S, o);
#pragma unroll
        for (int t = 0; t < V; ++t)
            if (lane + 32 * t < k) pc[i * k + lane + 32 * t] = e[t] / S;
    }
}

// ---- stable LSD radix sort of (key, item) pairs by key, 8 bits per pass ----

// Per tile digit counts, digit-major: counts[digit * nblocks + block].
__global__ void __launch_bounds__(kRadixThreads)
radix_count_kernel(const uint32_t* __restrict__ keys, int64_t n, int shift,
                   uint32_t* __restrict__ counts, int nblocks) {
    __shared__ uint32_t h[256];
    for (int b = blockIdx.x; b < nblocks; b += gridDim.x) {
        __syncthreads();
        h[threadIdx.x] = 0;
        __syncthreads();
        const int64_t e0 = (int64_t)b * kRadixTile;
        for (int t = threadIdx.x; t < kRadixTile; t += blockDim.x) {
            const int64_t e = e0 + t;
            if (e < n) atomicAdd(&h[(keys[e] >> shift) & 255u], 1u);
        }
        __syncthreads();
        counts[(int64_t)threadIdx.x * nblocks + b] = h[threadIdx.x];
    }
}

// Exclusive scan of n values in place (one CTA of 1024 threads, chunked).
__global__ void __launch_bounds__(1024) scan_inplace_kernel(uint32_t* __restrict__ a, int64_t n) {
    __shared__ uint32_t sw[32];
    __shared__ uint32_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
    for (int64_t base = 0; base < n; base += 4 * 1024) {
        uint32_t v[4], sum = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t e = base + threadIdx.x * 4 + q;
            v[q] = e < n ? a[e] : 0u;
            sum += v[q];
        }
        uint32_t x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFullA, x, o);
            if (lane >= o) x += y;
        }
        __syncthreads();
        if (lane == 31) sw[wid] = x;
        __syncthreads();
        if (wid == 0) {
            uint32_t t = sw[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(kFullA, t, o);
                if (lane >= o) t += y;
            }
            sw[lane] = t;
        }
        __syncthreads();
        uint32_t run = s_carry + x - sum + (wid ? sw[wid - 1] : 0u);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t e = base + threadIdx.x * 4 + q;
            if (e < n) a[e] = run;
            run += v[q];
        }
        __syncthreads();
        if (threadIdx.x == 0) s_carry += sw[31];
    }
}

// Places each item at its digit's offset for the block plus its stable rank
// within the block (items are visited in order, 256 at a time; in a warp the
// rank among equal digits comes from match_any; across the warps of a chunk,
// per-digit counts are scanned in warp order).
__global__ void __launch_bounds__(kRadixThreads)
radix_scatter_kernel(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ items,
                     int64_t n, int shift, const uint32_t* __restrict__ offsets, int nblocks,
                     uint32_t* __restrict__ keys_out, uint32_t* __restrict__ items_out) {
    __shared__ uint32_t run[256];
    __shared__ uint32_t wcnt[kRadixThreads / 32][256];
    const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
    const unsigned lt = (1u << lane) - 1u;
    for (int b = blockIdx.x; b < nblocks; b += gridDim.x) {
        __syncthreads();
        run[threadIdx.x] = offsets[(int64_t)threadIdx.x * nblocks + b];
        const int64_t e0 = (int64_t)b * kRadixTile;
        for (int c = 0; c < kRadixTile; c += kRadixThreads) {
            for (int t = threadIdx.x; t < (kRadixThreads / 32) * 256; t += blockDim.x)
                (&wcnt[0][0])[t] = 0;
            __syncthreads();
            const int64_t e = e0 + c + threadIdx.x;
            const bool in = e < n;
            const uint32_t key = in ? keys[e] : 0u;
            const uint32_t item = in ? items[e] : 0u;
            const int dg = in ? (int)((key >> shift) & 255u) : 256;
            const unsigned peers = __match_any_sync(kFullA, dg);
            const int rank_w = __popc(peers & lt);
            if (in && rank_w == 0) wcnt[wid][dg] = __popc(peers);
            __syncthreads();
            if (in) {
                uint32_t before = 0;
                for (int w = 0; w < wid; ++w) before += wcnt[w][dg];
                const uint32_t pos = run[dg] + before + rank_w;
                keys_out[pos] = key;
                items_out[pos] = item;
            }
            __syncthreads();
            // advance the running offsets by this chunk's counts
            {
                const int d = threadIdx.x;
                uint32_t tot = 0;
                for (int w = 0; w < kRadixThreads / 32; ++w) tot += wcnt[w][d];
                run[d] += tot;
            }
            __syncthreads();
        }
    }
}

// ---- symmetrisation ----

__global__ void edge_keys_kernel(const int32_t* __restrict__ knn_idx, int64_t nk,
                                 uint32_t* __restrict__ keys, uint32_t* __restrict__ items) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nk;
         e += (int64_t)gridDim.x * blockDim.x) {
        keys[e] = (uint32_t)knn_idx[e];  // target j
        items[e] = (uint32_t)e;          // edge id = i * k + m
    }
}

// in_ptr[j] = first sorted edge whose target is j (keys sorted): binary search
__global__ void in_ptr_kernel(const uint32_t* __restrict__ sorted_keys, int64_t nk, int64_t N,
                              int32_t* __restrict__ in_ptr) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= N;
         j += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = nk;
        while (lo < hi) {
            const int64_t mid = (lo + hi) / 2;
            if ((int64_t)sorted_keys[mid] < j) lo = mid + 1;
            else hi = mid;
        }
        in_ptr[j] = (int32_t)lo;
    }
}

// Per row i (warp): its out-list O sorted by column (bitonic in shared
// memory, k <= 256) and its in-list I (edges into i, sources increasing,
// from the stable sort). flag[m] = O[m] is also in I; F[m] = flags before m.
// Pass 0 writes the union's size k + |I| - F[k]; pass 1 writes the union in
// column order by co-ranking:
//   out-entry O[m] = j      -> m + #{s in I : s < j} - F[m]
//   in-only entry I[t] = s  -> #{o in O : o < s} + t - F[#{o in O : o < s}]
__global__ void __launch_bounds__(256)
symmetrise_kernel(const int32_t* __restrict__ knn_idx, const double* __restrict__ pc, int64_t N,
                  int k, const int32_t* __restrict__ in_ptr, const uint32_t* __restrict__ in_edge,
                  int pass, int32_t* __restrict__ row_len, const int32_t* __restrict__ row_ptr,
                  int32_t* __restrict__ col, float* __restrict__ val) {
    __shared__ int s_col[8][kKnnKMax];
    __shared__ double s_val[8][kKnnKMax];
    __shared__ int s_in[8][kKnnKMax];   // per out-entry: position in I, or -1
    __shared__ int s_F[8][kKnnKMax + 1];
    const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
    const int64_t nwarp = (int64_t)gridDim.x * blockDim.x / 32;
    const double inv2n = 1.0 / (2.0 * (double)N);
    int* oc = s_col[wid];
    double* ov = s_val[wid];
    int* oin = s_in[wid];
    int* F = s_F[wid];
    const uint32_t uk = (uint32_t)k;
    int M = 1;
    while (M < k) M <<= 1;
    const int V = (k + 31) / 32;  // contiguous out-entries per lane for the prefix
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; i < N; i += nwarp) {
        for (int m = lane; m < M; m += 32) {
            oc[m] = m < k ? knn_idx[i * k + m] : INT_MAX;
            ov[m] = m < k ? pc[i * k + m] : 0.0;
        }
        __syncwarp();
        for (int kk = 2; kk <= M; kk <<= 1)
            for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                for (int a = lane; a < M; a += 32) {
                    const int b = a ^ jj;
                    if (b > a) {
                        const bool up = (a & kk) == 0;
                        if ((oc[a] > oc[b]) == up) {
                            const int tc = oc[a]; oc[a] = oc[b]; oc[b] = tc;
                            const double tv = ov[a]; ov[a] = ov[b]; ov[b] = tv;
                        }
                    }
                }
                __syncwarp();
            }
        const int i0 = in_ptr[i], nin = in_ptr[i + 1] - i0;
        const uint32_t* ie = in_edge + i0;
        // flags and in-positions of the out-entries
        for (int m = lane; m < k; m += 32) {
            const int j = oc[m];
            int lo = 0, hi = nin;
            while (lo < hi) {
                const int mid = (lo + hi) / 2;
                if ((int)(ie[mid] / uk) < j) lo = mid + 1;
                else hi = mid;
            }
            oin[m] = (lo < nin && (int)(ie[lo] / uk) == j) ? lo : -1;
        }
        __syncwarp();
        // F = exclusive prefix of the flags (lane owns [lane V, lane V + V))
        int cnt = 0;
        for (int q = 0; q < V; ++q) {
            const int m = lane * V + q;
            cnt += (m < k && oin[m] >= 0) ? 1 : 0;
        }
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFullA, incl, o);
            if (lane >= o) incl += y;
        }
        int run = incl - cnt;
        for (int q = 0; q < V; ++q) {
            const int m = lane * V + q;
            if (m < k) {
                F[m] = run;
                run += oin[m] >= 0 ? 1 : 0;
            }
        }
        if (lane == 31) F[k] = incl;
        __syncwarp();
        const int matched = F[k];
        if (pass == 0) {
            if (lane == 0) row_len[i] = k + nin - matched;
        } else {
            const int64_t base = row_ptr[i];
            for (int m = lane; m < k; m += 32) {
                const int j = oc[m];
                double v = ov[m];
                int less_in;
                if (oin[m] >= 0) {
                    less_in = oin[m];
                    v += pc[ie[less_in]];
                } else {
                    int lo = 0, hi = nin;
                    while (lo < hi) {
                        const int mid = (lo + hi) / 2;
                        if ((int)(ie[mid] / uk) < j) lo = mid + 1;
                        else hi = mid;
                    }
                    less_in = lo;
                }
                const int64_t pos = base + m + less_in - F[m];
                col[pos] = j;
                val[pos] = (float)(v * inv2n);
            }
            for (int t = lane; t < nin; t += 32) {
                const uint32_t ed = ie[t];
                const int s = (int)(ed / uk);
                int lo = 0, hi = k;
                while (lo < hi) {
                    const int mid = (lo + hi) / 2;
                    if (oc[mid] < s) lo = mid + 1;
                    else hi = mid;
                }
                if (lo < k && oc[lo] == s) continue;  // written with its out-entry
                const int64_t pos = base + lo + t - F[lo];
                col[pos] = s;
                val[pos] = (float)(pc[ed] * inv2n);
            }
        }
        __syncwarp();
    }
}

}  // namespace fitsne

// ----------------------------------------------------------------------------
// C ABI
// ----------------------------------------------------------------------------
struct tsne_affinity {
    int64_t N = 0;
    int D = 0, k = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    int max_smem = 0;             // opt-in shared memory per block
    int knn_kind = 0;             // 0 knn_kernel, 1 knn_tiled_kernel, 2 tensor cores (+ knn_kernel)
    fitsne::KnnTc* tc = nullptr;  // workspace of the tensor-core kNN
    int64_t recomputed = 0;       // queries of the last compute left to knn_kernel
    int calib_exact = 0;          // 1: every bandwidth step in FP64 (FITSNE_CALIB_FP64=1; same results)
    int64_t Np = 0;               // N rounded up to the candidate tile
    float* Xt = nullptr;          // [D][Np] transposed, zero-padded X
    int32_t* knn_idx = nullptr;   // [N k]
    float* knn_d2 = nullptr;      // [N k]
    double* pc = nullptr;         // [N k] p_{j|i}
    uint32_t* keys[2] = {nullptr, nullptr};
    uint32_t* items[2] = {nullptr, nullptr};
    uint32_t* counts = nullptr;   // [256 nblocks]
    int32_t* in_ptr = nullptr;    // [N + 1]
    int32_t* row_ptr = nullptr;   // [N + 1]
    int32_t* col = nullptr;       // [2 N k]
    float* val = nullptr;         // [2 N k]
    int64_t nnz = -1;             // of the last compute
    int64_t launches = 0;
    cudaEvent_t ev[5] = {};       // phase boundaries of the last compute
};

namespace {

int aff_cuda_fail(cudaError_t e, const char* what) {
    return fitsne::set_error(TSNE_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define ACU(call, what)                                          \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return aff_cuda_fail(e_, what);   \
    } while (0)

void free_affinity(tsne_affinity* a) {
    if (!a) return;
    void* ps[] = {a->Xt, a->knn_idx, a->knn_d2, a->pc, a->keys[0], a->keys[1], a->items[0], a->items[1],
                  a->counts, a->in_ptr, a->row_ptr, a->col, a->val};
    for (void* p : ps)
        if (p) cudaFree(p);
    for (cudaEvent_t e : a->ev)
        if (e) cudaEventDestroy(e);
    fitsne::knn_tc_destroy(a->tc);
    delete a;
}

template <typename T>
int aff_alloc(T** p, size_t count, const char* what) {
    *p = nullptr;
    if (cudaMalloc((void**)p, (count ? count : 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fitsne::set_error(TSNE_ERR_OOM, "cudaMalloc of %zu bytes for %s failed",
                                 count * sizeof(T), what);
    }
    return TSNE_OK;
}

}  // namespace

extern "C" {

int tsne_affinity_create(int64_t N, int32_t D, int32_t k, void* stream, tsne_affinity** out) {
    fitsne::clear_error();
    if (!out) return fitsne::set_error(TSNE_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (D < 1 || D > fitsne::kKnnDMax)
        return fitsne::set_error(TSNE_ERR_INVALID_ARG, "D = %d outside [1, %d]", D, fitsne::kKnnDMax);
    if (k < 1 || k > fitsne::kKnnKMax)
        return fitsne::set_error(TSNE_ERR_INVALID_ARG, "k = %d outside [1, %d]", k, fitsne::kKnnKMax);
    if (N < 2 || N <= k)
        return fitsne::set_error(TSNE_ERR_INVALID_ARG, "N = %lld must exceed k = %d", (long long)N, k);
    const int64_t nk = N * (int64_t)k;
    if (2 * nk > INT32_MAX)  // edge ids (i k + m) and CSR offsets are 32-bit
        return fitsne::set_error(TSNE_ERR_INVALID_ARG, "2 N k = %lld exceeds 2^31 - 1", (long long)(2 * nk));
    tsne_affinity* a = new tsne_affinity();
    a->N = N;
    a->D = D;
    a->k = k;
    a->stream = (cudaStream_t)stream;
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&a->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&a->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    for (int e = 0; e < 5 && ce == cudaSuccess; ++e) ce = cudaEventCreate(&a->ev[e]);
    if (ce != cudaSuccess) { free_affinity(a); return aff_cuda_fail(ce, "device setup"); }
    const int64_t nblocks = (nk + fitsne::kRadixTile - 1) / fitsne::kRadixTile;
    // kernel choice: the tensor-core kernel from N = FITSNE_KNN_TC_MIN_N;
    // below it the tiled kernel where its shared memory fits and N is large,
    // else the row kernel. FITSNE_KNN_KERNEL=tc|tiled|rows in the
    // environment overrides the size rule (tests and tuning; "tiled" still
    // needs the memory to fit)
    const bool fits = fitsne::knn_tiled_smem_bytes(D, k) <= (size_t)a->max_smem;
    const bool tc_ok = fitsne::knn_tc_supported(D, k);
    a->knn_kind = (tc_ok && N >= FITSNE_KNN_TC_MIN_N) ? 2 : (fits && N >= FITSNE_KNN_TILED_MIN_N) ? 1 : 0;
    if (const char* ov = getenv("FITSNE_KNN_KERNEL")) {
        if (!strcmp(ov, "tc")) a->knn_kind = tc_ok ? 2 : 0;
        else if (!strcmp(ov, "tiled")) a->knn_kind = fits ? 1 : 0;
        else if (!strcmp(ov, "rows")) a->knn_kind = 0;
    }
    if (const char* ce = getenv("FITSNE_CALIB_FP64")) a->calib_exact = ce[0] == '1' ? 1 : 0;
    a->Np = (N + fitsne::kTileC - 1) / fitsne::kTileC * fitsne::kTileC;
    int rc = TSNE_OK;
    if (a->knn_kind == 1) rc = aff_alloc(&a->Xt, (size_t)D * (size_t)a->Np, "transposed X");
    if (!rc && a->knn_kind == 2) rc = fitsne::knn_tc_create(N, D, k, a->sm_count, &a->tc);
    if (!rc) rc = aff_alloc(&a->knn_idx, (size_t)nk, "kNN indices");
    if (!rc) rc = aff_alloc(&a->knn_d2, (size_t)nk, "kNN distances");
    if (!rc) rc = aff_alloc(&a->pc, (size_t)nk, "conditional affinities");
    for (int b = 0; b < 2 && !rc; ++b) {
        rc = aff_alloc(&a->keys[b], (size_t)nk, "sort keys");
        if (!rc) rc = aff_alloc(&a->items[b], (size_t)nk, "sort items");
    }
    if (!rc) rc = aff_alloc(&a->counts, (size_t)(256 * nblocks), "digit counts");
    if (!rc) rc = aff_alloc(&a->in_ptr, (size_t)(N + 1), "in-list offsets");
    if (!rc) rc = aff_alloc(&a->row_ptr, (size_t)(N + 1), "row_ptr");
    if (!rc) rc = aff_alloc(&a->col, (size_t)(2 * nk), "col");
    if (!rc) rc = aff_alloc(&a->val, (size_t)(2 * nk), "val");
    if (rc) { free_affinity(a); return rc; }
    *out = a;
    return TSNE_OK;
}

int tsne_affinity_destroy(tsne_affinity* a) {
    fitsne::clear_error();
    if (!a) return TSNE_OK;
    cudaStreamSynchronize(a->stream);
    free_affinity(a);
    return TSNE_OK;
}

int tsne_affinity_compute(tsne_affinity* a, const float* X, double perplexity, tsne_csr* P_out) {
    fitsne::clear_error();
    if (!a) return fitsne::set_error(TSNE_ERR_INVALID_ARG, "affinity object is NULL");
    if (!X || !P_out) return fitsne::set_error(TSNE_ERR_INVALID_ARG, "X or P_out is NULL");
    if (!(perplexity >= 1.0) || !(perplexity <= (double)a->k))
        return fitsne::set_error(TSNE_ERR_INVALID_ARG, "perplexity %g outside [1, k = %d]", perplexity, a->k);
    using namespace fitsne;
    const int64_t N = a->N, nk = N * (int64_t)a->k;
    const int k = a->k;
    cudaStream_t st = a->stream;
    a->nnz = -1;
    ACU(cudaEventRecord(a->ev[0], st), "event");
    // 1. exact kNN
    a->recomputed = 0;
    if (a->knn_kind == 2) {
        if (int rc = knn_tc_launch(a->tc, X, a->knn_idx, a->knn_d2, st, &a->launches)) return rc;
        int64_t left = 0;
        const int32_t* list = nullptr;
        if (int rc = knn_tc_leftover(a->tc, st, &left, &list)) return rc;
        a->recomputed = left;
        if (left > 0) {
            const int64_t nqb = (left + kKnnWarps * kKnnQ - 1) / (kKnnWarps * kKnnQ);
            const int grid = (int)std::min<int64_t>(nqb, 64LL * a->sm_count);
            ACU(cudaFuncSetAttribute(knn_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)knn_smem_bytes(a->D, k)),
                "kNN shared memory");
            knn_kernel<true><<<grid, kKnnWarps * 32, knn_smem_bytes(a->D, k), st>>>(
                X, N, a->D, k, 0, left, a->knn_idx, a->knn_d2, list);
            ACU(cudaGetLastError(), "kNN launch");
            a->launches += 1;
        }
        a->launches -= 1;  // the count below includes one kNN kernel
    } else if (a->knn_kind == 1) {
        const int64_t total = (int64_t)a->D * a->Np;
        transpose_pad_kernel<<<(int)std::min<int64_t>((total + 255) / 256, 8LL * a->sm_count), 256, 0, st>>>(
            X, N, a->D, a->Np, a->Xt);
        const int64_t nqb = (N + kTileQ - 1) / kTileQ;
        const size_t smem = knn_tiled_smem_bytes(a->D, k);
        ACU(cudaFuncSetAttribute(knn_tiled_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
            "kNN shared memory");
        knn_tiled_kernel<<<(int)std::min<int64_t>(nqb, 1 << 20), kTiledThreads, smem, st>>>(
            a->Xt, N, a->Np, a->D, k, a->knn_idx, a->knn_d2);
        ACU(cudaGetLastError(), "kNN launch");
        a->launches += 1;  // the transpose (the kNN kernel is counted below)
    } else {
        const int64_t nqb = (N + kKnnWarps * kKnnQ - 1) / (kKnnWarps * kKnnQ);
        const int grid = (int)std::min<int64_t>(nqb, 64LL * a->sm_count);
        // a per-function attribute: set for this workspace's size at each launch
        ACU(cudaFuncSetAttribute(knn_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)knn_smem_bytes(a->D, k)),
            "kNN shared memory");
        knn_kernel<false><<<grid, kKnnWarps * 32, knn_smem_bytes(a->D, k), st>>>(X, N, a->D, k, 0, N,
                                                                                  a->knn_idx, a->knn_d2, nullptr);
        ACU(cudaGetLastError(), "kNN launch");
    }
    ACU(cudaEventRecord(a->ev[1], st), "event");
    // 2. bandwidths
    {
        const int grid = (int)std::min<int64_t>((N + 7) / 8, 16LL * a->sm_count);
        calibrate_kernel<<<grid, 256, 0, st>>>(a->knn_d2, N, k, log(perplexity), a->pc, a->calib_exact);
        ACU(cudaGetLastError(), "calibrate launch");
    }
    ACU(cudaEventRecord(a->ev[2], st), "event");
    // 3. edges sorted by target (stable: sources increasing within a target)
    const int nblocks = (int)((nk + kRadixTile - 1) / kRadixTile);
    const int rgrid = std::min(nblocks, 8 * a->sm_count);
    {
        const int grid = (int)std::min<int64_t>((nk + 255) / 256, 8LL * a->sm_count);
        edge_keys_kernel<<<grid, 256, 0, st>>>(a->knn_idx, nk, a->keys[0], a->items[0]);
        ACU(cudaGetLastError(), "edge keys launch");
    }
    int bits = 1;
    while (bits < 31 && ((N - 1) >> bits) != 0) ++bits;
    int cur = 0, passes = 0;
    for (int shift = 0; shift < bits; shift += 8, ++passes) {
        radix_count_kernel<<<rgrid, kRadixThreads, 0, st>>>(a->keys[cur], nk, shift, a->counts, nblocks);
        scan_inplace_kernel<<<1, 1024, 0, st>>>(a->counts, 256LL * nblocks);
        radix_scatter_kernel<<<rgrid, kRadixThreads, 0, st>>>(a->keys[cur], a->items[cur], nk, shift, a->counts,
                                                               nblocks, a->keys[cur ^ 1], a->items[cur ^ 1]);
        ACU(cudaGetLastError(), "radix pass launch");
        cur ^= 1;
    }
    {
        const int grid = (int)std::min<int64_t>((N + 256) / 256, 8LL * a->sm_count);
        in_ptr_kernel<<<grid, 256, 0, st>>>(a->keys[cur], nk, N, a->in_ptr);
        ACU(cudaGetLastError(), "in-list offsets launch");
    }
    ACU(cudaEventRecord(a->ev[3], st), "event");
    // 4. symmetrise: union sizes, offsets, union
    const int sgrid = (int)std::min<int64_t>((N + 7) / 8, 16LL * a->sm_count);
    symmetrise_kernel<<<sgrid, 256, 0, st>>>(a->knn_idx, a->pc, N, k, a->in_ptr, a->items[cur], 0, a->row_ptr,
                                             nullptr, nullptr, nullptr);
    ACU(cudaMemsetAsync(a->row_ptr + N, 0, sizeof(int32_t), st), "row_ptr tail");
    scan_inplace_kernel<<<1, 1024, 0, st>>>(reinterpret_cast<uint32_t*>(a->row_ptr), N + 1);
    symmetrise_kernel<<<sgrid, 256, 0, st>>>(a->knn_idx, a->pc, N, k, a->in_ptr, a->items[cur], 1, nullptr,
                                             a->row_ptr, a->col, a->val);
    ACU(cudaGetLastError(), "symmetrise launch");
    ACU(cudaEventRecord(a->ev[4], st), "event");
    a->launches += 7 + 3 * passes;
    int32_t nnz = 0;
    ACU(cudaMemcpyAsync(&nnz, a->row_ptr + N, sizeof(int32_t), cudaMemcpyDeviceToHost, st), "nnz read-back");
    ACU(cudaStreamSynchronize(st), "affinity synchronise");
    a->nnz = nnz;
    P_out->row_ptr = a->row_ptr;
    P_out->col = a->col;
    P_out->val = a->val;
    P_out->nnz = nnz;
    return TSNE_OK;
}

int tsne_affinity_knn_copy(const tsne_affinity* a, int32_t* idx_host, float* d2_host, double* pcond_host) {
    fitsne::clear_error();
    if (!a) return fitsne::set_error(TSNE_ERR_INVALID_ARG, "affinity object is NULL");
    if (a->nnz < 0) return fitsne::set_error(TSNE_ERR_INVALID_ARG, "no affinities computed yet");
    const size_t nk = (size_t)a->N * (size_t)a->k;
    if (idx_host)
        ACU(cudaMemcpyAsync(idx_host, a->knn_idx, nk * sizeof(int32_t), cudaMemcpyDeviceToHost, a->stream), "copy");
    if (d2_host)
        ACU(cudaMemcpyAsync(d2_host, a->knn_d2, nk * sizeof(float), cudaMemcpyDeviceToHost, a->stream), "copy");
    if (pcond_host)
        ACU(cudaMemcpyAsync(pcond_host, a->pc, nk * sizeof(double), cudaMemcpyDeviceToHost, a->stream), "copy");
    ACU(cudaStreamSynchronize(a->stream), "copy synchronise");
    return TSNE_OK;
}

int tsne_affinity_phase_ms(const tsne_affinity* a, double* ms_out) {
    fitsne::clear_error();
    if (!a || !ms_out) return fitsne::set_error(TSNE_ERR_INVALID_ARG, "affinity object or ms_out is NULL");
    if (a->nnz < 0) return fitsne::set_error(TSNE_ERR_INVALID_ARG, "no affinities computed yet");
    for (int e = 0; e < 4; ++e) {
        float ms = 0.0f;
        ACU(cudaEventElapsedTime(&ms, a->ev[e], a->ev[e + 1]), "event time");
        ms_out[e] = ms;
    }
    return TSNE_OK;
}

int64_t tsne_affinity_launch_count(const tsne_affinity* a) { return a ? a->launches : 0; }

int tsne_affinity_knn_info(const tsne_affinity* a, int32_t* kernel_out, int64_t* recomputed_out) {
    fitsne::clear_error();
    if (!a) return fitsne::set_error(TSNE_ERR_INVALID_ARG, "affinity object is NULL");
    if (kernel_out) *kernel_out = a->knn_kind;
    if (recomputed_out) *recomputed_out = a->recomputed;
    return TSNE_OK;
}

}  // extern "C"
