// Per-point and per-entry kernels of the FIt-SNE gradient on sm_103a:
//   box_kernel      bounding box and interval rule (Sec. 2.2, 2.4, 2.5)
//   count/scatter   counting sort of the points by box (the "points in I_l"
//                   loops of Algorithm 1)
//   scan kernels    box offsets and the spread work list
//   spread_kernel   Step 1: w_m = sum_{y_i in I_l} L_m(y_i) q_i per box
//   force_kernel    attraction over the CSR rows (Sec. 3) fused with Step 3
//                   (interpolate back), the Appendix assembly of F_rep and,
//                   for a descent step, the gains/momentum update
//   kl_kernel       KL(P || Q) of Sec. 1.1 with FP64 sums
// None of these kernels uses global floating-point atomics except the spread
// of boxes holding more than one chunk of points.
#include <math.h>

#include <algorithm>

#include "fitsne_internal.cuh"

namespace fitsne {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Reduces a[0..NV) (NV a multiple of 32) across the warp so that, for every
// group g of 32 values, lane l ends with the warp total of value g*32 + l in
// a[g*32]. 31 shuffles per group instead of 5 per value. Integer T makes the
// result independent of the order of the additions.
template <int NV, typename T>
__device__ __forceinline__ void warp_transpose_reduce(T (&a)[NV], int lane) {
#pragma unroll
    for (int g = 0; g < NV / 32; ++g) {
        T* v = a + g * 32;
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            const bool upper = (lane & off) != 0;
#pragma unroll
            for (int i = 0; i < off; ++i) {
                T send = upper ? v[i] : v[i + off];
                T keep = upper ? v[i + off] : v[i];
                v[i] = keep + __shfl_xor_sync(kFull, send, off);
            }
        }
    }
}

template <int S>
__device__ __forceinline__ int box_of(const float* __restrict__ Y, int64_t i, const Params& P) {
    if (S == 2) {
        float2 y = reinterpret_cast<const float2*>(Y)[i];
        return interval_of(y.x, P) * P.n_int + interval_of(y.y, P);
    } else {
        return interval_of(Y[i], P);
    }
}

}  // namespace

// ----------------------------------------------------------------------------
// Bounding box: per-block min/max, then the last block to finish derives the
// box, N_int, node spacing and FFT length (Sec. 2.2, 2.4, 2.5). The FP32
// rule matches the oracle's bit for bit.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(kBoxThreads)
box_kernel(const float* __restrict__ Y, int64_t count, int s, int p, int n_int_fixed, int n_min,
           int n_int_max, int force, float f_y_min, float f_width, int f_n_int, int fx_shift,
           float* __restrict__ partial, unsigned* __restrict__ ticket, Params* __restrict__ params,
           const FftEntry* __restrict__ table, const int32_t* __restrict__ fft_of_n) {
    float lo = INFINITY, hi = -INFINITY;
    int bad = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t k0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if ((reinterpret_cast<uintptr_t>(Y) & 15) == 0) {
        const int64_t n4 = count / 4;
        const float4* Y4 = reinterpret_cast<const float4*>(Y);
        for (int64_t k = k0; k < n4; k += stride) {
            float4 v = __ldg(&Y4[k]);
            bad |= !isfinite(v.x) | !isfinite(v.y) | !isfinite(v.z) | !isfinite(v.w);
            lo = fminf(lo, fminf(fminf(v.x, v.y), fminf(v.z, v.w)));
            hi = fmaxf(hi, fmaxf(fmaxf(v.x, v.y), fmaxf(v.z, v.w)));
        }
        for (int64_t k = n4 * 4 + k0; k < count; k += stride) {
            float v = Y[k];
            bad |= !isfinite(v);
            lo = fminf(lo, v);
            hi = fmaxf(hi, v);
        }
    } else {
        for (int64_t k = k0; k < count; k += stride) {
            float v = Y[k];
            bad |= !isfinite(v);
            lo = fminf(lo, v);
            hi = fmaxf(hi, v);
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(kFull, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(kFull, hi, o));
    }
    __shared__ float s_lo[kBoxThreads / 32], s_hi[kBoxThreads / 32];
    __shared__ bool s_last;
    bad = __syncthreads_or(bad);
    const int wid = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (lane == 0) { s_lo[wid] = lo; s_hi[wid] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < kBoxThreads / 32; ++i) { lo = fminf(lo, s_lo[i]); hi = fmaxf(hi, s_hi[i]); }
        partial[2 * blockIdx.x] = bad ? NAN : lo;
        partial[2 * blockIdx.x + 1] = hi;
        __threadfence();
        s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the last block reduces the per-block partials
    int bad_p = 0;
    lo = INFINITY;
    hi = -INFINITY;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) {
        float a = __ldcg(&partial[2 * i]), b = __ldcg(&partial[2 * i + 1]);
        bad_p |= isnan(a);
        lo = fminf(lo, a);
        hi = fmaxf(hi, b);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(kFull, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(kFull, hi, o));
    }
    const bool any_bad = __syncthreads_or(bad_p);
    if (lane == 0) { s_lo[wid] = lo; s_hi[wid] = hi; }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int i = 0; i < kBoxThreads / 32; ++i) { lo = fminf(lo, s_lo[i]); hi = fmaxf(hi, s_hi[i]); }
    *ticket = 0u;
    Params P;
    P.error = __ldcg(&params->error);
    if (any_bad) { P.error = TSNE_ERR_NONFINITE; lo = 0.0f; hi = 1.0f; }
    float y_min, width;
    int n_int;
    if (force) {
        y_min = f_y_min;
        width = f_width;
        n_int = f_n_int;
    } else {
        y_min = lo;
        width = __fsub_rn(hi, lo);
        if (!(width > 0.0f)) width = 1.0f;
        if (n_int_fixed > 0) {
            n_int = n_int_fixed;
        } else {
            float c = ceilf(width);
            if (c > (float)n_int_max) c = (float)n_int_max;
            n_int = (int)c;
            if (n_int < n_min) n_int = n_min;
            if (n_int > n_int_max) n_int = n_int_max;
        }
    }
    P.y_min = y_min;
    P.width = width;
    P.n_int = n_int;
    P.b = __fdiv_rn(width, (float)n_int);
    P.inv_b = __fdiv_rn(1.0f, P.b);
    P.delta = __fdiv_rn(P.b, (float)p);
    P.inv_delta = __fdiv_rn((float)p, P.b);
    P.delta2 = __fmul_rn(P.delta, P.delta);
    P.fx_shift = fx_shift;
    P.fx_scale = ldexpf(1.0f, fx_shift);
    P.fx_inv = ldexpf(1.0f, -fx_shift);
    P.n = p * n_int;
    P.n_boxes = (s == 2) ? n_int * n_int : n_int;
    const int idx = fft_of_n[P.n];
    P.fft_idx = idx;
    P.L = table[idx].L;
    P.p_f = (float)p;
    P.pad = 0;
    P.n_chunks = 0;
    P.Z = 0.0;
    P.inv_Z = 0.0f;
    *params = P;
}

// ----------------------------------------------------------------------------
// Counting sort by box: histogram (warp-aggregated integer atomics), scan,
// scatter. Points of one box end up contiguous in sorted_y; their order
// within the box is not fixed, which the integer spread sums do not see.
// ----------------------------------------------------------------------------
// Each block takes kSortPts consecutive points. With at most kHistBins
// boxes the block first counts in a shared-memory histogram and touches the
// global counters once per box it met, which keeps boxes holding many points
// (tight clusters) from serialising on one global atomic; with more boxes
// (each then holds few points) it uses the global counters directly.
template <int S>
__global__ void __launch_bounds__(256)
count_kernel(const float* __restrict__ Y, int64_t N, const Params* __restrict__ params,
             int32_t* __restrict__ counts, long long* __restrict__ w) {
    extern __shared__ int32_t hist[];
    const Params P = *params;
    if (P.error) return;
    const int nb = P.n_boxes;
    {  // the spread grids of this iteration start at zero
        const int64_t G = (S == 2) ? (int64_t)P.n * P.n : P.n;
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < (S + 1) * G; g += stride)
            w[g] = 0;
    }
    const bool local = nb <= kHistBins;
    const int lane = threadIdx.x % 32;
    if (local) {
        for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0;
        __syncthreads();
    }
    const int64_t p0 = (int64_t)blockIdx.x * kSortPts;
    for (int k = 0; k < kSortPts / 256; ++k) {
        const int64_t i = p0 + k * 256 + threadIdx.x;
        const int box = (i < N) ? box_of<S>(Y, i, P) : -1;
        const unsigned peers = __match_any_sync(kFull, box);
        if (box >= 0 && lane == __ffs(peers) - 1) {
            if (local) atomicAdd(&hist[box], __popc(peers));
            else atomicAdd(&counts[box], __popc(peers));
        }
    }
    if (local) {
        __syncthreads();
        for (int b = threadIdx.x; b < nb; b += blockDim.x)
            if (hist[b]) atomicAdd(&counts[b], hist[b]);
    }
}

// Same partition: the block counts its points per box, reserves one range
// per box in the global cursors, then places each point at its box's range
// plus its rank inside the block.
template <int S>
__global__ void __launch_bounds__(256)
scatter_kernel(const float* __restrict__ Y, int64_t N, const Params* __restrict__ params,
               int32_t* __restrict__ cursor, float* __restrict__ sorted_y) {
    extern __shared__ int32_t hist[];
    constexpr int K = kSortPts / 256;
    const Params P = *params;
    if (P.error) return;
    const int nb = P.n_boxes;
    const bool local = nb <= kHistBins;
    const int lane = threadIdx.x % 32;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t p0 = (int64_t)blockIdx.x * kSortPts;
    int box[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int64_t i = p0 + k * 256 + threadIdx.x;
        box[k] = (i < N) ? box_of<S>(Y, i, P) : -1;
    }
    if (local) {
        for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const unsigned peers = __match_any_sync(kFull, box[k]);
            if (box[k] >= 0 && lane == __ffs(peers) - 1) atomicAdd(&hist[box[k]], __popc(peers));
        }
        __syncthreads();
        for (int b = threadIdx.x; b < nb; b += blockDim.x)
            if (hist[b]) hist[b] = atomicAdd(&cursor[b], hist[b]);
        __syncthreads();
    }
    int32_t* dst_cursor = local ? hist : cursor;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const unsigned peers = __match_any_sync(kFull, box[k]);
        const int leader = __ffs(peers) - 1;
        int pos = 0;
        if (box[k] >= 0 && lane == leader) pos = atomicAdd(&dst_cursor[box[k]], __popc(peers));
        pos = __shfl_sync(kFull, pos, leader) + __popc(peers & lt);
        if (box[k] >= 0) {
            const int64_t i = p0 + k * 256 + threadIdx.x;
            if (S == 2)
                reinterpret_cast<float2*>(sorted_y)[pos] = reinterpret_cast<const float2*>(Y)[i];
            else
                sorted_y[pos] = Y[i];
        }
    }
}

// Block-wide exclusive scan of one int per thread (1024 threads).
__device__ __forceinline__ int block_exclusive_scan(int v, int* smem_warp, int& total) {
    const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = (lane < (int)(blockDim.x / 32)) ? smem_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        smem_warp[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    total = smem_warp[blockDim.x / 32 - 1];
    int excl = x - v + (wid > 0 ? smem_warp[wid - 1] : 0);
    __syncthreads();
    return excl;
}

// Pass 1: per-block totals of points and of spread chunks (ceil(count/kChunk));
// the last block turns them into exclusive block offsets.
__global__ void __launch_bounds__(1024)
scan_blocks_kernel(const int32_t* __restrict__ counts, Params* params,
                   int32_t* __restrict__ block_pts, int32_t* __restrict__ block_chunks,
                   unsigned* __restrict__ ticket) {
    __shared__ int sw[32];
    __shared__ bool s_last;
    const int nb = params->n_boxes;
    const int base = blockIdx.x * kScanBlock + threadIdx.x * 2;
    int c0 = base < nb ? counts[base] : 0;
    int c1 = base + 1 < nb ? counts[base + 1] : 0;
    int pts = c0 + c1;
    int chk = (c0 + kChunk - 1) / kChunk + (c1 + kChunk - 1) / kChunk;
    int tp, tc;
    block_exclusive_scan(pts, sw, tp);
    block_exclusive_scan(chk, sw, tc);
    if (threadIdx.x == 0) {
        block_pts[blockIdx.x] = tp;
        block_chunks[blockIdx.x] = tc;
        __threadfence();
        s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    int carry_p = 0, carry_c = 0;
    for (unsigned start = 0; start < gridDim.x; start += blockDim.x) {
        const unsigned i = start + threadIdx.x;
        int vp = i < gridDim.x ? __ldcg(&block_pts[i]) : 0;
        int vc = i < gridDim.x ? __ldcg(&block_chunks[i]) : 0;
        int sp, sc;
        int ep = block_exclusive_scan(vp, sw, sp);
        int ec = block_exclusive_scan(vc, sw, sc);
        if (i < gridDim.x) {
            block_pts[i] = carry_p + ep;
            block_chunks[i] = carry_c + ec;
        }
        carry_p += sp;
        carry_c += sc;
    }
    if (threadIdx.x == 0) {
        params->n_chunks = carry_c;
        *ticket = 0u;
    }
}

// Pass 2: box offsets, scatter cursors, chunk -> box table; resets the counts
// for the next iteration. Each warp writes the chunk entries of its 64 boxes
// with its lanes in parallel (a box holding many points has many chunks).
template <int S, int PP>
__global__ void __launch_bounds__(1024)
scan_boxes_kernel(int32_t* __restrict__ counts, const Params* __restrict__ params,
                  const int32_t* __restrict__ block_pts, const int32_t* __restrict__ block_chunks,
                  int32_t* __restrict__ box_start, int32_t* __restrict__ cursor,
                  int32_t* __restrict__ chunk_start, int32_t* __restrict__ chunk_box, int64_t N) {
    __shared__ int sw[32];
    const Params P = *params;
    const int nb = P.n_boxes;
    if (blockIdx.x * kScanBlock >= nb) return;  // uniform per block
    const int lane = threadIdx.x % 32;
    const int base = blockIdx.x * kScanBlock + threadIdx.x * 2;
    int c[2] = {base < nb ? counts[base] : 0, base + 1 < nb ? counts[base + 1] : 0};
    int k[2] = {(c[0] + kChunk - 1) / kChunk, (c[1] + kChunk - 1) / kChunk};
    int tp, tc;
    int ep = block_exclusive_scan(c[0] + c[1], sw, tp) + block_pts[blockIdx.x];
    int ec = block_exclusive_scan(k[0] + k[1], sw, tc) + block_chunks[blockIdx.x];
    int ecb[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int b = base + u;
        ecb[u] = ec;
        if (b < nb) {
            box_start[b] = ep;
            cursor[b] = ep;
            chunk_start[b] = ec;
            counts[b] = 0;
            if (b == nb - 1) {
                box_start[nb] = (int32_t)N;
                chunk_start[nb] = ec + k[u];
            }
        }
        ep += c[u];
        ec += k[u];
    }
    // chunk -> box entries: the warp visits its lanes' boxes one by one
    for (int src = 0; src < 32; ++src) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int b = __shfl_sync(kFull, base + u, src);
            const int kb = __shfl_sync(kFull, k[u], src);
            const int eb = __shfl_sync(kFull, ecb[u], src);
            if (b < nb)
                for (int q = lane; q < kb; q += 32) chunk_box[eb + q] = b;
        }
    }
}

// ----------------------------------------------------------------------------
// Step 1 (spread): one warp per chunk of at most kChunk points of one box.
// For node g = (j1, j2) of the box and a point with local coordinates t
// (units of delta), the point adds W = L_j1(t1) L_j2(t2) to the charge grid
// w0 and W (t_m - j_m - 1/2) to the dipole grids d_m, the charge y(m) taken
// relative to the node it lands on: sum_g L_g(y) (y(m) - y~_g(m)) / delta.
// This equals the paper's spread of the charges y(m) less y~_g(m) w0[g]
// (exact: spreading is linear in the charge), and keeps every value O(1).
// Values are accumulated as 64-bit integers of x * 2^fx_shift, so the sums
// (in registers, across lanes, and the atomics of boxes with several chunks)
// do not depend on the order of the points: the grids are bitwise
// reproducible. Each lane accumulates its points; a transpose reduction
// gives lane v the warp total of value v.
// ----------------------------------------------------------------------------
template <int S, int PP>
__global__ void __launch_bounds__(256)
spread_kernel(const float* __restrict__ sorted_y, const int32_t* __restrict__ box_start,
              const int32_t* __restrict__ chunk_start, const int32_t* __restrict__ chunk_box,
              const Params* __restrict__ params, long long* __restrict__ w) {
    constexpr int NODES = (S == 2) ? PP * PP : PP;
    constexpr int NVAL = (S + 1) * NODES;
    constexpr int NV = (NVAL + 31) / 32 * 32;
    const Params P = *params;
    if (P.error) return;
    const int lane = threadIdx.x % 32;
    const int nwarp = gridDim.x * blockDim.x / 32;
    const int n = P.n;
    const int64_t G = (S == 2) ? (int64_t)n * n : n;
    const float sc = P.fx_scale;
    for (int q = (blockIdx.x * blockDim.x + threadIdx.x) / 32; q < P.n_chunks; q += nwarp) {
        const int box = chunk_box[q];
        const int bs = box_start[box];
        const int cnt = box_start[box + 1] - bs;
        const int ci = q - chunk_start[box];
        const int start = bs + ci * kChunk;
        const int len = min(kChunk, cnt - ci * kChunk);
        const int bx = (S == 2) ? box / P.n_int : box;
        const int by = (S == 2) ? box % P.n_int : 0;
        long long acc[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = 0;
        for (int k = lane; k < len; k += 32) {
            float L1[PP], L2[PP], e1[PP], e2[PP];
            if (S == 2) {
                const float2 y = reinterpret_cast<const float2*>(sorted_y)[start + k];
                const float t1 = local_t(y.x, bx, P), t2 = local_t(y.y, by, P);
                lagrange<PP>(t1, L1);
                lagrange<PP>(t2, L2);
#pragma unroll
                for (int j = 0; j < PP; ++j) {
                    e1[j] = t1 - ((float)j + 0.5f);
                    e2[j] = t2 - ((float)j + 0.5f);
                }
            } else {
                const float t1 = local_t(sorted_y[start + k], bx, P);
                lagrange<PP>(t1, L1);
#pragma unroll
                for (int j = 0; j < PP; ++j) e1[j] = t1 - ((float)j + 0.5f);
            }
#pragma unroll
            for (int j1 = 0; j1 < PP; ++j1) {
#pragma unroll
                for (int j2 = 0; j2 < (S == 2 ? PP : 1); ++j2) {
                    const float W = (S == 2) ? L1[j1] * L2[j2] : L1[j1];
                    const int node = (S == 2) ? j1 * PP + j2 : j1;
                    acc[node] += __float2ll_rn(W * sc);
                    acc[NODES + node] += __float2ll_rn((W * e1[j1]) * sc);
                    if (S == 2) acc[2 * NODES + node] += __float2ll_rn((W * e2[j2]) * sc);
                }
            }
        }
        warp_transpose_reduce<NV>(acc, lane);
        const bool multi = cnt > kChunk;
#pragma unroll
        for (int g = 0; g < NV / 32; ++g) {
            const int v = g * 32 + lane;
            if (v < NVAL) {
                const int ch = v / NODES, node = v % NODES;
                const int j1 = (S == 2) ? node / PP : node;
                const int j2 = (S == 2) ? node % PP : 0;
                const int64_t gi = (S == 2) ? (int64_t)(bx * PP + j1) * n + (by * PP + j2)
                                            : (int64_t)(bx * PP + j1);
                long long* dst = &w[ch * G + gi];
                if (multi)
                    atomicAdd(reinterpret_cast<unsigned long long*>(dst),
                              static_cast<unsigned long long>(acc[g * 32]));
                else
                    *dst = acc[g * 32];
            }
        }
    }
}

// ----------------------------------------------------------------------------
// Attraction + Step 3 + gradient (+ update). One warp per CSR row i:
//   A_i = sum_j p_ij (y_i - y_j) / (1 + |y_i - y_j|^2)                 (Sec. 3)
//   F_rep,i(m) = (h_{m+1}(y_i) - y_i(m) h_{s+2}(y_i)) / Z              (Appendix)
//   dY_i = 4 (alpha A_i + F_rep,i)                                     (Sec. 1.2)
// with the interpolated h of Step 3. The numerator is evaluated in the
// node-relative form: with u_m = v_m - y~(m) v_{s+2} at each node (computed
// by the convolution without cancellation, see fitsne_fft.cu),
//   h_{m+1}(y_i) - y_i(m) h_{s+2}(y_i)
//     = sum_g L_g(y_i) [u_m[g] + (y~_g(m) - y_i(m)) v_{s+2}[g]]
//     = delta sum_g L_g(y_i) [u'_m[g] + (j_m + 1/2 - t_m) v_{s+2}[g]],
// an identity in exact arithmetic whose terms stay O(1) in FP32.
// ----------------------------------------------------------------------------
struct StepArgs {
    float* Y_new;
    float* uY;
    float* gains;
    float momentum, lr, min_gain, gain_inc, gain_dec;
};

__device__ __forceinline__ float update_one(float y, float dy, float& u, float& g,
                                            const StepArgs& a) {
    const int sd = (dy > 0.0f) - (dy < 0.0f);
    const int su = (u > 0.0f) - (u < 0.0f);
    float gn = (sd != su) ? g + a.gain_inc : g * a.gain_dec;
    gn = fmaxf(gn, a.min_gain);
    g = gn;
    u = a.momentum * u - a.lr * gn * dy;
    return y + u;
}

#ifndef FITSNE_GATHER_L2_ONLY
#define FITSNE_GATHER_L2_ONLY 0  // 1: the Y[j] gathers bypass L1 (ld.global.cg)
#endif

// y_j from the shared-memory window [w0, w0 + wn) of a relabelled run when it
// holds j, else from global memory.
struct Window {
    const float* s;  // shared copy of Y[w0 .. w0 + wn)
    int w0, wn;
};

template <int S, bool WIN>
__device__ __forceinline__ void attract(float yi0, float yi1, int j, float v,
                                        const float* __restrict__ Y, const Window& win,
                                        float& a0, float& a1) {
    const unsigned off = (unsigned)(j - win.w0);
    const bool in = WIN && off < (unsigned)win.wn;
    if (S == 2) {
        float2 yj;
        if (in) yj = reinterpret_cast<const float2*>(win.s)[off];
        else yj = FITSNE_GATHER_L2_ONLY ? __ldcg(reinterpret_cast<const float2*>(Y) + j)
                                        : __ldg(reinterpret_cast<const float2*>(Y) + j);
        const float d0 = yi0 - yj.x, d1 = yi1 - yj.y;
        const float q = __fdividef(v, 1.0f + d0 * d0 + d1 * d1);
        a0 += q * d0;
        a1 += q * d1;
    } else {
        const float yj = in ? win.s[off] : (FITSNE_GATHER_L2_ONLY ? __ldcg(Y + j) : __ldg(Y + j));
        const float d0 = yi0 - yj;
        a0 += __fdividef(v, 1.0f + d0 * d0) * d0;
    }
}

template <int U>
__device__ __forceinline__ void load_slots(const int32_t* __restrict__ col,
                                           const float* __restrict__ val, int beg, int end,
                                           int lane, int (&jj)[U], float (&vv)[U]) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int e = beg + lane + 32 * u;
        jj[u] = e < end ? __ldcs(&col[e]) : 0;
        vv[u] = e < end ? __ldcs(&val[e]) : 0.0f;
    }
}

// Attraction of one row from its prefetched entries (and any beyond 32 U),
// summed over the warp.
template <int S, bool WIN, int U>
__device__ __forceinline__ void attract_row(const int32_t* __restrict__ col,
                                            const float* __restrict__ val,
                                            const float* __restrict__ Y, const Window& win,
                                            int beg, int end, float yi0, float yi1, int lane,
                                            const int (&jj)[U], const float (&vv)[U], float& a0,
                                            float& a1) {
    a0 = 0.0f;
    a1 = 0.0f;
#pragma unroll
    for (int u = 0; u < U; ++u)
        if (beg + lane + 32 * u < end) attract<S, WIN>(yi0, yi1, jj[u], vv[u], Y, win, a0, a1);
    for (int e = beg + lane + 32 * U; e < end; e += 32)
        attract<S, WIN>(yi0, yi1, __ldcs(&col[e]), __ldcs(&val[e]), Y, win, a0, a1);
    a0 = warp_sum(a0);
    if (S == 2) a1 = warp_sum(a1);
}

// A CTA takes chunks of kForceChunk = 256 consecutive points (rows of P);
// warp w of the CTA owns rows 32 w .. 32 w + 31 of the chunk. In a relabelled
// run (WIN) the CTA first copies the window of Y centred on the chunk's mean
// neighbour label into shared memory, and the attraction reads y_j there
// when the window holds j. Per 32-row block:
//  1. lane l takes point i0 + l: its row bounds, coordinates, optimizer state
//     (coalesced), its box, local coordinates and Lagrange weights, and the
//     Step 3 interpolation of the node values of its box -> F_rep;
//  2. the warp walks the 32 rows of P; each row's entries are spread over
//     the lanes, and row r + 1's entries are loaded before row r's are used;
//     the row sum lands in lane r;
//  3. lane l forms dY (or the update) of its point; stores are coalesced.
#ifndef FITSNE_FORCE_SLOTS
#define FITSNE_FORCE_SLOTS 6  // prefetched entries per lane per row
#endif
#ifndef FITSNE_FORCE_MINB
#define FITSNE_FORCE_MINB 4   // resident 256-thread blocks per SM the registers must allow
#endif

template <int S, int PP, bool STEP, bool WIN>
__global__ void __launch_bounds__(256, WIN ? 2 : FITSNE_FORCE_MINB)
force_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
             const float* __restrict__ val, const float* __restrict__ Y,
             const Params* __restrict__ params, const float4* __restrict__ hgrid, float alpha,
             float* __restrict__ dY, StepArgs sa, int64_t N,
             const int32_t* __restrict__ chunk_centre, int win_cap) {
    constexpr int U = FITSNE_FORCE_SLOTS;
    extern __shared__ float s_win[];
    const Params P = *params;
    if (P.error) return;
    const int lane = threadIdx.x % 32;
    const float fs = P.delta * P.inv_Z;
    const int n = P.n;
    Window win{s_win, 0, 0};
#ifndef FITSNE_FORCE_CONTIG
#define FITSNE_FORCE_CONTIG 0  // 1: each CTA takes a contiguous range of chunks
#endif
    const int64_t nch = (N + kForceChunk - 1) / kForceChunk;
    const int64_t c_lo = FITSNE_FORCE_CONTIG ? nch * blockIdx.x / gridDim.x : blockIdx.x;
    const int64_t c_hi = FITSNE_FORCE_CONTIG ? nch * (blockIdx.x + 1) / gridDim.x : nch;
    const int64_t c_step = FITSNE_FORCE_CONTIG ? 1 : gridDim.x;
    for (int64_t c = c_lo; c < c_hi; c += c_step) {
        if (WIN) {
            __syncthreads();  // the previous chunk's readers are done
            const int64_t wn = N < win_cap ? N : win_cap;
            int64_t w0 = (int64_t)chunk_centre[c] - wn / 2;
            if (w0 > N - wn) w0 = N - wn;
            if (w0 < 0) w0 = 0;
            w0 &= ~(int64_t)3;  // 16-byte aligned staging loads
            win.w0 = (int)w0;
            win.wn = (int)wn;
            for (int t = threadIdx.x; t < wn * S / 4; t += blockDim.x)
                reinterpret_cast<float4*>(s_win)[t] = __ldg(reinterpret_cast<const float4*>(Y + w0 * S) + t);
            for (int t = (int)(wn * S / 4) * 4 + threadIdx.x; t < wn * S; t += blockDim.x)
                s_win[t] = __ldg(Y + w0 * S + t);
            __syncthreads();
        }
        const int64_t i0 = c * kForceChunk + (threadIdx.x / 32) * 32;
        if (i0 >= N) continue;
        const int64_t i = i0 + lane;
        const bool live = i < N;
        const int nrows = (N - i0) < 32 ? (int)(N - i0) : 32;
        // 1. per-point work, one point per lane
        int rp_lo = 0, rp_hi = 0;
        float yi0 = 0.0f, yi1 = 0.0f, f0 = 0.0f, f1 = 0.0f;
        float2 us = make_float2(0.0f, 0.0f), gs = make_float2(0.0f, 0.0f);
        if (live) {
            rp_lo = __ldg(&row_ptr[i]);
            rp_hi = __ldg(&row_ptr[i + 1]);
            if (S == 2) {
                const float2 t = reinterpret_cast<const float2*>(Y)[i];
                yi0 = t.x;
                yi1 = t.y;
            } else {
                yi0 = Y[i];
            }
            if (STEP) {
                if (S == 2) {
                    us = reinterpret_cast<const float2*>(sa.uY)[i];
                    gs = reinterpret_cast<const float2*>(sa.gains)[i];
                } else {
                    us.x = sa.uY[i];
                    gs.x = sa.gains[i];
                }
            }
            // Step 3: (h_{m+1} - y(m) h_{s+2})(y_i) = delta sum_g L_g [u'_m + (j_m + 1/2 - t_m) v]
            const int l1 = interval_of(yi0, P);
            const float t1 = local_t(yi0, l1, P);
            float L1[PP];
            lagrange<PP>(t1, L1);
            if (S == 2) {
                const int l2 = interval_of(yi1, P);
                const float t2 = local_t(yi1, l2, P);
                float L2[PP];
                lagrange<PP>(t2, L2);
#pragma unroll
                for (int j1 = 0; j1 < PP; ++j1) {
                    const float4* row = hgrid + (int64_t)(l1 * PP + j1) * n + l2 * PP;
                    const float o1 = ((float)j1 + 0.5f) - t1;
#pragma unroll
                    for (int j2 = 0; j2 < PP; ++j2) {
                        const float4 h = __ldg(row + j2);  // (h1, u'1, u'2, v)
                        const float wt = L1[j1] * L2[j2];
                        const float o2 = ((float)j2 + 0.5f) - t2;
                        f0 += wt * __fmaf_rn(o1, h.w, h.y);
                        f1 += wt * __fmaf_rn(o2, h.w, h.z);
                    }
                }
            } else {
#pragma unroll
                for (int j1 = 0; j1 < PP; ++j1) {
                    const float4 h = __ldg(hgrid + l1 * PP + j1);
                    f0 += L1[j1] * __fmaf_rn(((float)j1 + 0.5f) - t1, h.w, h.y);
                }
            }
        }
        // 2. attraction, row by row, next row's entries in flight
        float A0 = 0.0f, A1 = 0.0f;
        int jA[U], jB[U];
        float vA[U], vB[U];
        {
            const int b0 = __shfl_sync(kFull, rp_lo, 0), e0 = __shfl_sync(kFull, rp_hi, 0);
            load_slots<U>(col, val, b0, e0, lane, jA, vA);
        }
        for (int r = 0; r < nrows; r += 2) {
            const int bA = __shfl_sync(kFull, rp_lo, r), eA = __shfl_sync(kFull, rp_hi, r);
            const int bB = __shfl_sync(kFull, rp_lo, r + 1), eB = __shfl_sync(kFull, rp_hi, r + 1);
            const bool hasB = r + 1 < nrows;
            if (hasB) load_slots<U>(col, val, bB, eB, lane, jB, vB);
            {
                const float y0 = __shfl_sync(kFull, yi0, r), y1 = __shfl_sync(kFull, yi1, r);
                float a0, a1;
                attract_row<S, WIN, U>(col, val, Y, win, bA, eA, y0, y1, lane, jA, vA, a0, a1);
                if (lane == r) { A0 = a0; A1 = a1; }
            }
            if (hasB) {
                if (r + 2 < nrows) {
                    const int bC = __shfl_sync(kFull, rp_lo, r + 2), eC = __shfl_sync(kFull, rp_hi, r + 2);
                    load_slots<U>(col, val, bC, eC, lane, jA, vA);
                }
                const float y0 = __shfl_sync(kFull, yi0, r + 1), y1 = __shfl_sync(kFull, yi1, r + 1);
                float a0, a1;
                attract_row<S, WIN, U>(col, val, Y, win, bB, eB, y0, y1, lane, jB, vB, a0, a1);
                if (lane == r + 1) { A0 = a0; A1 = a1; }
            }
        }
        // 3. gradient (and update) of this lane's point
        if (live) {
            const float g0 = 4.0f * (alpha * A0 + f0 * fs);
            const float g1 = (S == 2) ? 4.0f * (alpha * A1 + f1 * fs) : 0.0f;
            if (!STEP) {
                if (S == 2) reinterpret_cast<float2*>(dY)[i] = make_float2(g0, g1);
                else dY[i] = g0;
            } else {
                const float n0 = update_one(yi0, g0, us.x, gs.x, sa);
                if (S == 2) {
                    const float n1 = update_one(yi1, g1, us.y, gs.y, sa);
                    reinterpret_cast<float2*>(sa.uY)[i] = us;
                    reinterpret_cast<float2*>(sa.gains)[i] = gs;
                    reinterpret_cast<float2*>(sa.Y_new)[i] = make_float2(n0, n1);
                } else {
                    sa.uY[i] = us.x;
                    sa.gains[i] = gs.x;
                    sa.Y_new[i] = n0;
                }
            }
        }
    }
}

// ----------------------------------------------------------------------------
// KL(P || Q) = sum p log p + sum p log(1 + d^2) + (sum p) log Z over the stored
// entries (Sec. 1.1). Per-entry logarithms in FP32, all sums in FP64, reduced
// in a fixed order (per block, then by the last block).
// ----------------------------------------------------------------------------
template <int S>
__global__ void __launch_bounds__(256)
kl_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
          const float* __restrict__ val, const float* __restrict__ Y, int64_t N,
          const double* __restrict__ Z_dev, double Z_val, double* __restrict__ partial,
          unsigned* __restrict__ ticket, double* __restrict__ out) {
    const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
    const int64_t nwarp = (int64_t)gridDim.x * blockDim.x / 32;
    double acc = 0.0, psum = 0.0;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; i < N; i += nwarp) {
        float yi0, yi1 = 0.0f;
        if (S == 2) {
            float2 t = reinterpret_cast<const float2*>(Y)[i];
            yi0 = t.x;
            yi1 = t.y;
        } else {
            yi0 = Y[i];
        }
        for (int e = row_ptr[i] + lane; e < row_ptr[i + 1]; e += 32) {
            const float p = val[e];
            if (!(p > 0.0f)) continue;
            const int j = col[e];
            float d2;
            if (S == 2) {
                float2 yj = reinterpret_cast<const float2*>(Y)[j];
                float d0 = yi0 - yj.x, d1 = yi1 - yj.y;
                d2 = d0 * d0 + d1 * d1;
            } else {
                float d0 = yi0 - Y[j];
                d2 = d0 * d0;
            }
            acc += (double)p * ((double)logf(p) + (double)log1pf(d2));
            psum += (double)p;
        }
    }
    acc = warp_sum_d(acc);
    psum = warp_sum_d(psum);
    __shared__ double s_a[8], s_p[8];
    __shared__ bool s_last;
    if (lane == 0) { s_a[wid] = acc; s_p[wid] = psum; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, ps = 0.0;
        for (int k = 0; k < (int)(blockDim.x / 32); ++k) { a += s_a[k]; ps += s_p[k]; }
        partial[2 * blockIdx.x] = a;
        partial[2 * blockIdx.x + 1] = ps;
        __threadfence();
        s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    double a = 0.0, ps = 0.0;
    for (unsigned k = 0; k < gridDim.x; ++k) {
        a += __ldcg(&partial[2 * k]);
        ps += __ldcg(&partial[2 * k + 1]);
    }
    *ticket = 0u;
    const double Z = Z_dev ? __ldcg(Z_dev) : Z_val;
    *out = a + ps * log(Z);
}

// ----------------------------------------------------------------------------
// CSR check: row_ptr[0] = 0, monotone, row_ptr[N] = nnz, 0 <= col < N,
// col != row, 0 <= val < inf. Sets *flag to 1 on the first violation.
// ----------------------------------------------------------------------------
__global__ void validate_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                const float* __restrict__ val, int64_t N, int64_t nnz,
                                int32_t* __restrict__ flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const int64_t a = row_ptr[i], b = row_ptr[i + 1];
        bool bad = (a > b) || (a < 0) || (b > nnz) || (i == 0 && a != 0) || (i == N - 1 && b != nnz);
        if (!bad) {
            for (int64_t e = a; e < b; ++e) {
                const int64_t j = col[e];
                const float v = val[e];
                if (j < 0 || j >= N || j == i || !(v >= 0.0f) || isinf(v)) { bad = true; break; }
            }
        }
        if (bad) atomicExch(flag, 1);
    }
}

__global__ void fill_kernel(float* __restrict__ a, float v, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) a[i] = v;
}

// ----------------------------------------------------------------------------
// Launchers
// ----------------------------------------------------------------------------
static int grid_for(const tsne_plan* pl, int64_t items, int per_block, int per_sm) {
    int64_t b = (items + per_block - 1) / per_block;
    int64_t cap = (int64_t)pl->sm_count * per_sm;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t launch_box(tsne_plan* pl, const float* Y) {
    box_kernel<<<kBoxBlocks, kBoxThreads, 0, pl->stream>>>(
        Y, pl->N * pl->s, pl->s, pl->p, pl->n_int_fixed, pl->n_min, pl->n_int_max, pl->force_box,
        pl->force_y_min, pl->force_width, pl->force_n_int, pl->fx_shift, pl->box_partial,
        pl->tickets + 0,
        pl->params, pl->fft_table, pl->fft_of_n);
    pl->launches += 1;
    return cudaGetLastError();
}

template <int S, int PP>
static void sort_and_spread_impl(tsne_plan* pl, const float* Y) {
    const int gp = (int)((pl->N + kSortPts - 1) / kSortPts);
    const size_t hs = sizeof(int32_t) * kHistBins;
    count_kernel<S><<<gp, 256, hs, pl->stream>>>(Y, pl->N, pl->params, pl->counts, pl->w);
    scan_blocks_kernel<<<pl->scan_blocks, 1024, 0, pl->stream>>>(
        pl->counts, pl->params, pl->block_pts, pl->block_chunks, pl->tickets + 1);
    scan_boxes_kernel<S, PP><<<pl->scan_blocks, 1024, 0, pl->stream>>>(
        pl->counts, pl->params, pl->block_pts, pl->block_chunks, pl->box_start, pl->cursor,
        pl->chunk_start, pl->chunk_box, pl->N);
    scatter_kernel<S><<<gp, 256, hs, pl->stream>>>(Y, pl->N, pl->params, pl->cursor, pl->sorted_y);
    const int gs = grid_for(pl, pl->chunk_cap * 32, 256, 8);
    spread_kernel<S, PP><<<gs, 256, 0, pl->stream>>>(pl->sorted_y, pl->box_start, pl->chunk_start,
                                                     pl->chunk_box, pl->params, pl->w);
    pl->launches += 5;
}

#define FITSNE_DISPATCH(S_, FN, ...)                                   \
    switch (pl->p) {                                                   \
        case 2: FN<S_, 2>(__VA_ARGS__); break;                         \
        case 3: FN<S_, 3>(__VA_ARGS__); break;                         \
        case 4: FN<S_, 4>(__VA_ARGS__); break;                         \
        default: FN<S_, 5>(__VA_ARGS__); break;                        \
    }

cudaError_t launch_sort_and_spread(tsne_plan* pl, const float* Y) {
    if (pl->s == 2) { FITSNE_DISPATCH(2, sort_and_spread_impl, pl, Y); }
    else { FITSNE_DISPATCH(1, sort_and_spread_impl, pl, Y); }
    return cudaGetLastError();
}

template <int S, int PP, bool STEP, bool WIN>
static void force_impl(tsne_plan* pl, const tsne_csr& P, const float* Y, float alpha, float* dY,
                       StepArgs sa) {
    if (WIN) {
        const int64_t nch = (pl->N + kForceChunk - 1) / kForceChunk;
        const int ctas = (int)std::min<int64_t>(nch, 2LL * pl->sm_count);
        const int cap = FITSNE_WIN_BYTES / (int)(sizeof(float) * S);
        force_kernel<S, PP, STEP, true><<<ctas, 256, FITSNE_WIN_BYTES, pl->stream>>>(
            P.row_ptr, P.col, P.val, Y, pl->params, pl->hgrid, alpha, dY, sa, pl->N,
            pl->chunk_centre, cap);
    } else {
        const int g = grid_for(pl, pl->N, 256, 8);
        force_kernel<S, PP, STEP, false><<<g, 256, 0, pl->stream>>>(
            P.row_ptr, P.col, P.val, Y, pl->params, pl->hgrid, alpha, dY, sa, pl->N, nullptr, 0);
    }
    pl->launches += 1;
}

template <int S, int PP>
static void gradient_impl(tsne_plan* pl, const tsne_csr& P, const float* Y, float alpha,
                          float* dY) {
    force_impl<S, PP, false, false>(pl, P, Y, alpha, dY, StepArgs{});
}

#ifndef FITSNE_RELABEL_WINDOW
#define FITSNE_RELABEL_WINDOW 0  // 1: relabelled runs read y_j through a shared-memory window
#endif

template <int S, int PP>
static void step_impl(tsne_plan* pl, const tsne_csr& P, const float* Y, float alpha,
                      const StepArgs& sa) {
    if (pl->reordered && FITSNE_RELABEL_WINDOW) force_impl<S, PP, true, true>(pl, P, Y, alpha, nullptr, sa);
    else force_impl<S, PP, true, false>(pl, P, Y, alpha, nullptr, sa);
}

template <int S, int PP>
static cudaError_t configure_impl() {
    return cudaFuncSetAttribute(force_kernel<S, PP, true, true>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, FITSNE_WIN_BYTES);
}

cudaError_t force_configure(tsne_plan* pl) {
    cudaError_t e = cudaSuccess;
    switch (pl->p * 10 + pl->s) {
        case 21: e = configure_impl<1, 2>(); break;
        case 22: e = configure_impl<2, 2>(); break;
        case 31: e = configure_impl<1, 3>(); break;
        case 32: e = configure_impl<2, 3>(); break;
        case 41: e = configure_impl<1, 4>(); break;
        case 42: e = configure_impl<2, 4>(); break;
        case 51: e = configure_impl<1, 5>(); break;
        default: e = configure_impl<2, 5>(); break;
    }
    return e;
}

cudaError_t launch_gradient(tsne_plan* pl, const tsne_csr& P, const float* Y, float alpha,
                            float* dY) {
    if (pl->s == 2) { FITSNE_DISPATCH(2, gradient_impl, pl, P, Y, alpha, dY); }
    else { FITSNE_DISPATCH(1, gradient_impl, pl, P, Y, alpha, dY); }
    return cudaGetLastError();
}

cudaError_t launch_step(tsne_plan* pl, const tsne_csr& P, const float* Y, float* Y_new,
                        float* uY, float* gains, float alpha, float momentum, float lr,
                        float min_gain, float gain_inc, float gain_dec) {
    StepArgs sa{Y_new, uY, gains, momentum, lr, min_gain, gain_inc, gain_dec};
    if (pl->s == 2) { FITSNE_DISPATCH(2, step_impl, pl, P, Y, alpha, sa); }
    else { FITSNE_DISPATCH(1, step_impl, pl, P, Y, alpha, sa); }
    return cudaGetLastError();
}

cudaError_t launch_kl_raw(const tsne_csr& P, const float* Y, int64_t N, int s,
                          const double* Z_dev, double Z_val, double* partial, unsigned* ticket,
                          double* out, int blocks, cudaStream_t stream) {
    if (s == 2)
        kl_kernel<2><<<blocks, 256, 0, stream>>>(P.row_ptr, P.col, P.val, Y, N, Z_dev, Z_val,
                                                 partial, ticket, out);
    else
        kl_kernel<1><<<blocks, 256, 0, stream>>>(P.row_ptr, P.col, P.val, Y, N, Z_dev, Z_val,
                                                 partial, ticket, out);
    return cudaGetLastError();
}

cudaError_t launch_kl(tsne_plan* pl, const tsne_csr& P, const float* Y) {
    const int g = 4 * pl->sm_count;  // kl_partial holds 2 doubles per block
    pl->launches += 1;
    return launch_kl_raw(P, Y, pl->N, pl->s, &pl->params->Z, 0.0, pl->kl_partial, pl->tickets + 3,
                         pl->kl_out_dev, g, pl->stream);
}

cudaError_t launch_validate(tsne_plan* pl, const tsne_csr& P) {
    const int g = grid_for(pl, pl->N, 256, 8);
    validate_kernel<<<g, 256, 0, pl->stream>>>(P.row_ptr, P.col, P.val, pl->N, P.nnz,
                                               pl->valid_flag);
    pl->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_fill(tsne_plan* pl, float* a, float v, int64_t n) {
    const int g = grid_for(pl, n, 256, 8);
    fill_kernel<<<g, 256, 0, pl->stream>>>(a, v, n);
    pl->launches += 1;
    return cudaGetLastError();
}

}  // namespace fitsne
