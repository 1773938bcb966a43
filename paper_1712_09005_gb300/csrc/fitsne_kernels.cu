// Per-point and per-entry kernels of the FIt-SNE gradient on sm_103a, in
// job-table form (every launch serves all jobs of a table; see
// fitsne_internal.cuh):
//   box_kernel      bounding box, interval rule and schedule values
//                   (Sec. 2.2, 2.4, 2.5; Sec. 1.2 and Sec. 4 exaggeration)
//   count/scatter   counting sort of the points by box (the "points in I_l"
//                   loops of Algorithm 1)
//   scan kernels    box offsets and the spread work list
//   spread_kernel   Step 1: w_m = sum_{y_i in I_l} L_m(y_i) q_i per box
//   force_kernel    attraction over the CSR rows (Sec. 3) fused with Step 3
//                   (interpolate back), the Appendix assembly of F_rep and,
//                   for a descent step, the gains/momentum update
//   advance_kernel  moves each stepping job to its next iteration
//   kl_kernel       KL(P || Q) of Sec. 1.1 with FP64 sums
// No kernel uses floating-point atomics: the spread sums are integers.
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

__device__ __forceinline__ bool schedule_active(const Job& J, int ignore_schedule) {
    return ignore_schedule || J.mode == kModeGradient || J.dyn->iter < J.iter_end;
}

// Bounding-box work items of a job: one per 1024 coordinates, at most kBoxBlocks.
__device__ __forceinline__ int box_items(const Job& J, int s, int ignore_schedule) {
    if (!schedule_active(J, ignore_schedule)) return 1;
    const int64_t c = (J.N * s + 1023) / 1024;
    return (int)(c < 1 ? 1 : (c > kBoxBlocks ? kBoxBlocks : c));
}

__device__ __forceinline__ int sort_items(const Job& J) {
    const Params* P = J.params;
    return job_live(*P) ? (int)((J.N + kSortPts - 1) / kSortPts) : 0;
}

__device__ __forceinline__ int scan_items(const Job& J) {
    const Params* P = J.params;
    return job_live(*P) ? (P->n_boxes + kScanBlock - 1) / kScanBlock : 0;
}

}  // namespace

// The box, interval count, node spacing, FFT length and schedule values of
// a job's iteration `it` (Y in ybuf[cur]) from the exact min / max of its
// coordinates (Sec. 2.2, 2.4, 2.5; Sec. 1.2 and Sec. 4 exaggeration). The
// FP32 rule matches the oracle's bit for bit. One thread.
__device__ void box_finish(const Job& J, int s, int p, const Tables& tab, int ignore_schedule,
                           float lo, float hi, bool any_bad, int cur, int it) {
    Params P;
    P.error = __ldcg(&J.params->error);
    if (any_bad) { P.error = TSNE_ERR_NONFINITE; lo = 0.0f; hi = 1.0f; }
    float y_min, width;
    int n_int;
    if (J.force_box) {
        y_min = J.force_y_min;
        width = J.force_width;
        n_int = J.force_n_int;
    } else {
        y_min = lo;
        width = __fsub_rn(hi, lo);
        if (!(width > 0.0f)) width = 1.0f;
        if (J.n_int_fixed > 0) {
            n_int = J.n_int_fixed;
        } else {
            float c = ceilf(width);
            if (c > (float)J.n_int_max) c = (float)J.n_int_max;
            n_int = (int)c;
            if (n_int < J.n_min) n_int = J.n_min;
            if (n_int > J.n_int_max) n_int = J.n_int_max;
            if (J.n_int_table) n_int = J.n_int_table[n_int];
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
    P.fx_shift = J.fx_shift;
    P.fx_scale = ldexpf(1.0f, J.fx_shift);
    P.fx_inv = ldexpf(1.0f, -J.fx_shift);
    P.n = p * n_int;
    P.n_boxes = (s == 2) ? n_int * n_int : n_int;
    const int idx = tab.fft_of_n[P.n];
    P.fft_idx = idx;
    P.L = tab.fft[idx].L;
    P.p_f = (float)p;
    P.n_chunks = 0;
    P.Z = 0.0;
    P.inv_Z = 0.0f;
    P.active = 1;
    P.cur = cur;
    P.pad = 0;
    if (J.mode == kModeStep && !ignore_schedule) {
        float a = 1.0f;
        if (it < J.early_iters) a = J.early_alpha;
        else if (J.late_iters > 0 && it >= J.n_iter - J.late_iters) a = J.late_alpha;
        P.alpha = a;
        P.momentum = it < J.mom_switch_iter ? J.momentum_early : J.momentum_late;
    } else {
        P.alpha = J.alpha;
        P.momentum = 0.0f;
    }
    *J.params = P;
    J.dyn->error = P.error;
}

// ----------------------------------------------------------------------------
// Bounding box: per-item min/max, then the last item of a job to finish
// derives the box, N_int, node spacing, FFT length and the iteration's
// schedule values (Sec. 2.2, 2.4, 2.5). The FP32 rule matches the oracle's
// bit for bit. A job past its schedule gets one item that marks it inactive.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(kBoxThreads)
box_kernel(const Job* __restrict__ jobs, int njobs, int s, int p, int ignore_schedule,
           Tables tab, int advance_first) {
    __shared__ int32_t s_start[kMaxJobs + 1];
    __shared__ float s_lo[kBoxThreads / 32], s_hi[kBoxThreads / 32];
    __shared__ bool s_last;
    const int total = split_jobs(jobs, njobs, s_start,
                                 [&](const Job& J) { return box_items(J, s, ignore_schedule); });
    const int wid = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int j = job_of(s_start, njobs, item);
        const Job& J = jobs[j];
        const int k = item - s_start[j], nk = s_start[j + 1] - s_start[j];
        if (!schedule_active(J, ignore_schedule)) {
            if (threadIdx.x == 0) J.params->active = 0;
            continue;  // uniform over the block
        }
        // advance_first: the previous step's move to the next iteration (new Y
        // current, schedule index + 1) happens here instead of in a kernel of
        // its own; every item reads the advanced values, the last one stores them
        const int adv = (advance_first && J.mode == kModeStep) ? 1 : 0;
        const int cur = J.dyn->cur ^ adv;
        const int it_now = J.dyn->iter + adv;
        const float* __restrict__ Y = J.ybuf[cur];
        const int64_t count = J.N * s;
        float lo = INFINITY, hi = -INFINITY;
        int bad = 0;
        const int64_t stride = (int64_t)nk * blockDim.x;
        const int64_t k0 = (int64_t)k * blockDim.x + threadIdx.x;
        if ((reinterpret_cast<uintptr_t>(Y) & 15) == 0) {
            const int64_t n4 = count / 4;
            const float4* Y4 = reinterpret_cast<const float4*>(Y);
#pragma unroll 4
            for (int64_t q = k0; q < n4; q += stride) {
                float4 v = __ldg(&Y4[q]);
                bad |= !isfinite(v.x) | !isfinite(v.y) | !isfinite(v.z) | !isfinite(v.w);
                lo = fminf(lo, fminf(fminf(v.x, v.y), fminf(v.z, v.w)));
                hi = fmaxf(hi, fmaxf(fmaxf(v.x, v.y), fmaxf(v.z, v.w)));
            }
            for (int64_t q = n4 * 4 + k0; q < count; q += stride) {
                float v = Y[q];
                bad |= !isfinite(v);
                lo = fminf(lo, v);
                hi = fmaxf(hi, v);
            }
        } else {
            for (int64_t q = k0; q < count; q += stride) {
                float v = Y[q];
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
        bad = __syncthreads_or(bad);
        if (lane == 0) { s_lo[wid] = lo; s_hi[wid] = hi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int i = 1; i < kBoxThreads / 32; ++i) { lo = fminf(lo, s_lo[i]); hi = fmaxf(hi, s_hi[i]); }
            J.box_partial[2 * k] = bad ? NAN : lo;
            J.box_partial[2 * k + 1] = hi;
            __threadfence();
            s_last = (atomicAdd(&J.tickets[0], 1u) == (unsigned)nk - 1);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            // the last item of the job reduces the job's partials
            int bad_p = 0;
            lo = INFINITY;
            hi = -INFINITY;
            for (int i = threadIdx.x; i < nk; i += blockDim.x) {
                float a = __ldcg(&J.box_partial[2 * i]), b = __ldcg(&J.box_partial[2 * i + 1]);
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
            if (threadIdx.x == 0) {
                for (int i = 0; i < kBoxThreads / 32; ++i) { lo = fminf(lo, s_lo[i]); hi = fmaxf(hi, s_hi[i]); }
                J.tickets[0] = 0u;
                if (adv) {
                    J.dyn->cur = cur;
                    J.dyn->iter = it_now;
                }
                box_finish(J, s, p, tab, ignore_schedule, lo, hi, any_bad, cur, it_now);
            }
        }
        __syncthreads();  // shared state of this item is consumed
    }
}

// ----------------------------------------------------------------------------
// Counting sort by box: histogram (warp-aggregated integer atomics), scan,
// scatter. Points of one box end up contiguous in sorted_y; their order
// within the box is not fixed, which the integer spread sums do not see.
// ----------------------------------------------------------------------------
// Each work item takes kSortPts consecutive points of one job. With at most
// kHistBins boxes the block first counts in a shared-memory histogram and
// touches the global counters once per box it met, which keeps boxes holding
// many points (tight clusters) from serialising on one global atomic; with
// more boxes (each then holds few points) it uses the global counters
// directly. The items of a job also zero its spread grids.
template <int S>
__global__ void __launch_bounds__(256)
count_kernel(const Job* __restrict__ jobs, int njobs) {
    extern __shared__ int32_t hist[];
    __shared__ int32_t s_start[kMaxJobs + 1];
    const int total = split_jobs(jobs, njobs, s_start, [](const Job& J) { return sort_items(J); });
    const int lane = threadIdx.x % 32;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int j = job_of(s_start, njobs, item);
        const Job& J = jobs[j];
        const int k = item - s_start[j], nk = s_start[j + 1] - s_start[j];
        const Params P = *J.params;
        const float* __restrict__ Y = J.ybuf[P.cur];
        int32_t* __restrict__ counts = J.counts;
        const int64_t N = J.N;
        {  // the spread grids of this iteration start at zero
            long long* __restrict__ w = J.w;
            const int64_t G = (S == 2) ? (int64_t)P.n * P.n : P.n;
            const int64_t stride = (int64_t)nk * blockDim.x;
            for (int64_t g = (int64_t)k * blockDim.x + threadIdx.x; g < (S + 1) * G; g += stride)
                w[g] = 0;
        }
        const int nb = P.n_boxes;
        const bool local = nb <= kHistBins;
        if (local) {
            for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0;
            __syncthreads();
        }
        const int64_t p0 = (int64_t)k * kSortPts;
        for (int q = 0; q < kSortPts / 256; ++q) {
            const int64_t i = p0 + q * 256 + threadIdx.x;
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
        __syncthreads();
    }
}

// Same partition: the block counts its points per box, reserves one range
// per box in the global cursors, then places each point at its box's range
// plus its rank inside the block.
template <int S>
__global__ void __launch_bounds__(256)
scatter_kernel(const Job* __restrict__ jobs, int njobs) {
    extern __shared__ int32_t hist[];
    __shared__ int32_t s_start[kMaxJobs + 1];
    constexpr int K = kSortPts / 256;
    const int total = split_jobs(jobs, njobs, s_start, [](const Job& J) { return sort_items(J); });
    const int lane = threadIdx.x % 32;
    const unsigned lt = (1u << lane) - 1u;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int j = job_of(s_start, njobs, item);
        const Job& J = jobs[j];
        const int k = item - s_start[j];
        const Params P = *J.params;
        const float* __restrict__ Y = J.ybuf[P.cur];
        int32_t* __restrict__ cursor = J.cursor;
        float* __restrict__ sorted_y = J.sorted_y;
        const int64_t N = J.N;
        const int nb = P.n_boxes;
        const bool local = nb <= kHistBins;
        const int64_t p0 = (int64_t)k * kSortPts;
        int box[K];
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const int64_t i = p0 + q * 256 + threadIdx.x;
            box[q] = (i < N) ? box_of<S>(Y, i, P) : -1;
        }
        if (local) {
            for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0;
            __syncthreads();
#pragma unroll
            for (int q = 0; q < K; ++q) {
                const unsigned peers = __match_any_sync(kFull, box[q]);
                if (box[q] >= 0 && lane == __ffs(peers) - 1) atomicAdd(&hist[box[q]], __popc(peers));
            }
            __syncthreads();
            for (int b = threadIdx.x; b < nb; b += blockDim.x)
                if (hist[b]) hist[b] = atomicAdd(&cursor[b], hist[b]);
            __syncthreads();
        }
        int32_t* dst_cursor = local ? hist : cursor;
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const unsigned peers = __match_any_sync(kFull, box[q]);
            const int leader = __ffs(peers) - 1;
            int pos = 0;
            if (box[q] >= 0 && lane == leader) pos = atomicAdd(&dst_cursor[box[q]], __popc(peers));
            pos = __shfl_sync(kFull, pos, leader) + __popc(peers & lt);
            if (box[q] >= 0) {
                const int64_t i = p0 + q * 256 + threadIdx.x;
                if (S == 2)
                    reinterpret_cast<float2*>(sorted_y)[pos] = reinterpret_cast<const float2*>(Y)[i];
                else
                    sorted_y[pos] = Y[i];
            }
        }
        __syncthreads();
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

// Pass 1: per-item totals of points and of spread chunks (ceil(count/chunk));
// the last item of a job turns them into exclusive offsets.
__global__ void __launch_bounds__(1024)
scan_blocks_kernel(const Job* __restrict__ jobs, int njobs) {
    __shared__ int32_t s_start[kMaxJobs + 1];
    __shared__ int sw[32];
    __shared__ bool s_last;
    const int total = split_jobs(jobs, njobs, s_start, [](const Job& J) { return scan_items(J); });
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int j = job_of(s_start, njobs, item);
        const Job& J = jobs[j];
        const int k = item - s_start[j], nk = s_start[j + 1] - s_start[j];
        const int nb = J.params->n_boxes;
        const int ch = J.chunk;
        const int32_t* __restrict__ counts = J.counts;
        const int base = k * kScanBlock + threadIdx.x * 2;
        const int c0 = base < nb ? counts[base] : 0;
        const int c1 = base + 1 < nb ? counts[base + 1] : 0;
        const int pts = c0 + c1;
        const int chk = (c0 + ch - 1) / ch + (c1 + ch - 1) / ch;
        int tp, tc;
        block_exclusive_scan(pts, sw, tp);
        block_exclusive_scan(chk, sw, tc);
        if (threadIdx.x == 0) {
            J.block_pts[k] = tp;
            J.block_chunks[k] = tc;
            __threadfence();
            s_last = (atomicAdd(&J.tickets[1], 1u) == (unsigned)nk - 1);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            int carry_p = 0, carry_c = 0;
            for (int start = 0; start < nk; start += blockDim.x) {
                const int i = start + threadIdx.x;
                const int vp = i < nk ? __ldcg(&J.block_pts[i]) : 0;
                const int vc = i < nk ? __ldcg(&J.block_chunks[i]) : 0;
                int sp, sc;
                const int ep = block_exclusive_scan(vp, sw, sp);
                const int ec = block_exclusive_scan(vc, sw, sc);
                if (i < nk) {
                    J.block_pts[i] = carry_p + ep;
                    J.block_chunks[i] = carry_c + ec;
                }
                carry_p += sp;
                carry_c += sc;
            }
            if (threadIdx.x == 0) {
                J.params->n_chunks = carry_c;
                J.tickets[1] = 0u;
            }
        }
        __syncthreads();
    }
}

// Pass 2: box offsets, scatter cursors, chunk -> box table; resets the counts
// for the next iteration. Each warp writes the chunk entries of its 64 boxes
// with its lanes in parallel (a box holding many points has many chunks).
__global__ void __launch_bounds__(1024)
scan_boxes_kernel(const Job* __restrict__ jobs, int njobs) {
    __shared__ int32_t s_start[kMaxJobs + 1];
    __shared__ int sw[32];
    const int total = split_jobs(jobs, njobs, s_start, [](const Job& J) { return scan_items(J); });
    const int lane = threadIdx.x % 32;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int j = job_of(s_start, njobs, item);
        const Job& J = jobs[j];
        const int k = item - s_start[j];
        const int nb = J.params->n_boxes;
        const int ch = J.chunk;
        int32_t* __restrict__ counts = J.counts;
        int32_t* __restrict__ box_start = J.box_start;
        int32_t* __restrict__ cursor = J.cursor;
        int32_t* __restrict__ chunk_start = J.chunk_start;
        int32_t* __restrict__ chunk_box = J.chunk_box;
        const int base = k * kScanBlock + threadIdx.x * 2;
        int c[2] = {base < nb ? counts[base] : 0, base + 1 < nb ? counts[base + 1] : 0};
        int kk[2] = {(c[0] + ch - 1) / ch, (c[1] + ch - 1) / ch};
        int tp, tc;
        int ep = block_exclusive_scan(c[0] + c[1], sw, tp) + J.block_pts[k];
        int ec = block_exclusive_scan(kk[0] + kk[1], sw, tc) + J.block_chunks[k];
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
                    box_start[nb] = (int32_t)J.N;
                    chunk_start[nb] = ec + kk[u];
                }
            }
            ep += c[u];
            ec += kk[u];
        }
        // chunk -> box entries: the warp visits its lanes' boxes one by one
        for (int src = 0; src < 32; ++src) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int b = __shfl_sync(kFull, base + u, src);
                const int kb = __shfl_sync(kFull, kk[u], src);
                const int eb = __shfl_sync(kFull, ecb[u], src);
                if (b < nb)
                    for (int q = lane; q < kb; q += 32) chunk_box[eb + q] = b;
            }
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------
// Step 1 (spread): one warp per chunk of at most J.chunk points of one box.
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
spread_kernel(const Job* __restrict__ jobs, int njobs) {
    constexpr int NODES = (S == 2) ? PP * PP : PP;
    constexpr int NVAL = (S + 1) * NODES;
    constexpr int NV = (NVAL + 31) / 32 * 32;
    __shared__ int32_t s_start[kMaxJobs + 1];
    const int total = split_jobs(jobs, njobs, s_start, [](const Job& J) {
        const Params* P = J.params;
        return job_live(*P) ? P->n_chunks : 0;
    });
    const int lane = threadIdx.x % 32;
    const int nwarp = gridDim.x * blockDim.x / 32;
    for (int q = (blockIdx.x * blockDim.x + threadIdx.x) / 32; q < total; q += nwarp) {
        const int jb = job_of(s_start, njobs, q);
        const Job& J = jobs[jb];
        const Params P = *J.params;
        const int ql = q - s_start[jb];
        const int chunk = J.chunk;
        const float* __restrict__ sorted_y = J.sorted_y;
        long long* __restrict__ w = J.w;
        const int n = P.n;
        const int64_t G = (S == 2) ? (int64_t)n * n : n;
        const float sc = P.fx_scale;
        const int box = J.chunk_box[ql];
        const int bs = J.box_start[box];
        const int cnt = J.box_start[box + 1] - bs;
        const int ci = ql - J.chunk_start[box];
        const int start = bs + ci * chunk;
        const int len = min(chunk, cnt - ci * chunk);
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
                for (int jj = 0; jj < PP; ++jj) {
                    e1[jj] = t1 - ((float)jj + 0.5f);
                    e2[jj] = t2 - ((float)jj + 0.5f);
                }
            } else {
                const float t1 = local_t(sorted_y[start + k], bx, P);
                lagrange<PP>(t1, L1);
#pragma unroll
                for (int jj = 0; jj < PP; ++jj) e1[jj] = t1 - ((float)jj + 0.5f);
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
        const bool multi = cnt > chunk;
#pragma unroll
        for (int g = 0; g < NV / 32; ++g) {
            const int v = g * 32 + lane;
            if (v < NVAL) {
                const int chn = v / NODES, node = v % NODES;
                const int j1 = (S == 2) ? node / PP : node;
                const int j2 = (S == 2) ? node % PP : 0;
                const int64_t gi = (S == 2) ? (int64_t)(bx * PP + j1) * n + (by * PP + j2)
                                            : (int64_t)(bx * PP + j1);
                long long* dst = &w[chn * G + gi];
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

// One attraction term p_ij (y_i - y_j) / (1 + |y_i - y_j|^2) added to (a0, a1).
template <int S>
__device__ __forceinline__ void attract(float yi0, float yi1, int j, float v,
                                        const float* __restrict__ Y, float& a0, float& a1) {
    if (S == 2) {
        const float2 yj = __ldg(reinterpret_cast<const float2*>(Y) + j);
        const float d0 = yi0 - yj.x, d1 = yi1 - yj.y;
        const float q = __fdividef(v, 1.0f + d0 * d0 + d1 * d1);
        a0 += q * d0;
        a1 += q * d1;
    } else {
        const float d0 = yi0 - __ldg(Y + j);
        a0 += __fdividef(v, 1.0f + d0 * d0) * d0;
    }
}

// Rows are taken kRowLanes lanes at a time (32 / kRowLanes rows per warp
// step; 32 measured fastest on GB300). Entries of one row [beg, end) are
// shared out over its lanes in windows of 4 kRowLanes: lane g of the row's
// group takes entries beg + 4 kRowLanes w + kRowLanes q + g (q = 0..3, those
// below end) of window w = 0, 1, ... in that order, and the group's partial
// sums are combined by an xor tree over its lanes. Each load of col and val
// is then one contiguous run of kRowLanes entries (a lane stride of 4 bytes,
// about 5 sectors per 32 entries, where a stride of 16 bytes touched 16).
// The order depends only on the row's own entries (not on where the row sits
// in memory), so every force kernel, and a relabelled copy of P whose rows
// keep their entry order, give bitwise equal row sums. RowBuf holds the first
// W windows of a lane's row, loaded ahead of use.
#ifndef FITSNE_ROW_LANES
#define FITSNE_ROW_LANES 32
#endif
constexpr int kRowLanes = FITSNE_ROW_LANES;
static_assert(kRowLanes == 8 || kRowLanes == 16 || kRowLanes == 32, "lanes per row");

// Loads of the CSR stream, read once per iteration: no L1 allocation, so
// the SM's L1 holds the gathered coordinates (slightly faster than
// evict-first streaming loads, which still pass through L1).
template <typename T>
__device__ __forceinline__ T ld_csr(const T* p) {
    static_assert(sizeof(T) == 4, "32-bit CSR entries");
    unsigned r;
    asm volatile("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(r) : "l"(p));
    T v;
    memcpy(&v, &r, 4);
    return v;
}

template <int W>
struct RowBuf {
    int c[4 * W];
    float v[4 * W];
    int base;  // beg + g: this lane's first entry
    int rem;   // end - base: the lane takes offsets 4 kRowLanes w + kRowLanes q below rem
};

// Masked streaming loads of the first W windows of a row; g: the lane's
// index in its row group.
template <int W>
__device__ __forceinline__ void row_load(RowBuf<W>& b, const int32_t* __restrict__ col,
                                         const float* __restrict__ val, int beg, int end, int g) {
    b.base = beg + g;
    b.rem = end - b.base;
    const int32_t* __restrict__ cp = col + b.base;
    const float* __restrict__ vp = val + b.base;
#pragma unroll
    for (int w = 0; w < W; ++w)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int off = 4 * kRowLanes * w + kRowLanes * q;
            const bool in = off < b.rem;
            b.c[4 * w + q] = in ? ld_csr(cp + off) : 0;
            b.v[4 * w + q] = in ? ld_csr(vp + off) : 0.0f;
        }
}

// This lane's share of the attraction of the row held in b (and of the
// row's windows beyond W), not yet combined over the row's lanes.
template <int S, int W>
__device__ __forceinline__ void row_attract(const RowBuf<W>& b, const int32_t* __restrict__ col,
                                            const float* __restrict__ val,
                                            const float* __restrict__ Y, float yi0, float yi1,
                                            float& a0, float& a1) {
    a0 = 0.0f;
    a1 = 0.0f;
    const int32_t* __restrict__ cp = col + b.base;
    const float* __restrict__ vp = val + b.base;
    // windows past the buffered ones: each window's col/val loads are issued
    // one window ahead of its gathers (the first before the buffered
    // windows' gathers), so the CSR latency overlaps the gather latency
    // (0.432 -> 0.409 ms per launch at N = 1M; holding more windows per row,
    // or more rows in flight at 3 blocks per SM, measured slower)
    int cn[4];
    float vn[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int off = 4 * kRowLanes * W + kRowLanes * q;
        const bool in = off < b.rem;
        cn[q] = in ? ld_csr(cp + off) : 0;
        vn[q] = in ? ld_csr(vp + off) : 0.0f;
    }
#pragma unroll
    for (int w = 0; w < W; ++w)
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (4 * kRowLanes * w + kRowLanes * q < b.rem)
                attract<S>(yi0, yi1, b.c[4 * w + q], b.v[4 * w + q], Y, a0, a1);
    for (int wb = 4 * kRowLanes * W; wb < b.rem; wb += 4 * kRowLanes) {
        int c[4];
        float v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            c[q] = cn[q];
            v[q] = vn[q];
            const int off = wb + 4 * kRowLanes + kRowLanes * q;
            const bool in = off < b.rem;
            cn[q] = in ? ld_csr(cp + off) : 0;
            vn[q] = in ? ld_csr(vp + off) : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (wb + kRowLanes * q < b.rem) attract<S>(yi0, yi1, c[q], v[q], Y, a0, a1);
    }
}

// Sum over the lanes of a row group (xor tree inside aligned groups).
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = kRowLanes / 2; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

#ifndef FITSNE_FORCE_WINDOWS
#define FITSNE_FORCE_WINDOWS 1  // windows of a row loaded ahead
#endif
#ifndef FITSNE_FORCE_DEPTH
#define FITSNE_FORCE_DEPTH 2    // row steps whose windows are in flight
#endif
#ifndef FITSNE_FORCE_MINB
#define FITSNE_FORCE_MINB 4     // resident 256-thread blocks per SM the registers must allow
#endif

// Points i0 .. i0 + 31 (fewer at the end) of job J, one warp:
//  1. lane l takes point i0 + l: its row bounds, coordinates, its box, local
//     coordinates and Lagrange weights, and the Step 3 interpolation of the
//     node values of its box -> F_rep;
//  2. the warp walks the 32 rows of P; each row's entries are spread over
//     the lanes, and row r + 1's entries are loaded before row r's are used;
//     the row sum lands in lane r;
//  3. lane l forms dY (or the update) of its point; the job's output pointers
//     and schedule values are read only now; stores are coalesced.
template <int S, int PP, bool STEP>
__device__ __forceinline__ void force_block(const Job& J, const Params* __restrict__ Pp,
                                            const float* __restrict__ Y, int64_t i0, int64_t N,
                                            int lane) {
    constexpr int W = FITSNE_FORCE_WINDOWS;
    constexpr int DEPTH = FITSNE_FORCE_DEPTH;
    const int32_t* __restrict__ col = J.col;
    const float* __restrict__ val = J.val;
    const int64_t i = i0 + lane;
    const bool live = i < N;
    const int nrows = (N - i0) < 32 ? (int)(N - i0) : 32;
    // 1. per-point work, one point per lane
    int rp_lo = 0, rp_hi = 0;
    float yi0 = 0.0f, yi1 = 0.0f, f0 = 0.0f, f1 = 0.0f;
    if (live) {
        const int32_t* __restrict__ row_ptr = J.row_ptr;
        rp_lo = __ldg(&row_ptr[i]);
        rp_hi = __ldg(&row_ptr[i + 1]);
        if (S == 2) {
            const float2 t = reinterpret_cast<const float2*>(Y)[i];
            yi0 = t.x;
            yi1 = t.y;
        } else {
            yi0 = Y[i];
        }
        // Step 3: (h_{m+1} - y(m) h_{s+2})(y_i) = delta sum_g L_g [u'_m + (j_m + 1/2 - t_m) v]
        const Params& P = *Pp;
        const float4* __restrict__ hgrid = J.hgrid;
        const int n = P.n;
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
    // 2. attraction: each warp step takes 32 / kRowLanes rows (lane group g
    //    of the step works on row step * RPW + lane / kRowLanes); DEPTH steps'
    //    entries are in flight; a row's sum is handed to the lane of its point
    constexpr int RPW = 32 / kRowLanes;
    const int sub = lane / kRowLanes, g = lane % kRowLanes;
    const int nsteps = (nrows + RPW - 1) / RPW;
    float A0 = 0.0f, A1 = 0.0f;
    RowBuf<W> buf[DEPTH];
#pragma unroll
    for (int d = 0; d < DEPTH; ++d) {
        const int r = d * RPW + sub;
        const int rs = r < nrows ? r : 0;
        const int bg = __shfl_sync(kFull, rp_lo, rs), en = __shfl_sync(kFull, rp_hi, rs);
        if (d < nsteps) row_load<W>(buf[d], col, val, bg, r < nrows ? en : bg, g);
    }
    for (int s0 = 0; s0 < nsteps; s0 += DEPTH) {
#pragma unroll
        for (int d = 0; d < DEPTH; ++d) {
            const int st = s0 + d;
            if (st < nsteps) {
                const int r = st * RPW + sub;
                const int rs = r < nrows ? r : 0;
                const float y0 = __shfl_sync(kFull, yi0, rs), y1 = __shfl_sync(kFull, yi1, rs);
                float a0, a1;
                row_attract<S, W>(buf[d], col, val, Y, y0, y1, a0, a1);
                a0 = group_sum(a0);
                if (S == 2) a1 = group_sum(a1);
                const int from = (lane - st * RPW) * kRowLanes;  // group of this lane's row
                const float t0 = __shfl_sync(kFull, a0, from & 31), t1 = __shfl_sync(kFull, a1, from & 31);
                if (lane >= st * RPW && lane < st * RPW + RPW) { A0 = t0; A1 = t1; }
                const int sn = st + DEPTH;
                if (sn < nsteps) {
                    const int rn = sn * RPW + sub;
                    const int rns = rn < nrows ? rn : 0;
                    const int bg = __shfl_sync(kFull, rp_lo, rns), en = __shfl_sync(kFull, rp_hi, rns);
                    row_load<W>(buf[d], col, val, bg, rn < nrows ? en : bg, g);
                }
            }
        }
    }
    // 3. gradient (and update) of this lane's point
    if (live) {
        const Params& P = *Pp;
        const float fs = P.delta * P.inv_Z;
        const float alpha = P.alpha;
        const float g0 = 4.0f * (alpha * A0 + f0 * fs);
        const float g1 = (S == 2) ? 4.0f * (alpha * A1 + f1 * fs) : 0.0f;
        if (!STEP) {
            float* __restrict__ dY = J.dY;
            if (S == 2) reinterpret_cast<float2*>(dY)[i] = make_float2(g0, g1);
            else dY[i] = g0;
        } else {
            const StepArgs sa{J.ybuf[P.cur ^ 1], J.uY, J.gains, P.momentum, J.lr, J.min_gain,
                              J.gain_inc, J.gain_dec};
            float2 us, gs;
            if (S == 2) {
                us = reinterpret_cast<const float2*>(sa.uY)[i];
                gs = reinterpret_cast<const float2*>(sa.gains)[i];
            } else {
                us = make_float2(sa.uY[i], 0.0f);
                gs = make_float2(sa.gains[i], 0.0f);
            }
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

// A work item is a chunk of kForceChunk = 256 consecutive points (rows of P)
// of one job; warp w of the CTA owns rows 32 w .. 32 w + 31 of the chunk.
template <int S, int PP, bool STEP>
__global__ void __launch_bounds__(256, FITSNE_FORCE_MINB)
force_kernel(const Job* __restrict__ jobs, int njobs) {
    __shared__ int32_t s_start[kMaxJobs + 1];
    const int total = split_jobs(jobs, njobs, s_start, [](const Job& J) {
        const Params* P = J.params;
        return job_live(*P) ? (int)((J.N + kForceChunk - 1) / kForceChunk) : 0;
    });
    const int lane = threadIdx.x % 32;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int jb = job_of(s_start, njobs, item);
        const Job& J = jobs[jb];
        const int64_t c = item - s_start[jb];
        const int64_t N = J.N;
        const int64_t i0 = c * kForceChunk + (threadIdx.x / 32) * 32;
        if (i0 >= N) continue;
        const Params* __restrict__ Pp = J.params;
        const float* __restrict__ Y = J.ybuf[Pp->cur];
        force_block<S, PP, STEP>(J, Pp, Y, i0, N, lane);
    }
}

__device__ __forceinline__ unsigned sm_id() {
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned sm_id_count() {
    unsigned r;
    asm volatile("mov.u32 %0, %%nsmid;" : "=r"(r));
    return r;
}

// The step (or gradient) with SM-local work. The 32-row blocks of all jobs
// of the table (job after job) are cut into n_regions contiguous regions
// (n_regions >= the SM id range); the warps resident on the SM with id r take
// the blocks of region r, in order, through the region's counter next[r].
// So the warps of an SM work on one contiguous range of rows: in a relabelled
// run these are close in the embedding and share most neighbours, and in a
// batch of small jobs they belong to one job; either way the y_j they gather
// form one working set that the SM's L1 holds. A warp whose own region is
// used up moves on to regions r + 1, r + 2, ... (cyclically) to help SMs that
// are behind, and stops as soon as the count of claimed blocks
// (next[n_regions]) reaches the total, so the tail costs no more than the
// last claims. The loop ends: every probe either claims a block (finitely
// many) or moves to the next region (at most n_regions moves).
// next[0 .. n_regions] must be zero at launch.
template <int S, int PP, bool STEP>
__global__ void __launch_bounds__(256, FITSNE_FORCE_MINB)
force_region_kernel(const Job* __restrict__ jobs, int njobs, unsigned* __restrict__ next,
                    int n_regions) {
    __shared__ int32_t s_start[kMaxJobs + 1];
    const int nblk = split_jobs(jobs, njobs, s_start, [](const Job& J) {
        const Params* P = J.params;
        return job_live(*P) ? (int)((J.N + 31) / 32) : 0;
    });
    const int lane = threadIdx.x % 32;
    const int home = (int)(sm_id() % (unsigned)n_regions);
    unsigned* claimed = next + n_regions;
    for (int hop = 0; hop < n_regions;) {
        const int r = (home + hop) % n_regions;
        const int b0 = (int)((int64_t)nblk * r / n_regions), b1 = (int)((int64_t)nblk * (r + 1) / n_regions);
        int blk = -1;
        if (lane == 0) {
            if (hop == 0 || *(volatile unsigned*)claimed < (unsigned)nblk) {
                const unsigned k = atomicAdd(&next[r], 1u);
                if (b0 + (int64_t)k < b1) {
                    blk = b0 + (int)k;
                    atomicAdd(claimed, 1u);
                }
            } else {
                blk = -2;  // every block is claimed: done
            }
        }
        blk = __shfl_sync(kFull, blk, 0);
        if (blk == -2) break;
        if (blk < 0) { ++hop; continue; }
        const int jb = job_of(s_start, njobs, blk);
        const Job& J = jobs[jb];
        const Params* __restrict__ Pp = J.params;
        const float* __restrict__ Y = J.ybuf[Pp->cur];
        force_block<S, PP, STEP>(J, Pp, Y, (int64_t)(blk - s_start[jb]) * 32, J.N, lane);
    }
}

// Moves every stepping job that took part in this iteration to the next one:
// the new Y becomes current and the schedule index advances.
__global__ void advance_kernel(const Job* __restrict__ jobs, int njobs) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= njobs) return;
    const Job& J = jobs[j];
    if (J.mode != kModeStep) return;
    if (!J.params->active) return;
    JobDyn* d = J.dyn;
    d->cur ^= 1;
    d->iter += 1;
}

// ----------------------------------------------------------------------------
// KL(P || Q) = sum p log p + sum p log(1 + d^2) + (sum p) log Z over the stored
// entries (Sec. 1.1). Distances, logarithms and sums in FP64 from the FP32
// coordinates and values, reduced in a fixed order (per block, then by the
// last block).
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
            double d2;
            if (S == 2) {
                const float2 yj = reinterpret_cast<const float2*>(Y)[j];
                const double d0 = (double)yi0 - (double)yj.x, d1 = (double)yi1 - (double)yj.y;
                d2 = d0 * d0 + d1 * d1;
            } else {
                const double d0 = (double)yi0 - (double)Y[j];
                d2 = d0 * d0;
            }
            acc += (double)p * (log((double)p) + log1p(d2));
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
// Launchers. Grids are sized from the table's capacities (TableCaps) only.
// ----------------------------------------------------------------------------
static int grid_cap(int64_t items, int per_block, int64_t cap) {
    int64_t b = (items + per_block - 1) / per_block;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t launch_box(const Job* jobs, const TableCaps& c, const Tables& t, int ignore_schedule,
                       cudaStream_t st, int advance_first) {
    const int g = grid_cap(c.sum_box_items, 1, 4LL * c.sm_count);
    box_kernel<<<g, kBoxThreads, 0, st>>>(jobs, c.njobs, c.s, c.p, ignore_schedule, t, advance_first);
    return cudaGetLastError();
}

template <int S, int PP>
static void sort_and_spread_impl(const Job* jobs, const TableCaps& c, cudaStream_t st) {
    const int gp = grid_cap(c.sum_N, kSortPts, 8LL * c.sm_count);
    const size_t hs = sizeof(int32_t) * kHistBins;
    count_kernel<S><<<gp, 256, hs, st>>>(jobs, c.njobs);
    const int gsc = grid_cap((int64_t)c.njobs * c.max_scan_items, 1, 2LL * c.sm_count);
    scan_blocks_kernel<<<gsc, 1024, 0, st>>>(jobs, c.njobs);
    scan_boxes_kernel<<<gsc, 1024, 0, st>>>(jobs, c.njobs);
    scatter_kernel<S><<<gp, 256, hs, st>>>(jobs, c.njobs);
    // one resident wave (the kernel's registers allow two 256-thread CTAs per SM);
    // warps loop over the chunks
    const int gs = grid_cap(c.sum_chunk_cap * 32, 256, 2LL * c.sm_count);
    spread_kernel<S, PP><<<gs, 256, 0, st>>>(jobs, c.njobs);
}

#define FITSNE_DISPATCH(S_, FN, ...)                                   \
    switch (c.p) {                                                     \
        case 2: FN<S_, 2>(__VA_ARGS__); break;                         \
        case 3: FN<S_, 3>(__VA_ARGS__); break;                         \
        case 4: FN<S_, 4>(__VA_ARGS__); break;                         \
        default: FN<S_, 5>(__VA_ARGS__); break;                        \
    }

cudaError_t launch_sort_and_spread(const Job* jobs, const TableCaps& c, cudaStream_t st) {
    if (c.s == 2) { FITSNE_DISPATCH(2, sort_and_spread_impl, jobs, c, st); }
    else { FITSNE_DISPATCH(1, sort_and_spread_impl, jobs, c, st); }
    return cudaGetLastError();
}

template <int S, int PP>
static void forces_impl(const Job* jobs, const TableCaps& c, int step, cudaStream_t st) {
    const int g = grid_cap(c.sum_N, kForceChunk, 8LL * c.sm_count);
    if (step) force_kernel<S, PP, true><<<g, 256, 0, st>>>(jobs, c.njobs);
    else force_kernel<S, PP, false><<<g, 256, 0, st>>>(jobs, c.njobs);
}

template <int S, int PP>
static void region_impl(const Job* jobs, int njobs, int step, unsigned* next, int n_regions,
                        int sm_count, cudaStream_t st) {
    const int g = FITSNE_FORCE_MINB * sm_count;
    if (step) force_region_kernel<S, PP, true><<<g, 256, 0, st>>>(jobs, njobs, next, n_regions);
    else force_region_kernel<S, PP, false><<<g, 256, 0, st>>>(jobs, njobs, next, n_regions);
}

cudaError_t launch_forces_region(const Job* jobs, const TableCaps& c, int step, unsigned* next,
                                 int n_regions, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(next, 0, sizeof(unsigned) * (n_regions + 1), st);
    if (e != cudaSuccess) return e;
    if (c.s == 2) { FITSNE_DISPATCH(2, region_impl, jobs, c.njobs, step, next, n_regions, c.sm_count, st); }
    else { FITSNE_DISPATCH(1, region_impl, jobs, c.njobs, step, next, n_regions, c.sm_count, st); }
    return cudaGetLastError();
}

__global__ void sm_id_count_kernel(int* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *out = (int)sm_id_count();
}

cudaError_t query_sm_id_count(int* out_dev, cudaStream_t st) {
    sm_id_count_kernel<<<1, 32, 0, st>>>(out_dev);
    return cudaGetLastError();
}

cudaError_t launch_forces(const Job* jobs, const TableCaps& c, int step, cudaStream_t st) {
    if (c.s == 2) { FITSNE_DISPATCH(2, forces_impl, jobs, c, step, st); }
    else { FITSNE_DISPATCH(1, forces_impl, jobs, c, step, st); }
    return cudaGetLastError();
}

cudaError_t launch_advance(const Job* jobs, int njobs, cudaStream_t st) {
    advance_kernel<<<(njobs + 255) / 256, 256, 0, st>>>(jobs, njobs);
    return cudaGetLastError();
}

int phase_launches(int s) { return 1 + 5 + (s == 2 ? 3 : 1) + 1; }

__global__ void job_write_kernel(Job* __restrict__ dst, Job job, JobDyn* __restrict__ dyn_dst,
                                 JobDyn dyn, int with_dyn) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        *dst = job;
        if (with_dyn) *dyn_dst = dyn;
    }
}

__global__ void copy_current_kernel(const Job* __restrict__ row, int64_t count,
                                    float* __restrict__ dst) {
    const float* __restrict__ src = row->ybuf[row->dyn->cur];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
        dst[i] = src[i];
}

cudaError_t launch_copy_current(const Job* row, int64_t count, float* dst, cudaStream_t st) {
    int64_t b = (count + 255) / 256;
    if (b > 1024) b = 1024;
    if (b < 1) b = 1;
    copy_current_kernel<<<(int)b, 256, 0, st>>>(row, count, dst);
    return cudaGetLastError();
}

cudaError_t launch_job_write(Job* dst, const Job& job, JobDyn* dyn_dst, const JobDyn* dyn,
                             cudaStream_t st) {
    JobDyn d{};
    if (dyn) d = *dyn;
    job_write_kernel<<<1, 32, 0, st>>>(dst, job, dyn_dst, d, dyn != nullptr);
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

cudaError_t launch_validate(const tsne_csr& P, int64_t N, int32_t* flag, int sm_count,
                            cudaStream_t st) {
    const int g = grid_cap(N, 256, 8LL * sm_count);
    validate_kernel<<<g, 256, 0, st>>>(P.row_ptr, P.col, P.val, N, P.nnz, flag);
    return cudaGetLastError();
}

cudaError_t launch_fill(float* a, float v, int64_t n, int sm_count, cudaStream_t st) {
    const int g = grid_cap(n, 256, 8LL * sm_count);
    fill_kernel<<<g, 256, 0, st>>>(a, v, n);
    return cudaGetLastError();
}

}  // namespace fitsne
