// Exact k nearest neighbours with the distance tiles on the tensor cores.
//
// The squared distances of the kNN (Sec. 1.1 restricted to the k nearest
// points, Sec. 3) are |q|^2 + |c|^2 - 2 q.c; the dot products of a tile of
// 128 queries with a tile of 128 candidates are one 128 x 128 x 64 product:
// tcgen05.mma (kind::tf32) with the points split into TF32 head and tail
// (three MMAs per K-step: FP32-accurate products), accumulated in tensor
// memory. That form loses digits to cancellation (points far from the
// origin, neighbours close to each other), so it only shortlists: each query
// keeps every candidate whose approximate distance is within 2 eps of its
// running k'-th smallest one (k' = k + 32), where eps bounds the difference
// between the approximate value and the exact FP32 difference-form distance
// (derived below). At the end the shortlist's distances are recomputed in
// the difference form of the other kNN kernels (sum over d of (q_d - c_d)^2,
// one FMA per d, in order) and the k smallest by (distance, index) are the
// result: the same lists and distances, bit for bit, as knn_kernel, whenever
// the shortlist is provably complete. It is complete when it never
// overflowed and holds at least k entries: every point of the true top k has
// an approximate distance at most its exact one + eps <= the k-th exact
// distance + eps <= (the final k'-th approximate distance + eps) + eps. A
// query that fails the test is flagged and recomputed by knn_kernel.
//
// CTA (256 threads, persistent over query tiles): warp 0 issues the TMA
// loads (query tile once, candidate tiles through a 2-stage ring), warp 1
// owns the tensor memory (two 128-column accumulators) and issues the MMAs,
// warps 4..7 read the accumulators back (thread = query) and keep the
// shortlists in global memory (L2-resident, 512 entries per query).
#include <limits.h>
#include <math.h>

#include <algorithm>

#include "fitsne_internal.cuh"
#include "fitsne_tc.cuh"

namespace fitsne {
namespace knntc {

using namespace tc;

constexpr int kQ = 128;          // queries per tile (tensor-memory lanes)
constexpr int kC = 128;          // candidates per tile (accumulator columns)
constexpr int kDp = 64;          // padded dimension: two 32-float swizzle rows
constexpr int kStagesC = 2;      // candidate tiles in flight
constexpr int kBuf = 512;        // shortlist capacity per query
constexpr int kThreads = 256;
constexpr int kEpiWarpFirst = 4;  // warps 4..7 (warp % 4 = tensor-memory lane quarter)
constexpr uint32_t kIdesc = idesc_tf32(kQ, kC);
constexpr uint32_t kHalf = 128 * 32 * 4;         // one 32-float K chunk of 128 rows: 16 KB
constexpr uint32_t kTile = 2 * kHalf;            // 128 rows x 64: 32 KB (head or tail)
constexpr uint32_t kSmQ = 0;                     // query head | tail (64 KB)
constexpr uint32_t kSmC = 2 * kTile;             // candidate stages: head | tail (64 KB each)
constexpr uint32_t kSmem = kSmC + kStagesC * 2 * kTile + 1024;
static_assert(kSmem <= 232448, "shared memory of a kNN CTA");

// Column sums of X in FP64, one partial row per CTA (summed in order by
// centre_finish_kernel: a deterministic centre).
__global__ void column_partial_kernel(const float* __restrict__ X, int64_t N, int D, double* __restrict__ part) {
    __shared__ double s[256];
    const int d = threadIdx.x % kDp, g = threadIdx.x / kDp;  // 4 row groups of 64 columns
    double acc = 0.0;
    if (d < D)
        for (int64_t i = (int64_t)blockIdx.x * 4 + g; i < N; i += (int64_t)gridDim.x * 4) acc += (double)X[i * D + d];
    s[threadIdx.x] = acc;
    __syncthreads();
    if (g == 0) part[(int64_t)blockIdx.x * kDp + d] = s[d] + s[d + 64] + s[d + 128] + s[d + 192];
}

__global__ void centre_finish_kernel(const double* __restrict__ part, int nparts, int64_t N, int D,
                                     float* __restrict__ centre, unsigned* __restrict__ nmax) {
    const int d = threadIdx.x;
    if (d == 0) *nmax = 0u;
    if (d >= kDp) return;
    double acc = 0.0;
    for (int b = 0; b < nparts; ++b) acc += part[(int64_t)b * kDp + d];
    centre[d] = d < D ? (float)(acc / (double)N) : 0.0f;
}

// Rows of X - centre as the tensor cores read them: head and tail (Np x 64,
// zero past D and past N) and their squared norms |x - centre|^2 (FP32, one
// FMA per d in order), with the largest norm in nmax (+inf bits if a norm is
// not finite: every query is then recomputed by the row kernel). Distances
// do not depend on the centre; small norms keep the bound below small.
__global__ void split_points_kernel(const float* __restrict__ X, int64_t N, int D, int64_t Np,
                                    const float* __restrict__ centre, float* __restrict__ Xh,
                                    float* __restrict__ Xl, float* __restrict__ nrm, unsigned* __restrict__ nmax) {
    unsigned m = 0u;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < Np * kDp;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / kDp;
        const int d = (int)(e - i * kDp);
        const float x = (i < N && d < D) ? X[i * D + d] - centre[d] : 0.0f;
        const float h = tf32_head(x);
        Xh[e] = h;
        Xl[e] = x - h;
        if (d == 0) {
            float s = 0.0f;
            if (i < N)
                for (int t = 0; t < D; ++t) {
                    const float y = X[i * D + t] - centre[t];
                    s = fmaf(y, y, s);
                }
            nrm[i] = s;
            m = max(m, (s <= 3.402823466e38f) ? __float_as_uint(s) : 0x7F800000u);
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x % 32 == 0 && m) atomicMax(nmax, m);
}

// (d, idx) lexicographic order (the oracle's stable order of distances).
__device__ __forceinline__ bool pair_less(float d, int i, float e, int j) {
    return d < e || (d == e && i < j);
}

// Monotone map of floats to unsigned keys (negative values below positive).
__device__ __forceinline__ uint32_t order_key(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_value(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSlots = kBuf / 32;  // shortlist entries per lane when a warp holds one list
constexpr int kChunk = 32;         // accumulator columns per tensor-memory load

// The r-th smallest (0-based) of the keys the warp holds, by a bitwise radix
// select over the 32 key bits (empty slots hold 0xffffffff; r must be below
// the number of real keys).
__device__ __forceinline__ uint32_t warp_select(const uint32_t (&key)[kSlots], int r) {
    uint32_t want = 0u, mask = 0u;
#pragma unroll 1
    for (int bit = 31; bit >= 0; --bit) {
        const uint32_t m2 = mask | (1u << bit);
        unsigned c = 0u;
#pragma unroll
        for (int j = 0; j < kSlots; ++j) c += ((key[j] & m2) == want) ? 1u : 0u;
        c = __reduce_add_sync(kFull, c);
        if ((unsigned)r >= c) {
            r -= (int)c;
            want |= 1u << bit;
        }
        mask = m2;
    }
    return want;
}

// One shortlist (n entries at bl) compacted by the whole warp: with r >= 0
// the limit first drops to (the r-th smallest approximate distance) + band;
// the entries at or below the limit are written back packed, in order.
// Returns the new count; lim is updated (both warp-uniform).
__device__ int shortlist_compact(float2* __restrict__ bl, int n, int r, float band, float& lim, int lane) {
    float v[kSlots];
    int id[kSlots];
    uint32_t key[kSlots];
#pragma unroll
    for (int j = 0; j < kSlots; ++j) {
        const int t = lane + 32 * j;
        v[j] = INFINITY;
        id[j] = 0;
        key[j] = 0xFFFFFFFFu;
        if (t < n) {
            const float2 e = bl[t];
            v[j] = e.x;
            id[j] = __float_as_int(e.y);
            key[j] = order_key(e.x);
        }
    }
    if (r >= 0) lim = fminf(lim, key_value(warp_select(key, r)) + band);
    // positions written while packing slot j stay below 32 (j + 1), the
    // first position a later slot reads
    int base = 0;
#pragma unroll
    for (int j = 0; j < kSlots; ++j) {
        const bool keep = lane + 32 * j < n && v[j] <= lim;
        const unsigned bal = __ballot_sync(kFull, keep);
        if (keep) bl[base + __popc(bal & ((1u << lane) - 1u))] = make_float2(v[j], __int_as_float(id[j]));
        base += __popc(bal);
    }
    __syncwarp();
    return base;
}

// Exact distances of the n shortlisted candidates of query q (the
// difference form of knn_kernel: q_d - c_d, one FMA per d in order, a
// non-finite sum as +inf), then each entry's rank in (distance, index)
// order; ranks below k are the query's list. qrow: this warp's shared row.
__device__ void shortlist_rerank(const float2* __restrict__ bl, int n, int64_t q, const float* __restrict__ X,
                                 int D, int k, float* qrow, int32_t* __restrict__ out_idx,
                                 float* __restrict__ out_d2, int lane) {
    for (int d = lane; d < D; d += 32) qrow[d] = X[q * D + d];
    __syncwarp();
    const int nslots = (n + 31) / 32;
    float dv[kSlots];
    int id[kSlots], rank[kSlots];
#pragma unroll
    for (int j = 0; j < kSlots; ++j) {
        dv[j] = INFINITY;
        id[j] = INT_MAX;
        rank[j] = 0;
        if (j < nslots && lane + 32 * j < n) {
            id[j] = __float_as_int(bl[lane + 32 * j].y);
            const float* __restrict__ c = X + (int64_t)id[j] * D;
            float acc = 0.0f;
            for (int d = 0; d < D; ++d) {
                const float t = qrow[d] - c[d];
                acc = fmaf(t, t, acc);
            }
            dv[j] = (acc <= 3.402823466e38f) ? acc : INFINITY;
        }
    }
#pragma unroll
    for (int sj = 0; sj < kSlots; ++sj) {
        if (sj >= nslots) break;
#pragma unroll 4
        for (int sl = 0; sl < 32; ++sl) {
            const float od = __shfl_sync(kFull, dv[sj], sl);
            const int oi = __shfl_sync(kFull, id[sj], sl);
            if (sj * 32 + sl < n) {
#pragma unroll
                for (int j = 0; j < kSlots; ++j)
                    if (j < nslots) rank[j] += pair_less(od, oi, dv[j], id[j]) ? 1 : 0;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < kSlots; ++j)
        if (j < nslots && lane + 32 * j < n && rank[j] < k) {
            out_idx[q * k + rank[j]] = id[j];
            out_d2[q * k + rank[j]] = dv[j];
        }
    __syncwarp();
}

// |approximate - exact FP32 difference-form distance| <= kGamma (|q|^2 + |c|^2)
// (norms of the centred points) for D <= 64, summing worst cases: the norms'
// FP32 sums (64 u each), the 3xTF32 products (head x tail terms within
// 2^-21, the tail x tail term dropped), up to 24 accumulations in the tensor
// cores' FP32 accumulator at a few units of rounding each, the final
// additions, the centring, and the difference form's own 65 u: about
// 2.4e-5; the constant keeps a factor 2.5 over it.
constexpr float kGamma = 6.0e-5f;

struct Args {
    const float* X;        // N x D row-major (the exact re-rank)
    const float* nrm;      // [Np] |x - centre|^2
    const unsigned* nmax;  // largest norm (float bits)
    int64_t N;
    int D, k;
    int ksteps;            // K-steps of 8 that cover D
    int nqt, nct;          // query and candidate tiles
    float2* buf;           // [gridDim][kQ][kBuf] shortlists (distance, index bits)
    int32_t* out_idx;      // [N k]
    float* out_d2;         // [N k]
    int32_t* flagged;      // [N] queries left to the row kernel
    unsigned* nflagged;
    int* err;
};

__global__ void __launch_bounds__(kThreads, 1)
knn_tc_kernel(const __grid_constant__ CUtensorMap mapH, const __grid_constant__ CUtensorMap mapL, Args g) {
    extern __shared__ unsigned char smem_dyn[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t q_full, c_full[kStagesC], c_empty[kStagesC], tfull[2], tempty[2];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(16) float s_nc[2][kC];
    __shared__ float s_qrow[4][kDp];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&q_full), 1);
        for (int s = 0; s < kStagesC; ++s) {
            mbar_init(smem_u32(&c_full[s]), 1);
            mbar_init(smem_u32(&c_empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&tfull[b]), 1);
            mbar_init(smem_u32(&tempty[b]), 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_shared();
    }
    if (warp == 1) {  // two 128-column FP32 accumulators
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&s_tmem)), "r"(2 * kC) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const float ncmax = __uint_as_float(*g.nmax);
    bool failed = false;  // a wait gave up: the thread stops working but still meets its barriers
    int64_t it0 = 0;      // (query tile, candidate tile) pairs before this query tile
    for (int qt = blockIdx.x, qn = 0; qt < g.nqt; qt += gridDim.x, ++qn, it0 += g.nct) {
        tc_fence_before();
        __syncthreads();  // the previous query tile is finished: its MMAs are complete
        tc_fence_after();
        if (warp == 0) {
            if (lane == 0 && !failed) {  // TMA producer
                const uint32_t qb = smem_u32(&q_full);
                mbar_expect_tx(qb, 2 * kTile);
                for (int h = 0; h < 2; ++h)
                    for (int kc = 0; kc < 2; ++kc)
                        tma_load_2d(smem_u32(smem + kSmQ + h * kTile + kc * kHalf), h ? &mapL : &mapH, kc * 32,
                                    qt * kQ, qb);
                int64_t issued = it0;
                for (int ct = 0; ct < g.nct; ++ct) {
                    const int64_t it = it0 + ct;
                    const int s = (int)(it % kStagesC);
                    if (!mbar_wait(smem_u32(&c_empty[s]), ((uint32_t)(it / kStagesC) & 1u) ^ 1u, g.err)) {
                        failed = true;
                        break;
                    }
                    unsigned char* st = smem + kSmC + s * 2 * kTile;
                    const uint32_t fb = smem_u32(&c_full[s]);
                    mbar_expect_tx(fb, 2 * kTile);
                    for (int h = 0; h < 2; ++h)
                        for (int kc = 0; kc < 2; ++kc)
                            tma_load_2d(smem_u32(st + h * kTile + kc * kHalf), h ? &mapL : &mapH, kc * 32,
                                        ct * kC, fb);
                    issued = it + 1;
                }
                // nothing may land in shared memory after the CTA moves on
                mbar_wait_drain(qb, (uint32_t)qn & 1u);
                for (int64_t it = std::max(it0, issued - kStagesC); it < issued; ++it)
                    mbar_wait_drain(smem_u32(&c_full[it % kStagesC]), (uint32_t)(it / kStagesC) & 1u);
            }
        } else if (warp == 1) {
            if (lane == 0 && !failed) {  // MMA issuer
                if (!mbar_wait(smem_u32(&q_full), (uint32_t)qn & 1u, g.err)) failed = true;
                const uint64_t qh = sw128_desc(smem_u32(smem + kSmQ));
                const uint64_t ql = sw128_desc(smem_u32(smem + kSmQ + kTile));
                int64_t last = -1;
                for (int ct = 0; ct < g.nct && !failed; ++ct) {
                    const int64_t it = it0 + ct;
                    const int s = (int)(it % kStagesC), b = (int)(it & 1);
                    if (!mbar_wait(smem_u32(&tempty[b]), ((uint32_t)(it >> 1) & 1u) ^ 1u, g.err) ||
                        !mbar_wait(smem_u32(&c_full[s]), (uint32_t)(it / kStagesC) & 1u, g.err)) {
                        failed = true;
                        break;
                    }
                    tc_fence_after();
                    const unsigned char* st = smem + kSmC + s * 2 * kTile;
                    const uint64_t ch = sw128_desc(smem_u32(st));
                    const uint64_t cl = sw128_desc(smem_u32(st + kTile));
                    const uint32_t acc = tmem + (uint32_t)(b * kC);
                    for (int ks = 0; ks < g.ksteps; ++ks) {
                        // K-step ks: chunk ks / 4 (16 KB apart), 32 bytes = 2 address units per step
                        const uint64_t o = (uint64_t)((ks >> 2) * (kHalf >> 4) + 2 * (ks & 3));
                        mma_tf32(acc, qh + o, ch + o, kIdesc, ks ? 1u : 0u);
                        mma_tf32(acc, qh + o, cl + o, kIdesc, 1u);
                        mma_tf32(acc, ql + o, ch + o, kIdesc, 1u);
                    }
                    mma_commit(smem_u32(&c_empty[s]));
                    mma_commit(smem_u32(&tfull[b]));
                    last = it;
                }
                if (last >= 0) mbar_wait_drain(smem_u32(&tfull[last & 1]), (uint32_t)(last >> 1) & 1u);
            }
        } else if (warp >= kEpiWarpFirst) {
            // epilogue: thread = query (tensor-memory lane); shortlist in global memory
            const int quarter = warp % 4;
            const int ql_ = 32 * quarter + lane;
            const int64_t q = (int64_t)qt * kQ + ql_;
            const bool live = q < g.N;
            const float nq = live ? g.nrm[q] : 0.0f;
            const float band = 2.0f * kGamma * (nq + ncmax);
            const bool finite = band <= 3.402823466e38f;
            float2* const warp_buf = g.buf + ((int64_t)blockIdx.x * kQ + 32 * quarter) * kBuf;
            float2* const bl = warp_buf + (int64_t)lane * kBuf;
            float lim = INFINITY;
            int cnt = 0;
            bool open = live && finite;  // still collecting (not overflowed)
            const uint32_t lane_addr = tmem + ((uint32_t)(32 * quarter) << 16);
            for (int ct = 0; ct < g.nct; ++ct) {
                const int64_t it = it0 + ct;
                const int b = (int)(it & 1);
                const int64_t cidx = (int64_t)ct * kC + ql_;
                s_nc[b][ql_] = cidx < g.N ? g.nrm[cidx] : __int_as_float(0x7FC00000);  // NaN: never kept
                asm volatile("bar.sync 1, 128;" ::: "memory");
                bool ok = failed || mbar_wait(smem_u32(&tfull[b]), (uint32_t)(it >> 1) & 1u, g.err);
                failed = __any_sync(kFull, failed || !ok);
                if (!failed) {
                    tc_fence_after();
#pragma unroll 1
                    for (int cc = 0; cc < kC; cc += kChunk) {
                        // lists that might not take a whole chunk are compacted first
                        __syncwarp();
                        unsigned need = __ballot_sync(kFull, open && cnt > kBuf - kChunk);
                        while (need) {
                            const int L = __ffs(need) - 1;
                            need &= need - 1;
                            float limL = __shfl_sync(kFull, lim, L);
                            const int n2 = shortlist_compact(warp_buf + (int64_t)L * kBuf,
                                                             __shfl_sync(kFull, cnt, L), g.k - 1,
                                                             __shfl_sync(kFull, band, L), limL, lane);
                            if (lane == L) {
                                cnt = n2;
                                lim = limL;
                                if (n2 > kBuf - kBuf / 4) open = false;  // too many near-ties: row kernel
                            }
                        }
                        float dots[kChunk];
                        tmem_ld32(lane_addr + (uint32_t)(b * kC + cc), dots);
                        if (open) {
                            const float4* nc4 = reinterpret_cast<const float4*>(&s_nc[b][cc]);
                            const int c0 = ct * kC + cc;
                            const int jself = (int)(q - c0);
                            if (jself >= 0 && jself < kChunk) {
#pragma unroll
                                for (int j4 = 0; j4 < kChunk / 4; ++j4) {
                                    const float4 n4 = nc4[j4];
                                    const float nn[4] = {n4.x, n4.y, n4.z, n4.w};
#pragma unroll
                                    for (int u = 0; u < 4; ++u) {
                                        const int j = 4 * j4 + u;
                                        const float d = fmaf(-2.0f, dots[j], nq + nn[u]);
                                        if (d <= lim && j != jself) bl[cnt++] = make_float2(d, __int_as_float(c0 + j));
                                    }
                                }
                            } else {
#pragma unroll
                                for (int j4 = 0; j4 < kChunk / 4; ++j4) {
                                    const float4 n4 = nc4[j4];
                                    const float nn[4] = {n4.x, n4.y, n4.z, n4.w};
#pragma unroll
                                    for (int u = 0; u < 4; ++u) {
                                        const int j = 4 * j4 + u;
                                        const float d = fmaf(-2.0f, dots[j], nq + nn[u]);
                                        if (d <= lim) bl[cnt++] = make_float2(d, __int_as_float(c0 + j));
                                    }
                                }
                            }
                        }
                    }
                    tc_fence_before();
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&tempty[b]));
            }
            // final limit (the k-th smallest + band), exact re-rank, lists
            const bool done = open && !failed && cnt >= g.k;
            __syncwarp();
            unsigned m = __ballot_sync(kFull, done);
            while (m) {
                const int L = __ffs(m) - 1;
                m &= m - 1;
                float limL = __shfl_sync(kFull, lim, L);
                float2* blL = warp_buf + (int64_t)L * kBuf;
                const int n2 = shortlist_compact(blL, __shfl_sync(kFull, cnt, L), g.k - 1,
                                                 __shfl_sync(kFull, band, L), limL, lane);
                shortlist_rerank(blL, n2, (int64_t)qt * kQ + 32 * quarter + L, g.X, g.D, g.k, s_qrow[quarter],
                                 g.out_idx, g.out_d2, lane);
            }
            if (live && !done) g.flagged[atomicAdd(g.nflagged, 1u)] = (int32_t)q;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kC) : "memory");
    }
}

}  // namespace knntc

using namespace knntc;

// ----------------------------------------------------------------------------
// Host
// ----------------------------------------------------------------------------
struct KnnTc {
    int64_t N = 0, Np = 0;
    int D = 0, k = 0, grid = 0, nparts = 0;
    float* Xh = nullptr;       // [Np][64] heads of the centred points
    float* Xl = nullptr;       // [Np][64] tails
    float* nrm = nullptr;      // [Np]
    float* centre = nullptr;   // [64]
    double* part = nullptr;    // [nparts][64]
    unsigned* ctl = nullptr;   // [0] leftover count, [1] error word, [2] largest norm
    float2* buf = nullptr;     // [grid][kQ][kBuf]
    int32_t* leftover = nullptr;  // [N]
    CUtensorMap mapH, mapL;
};

bool knn_tc_supported(int D, int k) { return D >= 1 && D <= knntc::kDp && k >= 1 && k <= kBuf / 2; }

void knn_tc_destroy(KnnTc* w) {
    if (!w) return;
    void* ps[] = {w->Xh, w->Xl, w->nrm, w->centre, w->part, w->ctl, w->buf, w->leftover};
    for (void* p : ps)
        if (p) cudaFree(p);
    delete w;
}

namespace {
template <typename T>
int tc_alloc(T** p, size_t count, const char* what) {
    *p = nullptr;
    if (cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(TSNE_ERR_OOM, "cudaMalloc of %zu bytes for %s failed", count * sizeof(T), what);
    }
    return TSNE_OK;
}
}  // namespace

int knn_tc_create(int64_t N, int D, int k, int sm_count, KnnTc** out) {
    *out = nullptr;
    if (!knn_tc_supported(D, k) || N <= k)
        return set_error(TSNE_ERR_INVALID_ARG, "tensor-core kNN: D = %d, k = %d, N = %lld unsupported", D, k,
                         (long long)N);
    KnnTc* w = new KnnTc();
    w->N = N;
    w->D = D;
    w->k = k;
    w->Np = (N + kQ - 1) / kQ * kQ;
    const int64_t nqt = w->Np / kQ;
    w->grid = (int)std::min<int64_t>(nqt, std::max(1, sm_count));
    w->nparts = (int)std::min<int64_t>((N + 3) / 4, 1024);
    int rc = tc_alloc(&w->Xh, (size_t)(w->Np * kDp), "kNN heads");
    if (!rc) rc = tc_alloc(&w->Xl, (size_t)(w->Np * kDp), "kNN tails");
    if (!rc) rc = tc_alloc(&w->nrm, (size_t)w->Np, "kNN norms");
    if (!rc) rc = tc_alloc(&w->centre, (size_t)kDp, "kNN centre");
    if (!rc) rc = tc_alloc(&w->part, (size_t)w->nparts * kDp, "kNN column sums");
    if (!rc) rc = tc_alloc(&w->ctl, 4, "kNN control words");
    if (!rc) rc = tc_alloc(&w->buf, (size_t)w->grid * kQ * kBuf, "kNN shortlists");
    if (!rc) rc = tc_alloc(&w->leftover, (size_t)N, "kNN leftover queries");
    if (!rc) {
        const int r1 = encode_map_f32_2d(&w->mapH, w->Xh, w->Np, kDp, kDp, 32, kQ);
        const int r2 = r1 ? r1 : encode_map_f32_2d(&w->mapL, w->Xl, w->Np, kDp, kDp, 32, kQ);
        if (r2 < 0) rc = set_error(TSNE_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
        else if (r2) rc = set_error(TSNE_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", r2);
    }
    if (rc) {
        knn_tc_destroy(w);
        return rc;
    }
    *out = w;
    return TSNE_OK;
}

int knn_tc_launch(KnnTc* w, const float* X, int32_t* out_idx, float* out_d2, cudaStream_t st, int64_t* launches) {
    cudaError_t e = cudaMemsetAsync(w->ctl, 0, 4 * sizeof(unsigned), st);
    if (e == cudaSuccess) {
        column_partial_kernel<<<w->nparts, 256, 0, st>>>(X, w->N, w->D, w->part);
        centre_finish_kernel<<<1, kDp, 0, st>>>(w->part, w->nparts, w->N, w->D, w->centre, w->ctl + 2);
        const int64_t total = w->Np * kDp;
        split_points_kernel<<<(int)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, st>>>(
            X, w->N, w->D, w->Np, w->centre, w->Xh, w->Xl, w->nrm, w->ctl + 2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaFuncSetAttribute(knn_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e == cudaSuccess) {
        Args g;
        g.X = X;
        g.nrm = w->nrm;
        g.nmax = w->ctl + 2;
        g.N = w->N;
        g.D = w->D;
        g.k = w->k;
        g.ksteps = (w->D + 7) / 8;
        g.nqt = (int)(w->Np / kQ);
        g.nct = (int)(w->Np / kC);
        g.buf = w->buf;
        g.out_idx = out_idx;
        g.out_d2 = out_d2;
        g.flagged = w->leftover;
        g.nflagged = w->ctl;
        g.err = reinterpret_cast<int*>(w->ctl + 1);
        knn_tc_kernel<<<w->grid, kThreads, kSmem, st>>>(w->mapH, w->mapL, g);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return set_error(TSNE_ERR_CUDA, "tensor-core kNN launch: %s", cudaGetErrorString(e));
    *launches += 4;
    return TSNE_OK;
}

int knn_tc_leftover(KnnTc* w, cudaStream_t st, int64_t* count, const int32_t** list) {
    unsigned h[2] = {0u, 0u};
    cudaError_t e = cudaMemcpyAsync(h, w->ctl, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(TSNE_ERR_CUDA, "tensor-core kNN read-back: %s", cudaGetErrorString(e));
    if (h[1]) return set_error(TSNE_ERR_TIMEOUT, "tensor-core kNN: a pipeline wait gave up");
    *count = (int64_t)h[0];
    *list = w->leftover;
    return TSNE_OK;
}

}  // namespace fitsne
