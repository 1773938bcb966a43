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
constexpr int kAcc = 4;           // accumulator buffers (4 x 128 columns: all of tensor memory)
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

// Squared norms |x - centre|^2 of the rows (FP32, one FMA per d in order;
// 0 past N) and the largest in nmax (+inf bits if a norm is not finite:
// every query is then recomputed by the row kernel). Distances do not
// depend on the centre; small norms keep the bound below small.
__global__ void norms_kernel(const float* __restrict__ X, int64_t N, int D, int64_t Np,
                             const float* __restrict__ centre, float* __restrict__ nrm, unsigned* __restrict__ nmax) {
    unsigned m = 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Np; i += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.0f;
        if (i < N)
            for (int t = 0; t < D; ++t) {
                const float y = X[i * D + t] - centre[t];
                s = fmaf(y, y, s);
            }
        nrm[i] = s;
        m = max(m, (s <= 3.402823466e38f) ? __float_as_uint(s) : 0x7F800000u);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x % 32 == 0 && m) atomicMax(nmax, m);
}

// The operands as the tensor cores read them (Np x 64 FP32 each, TF32 head
// and tail): queries -2 (x - centre), candidates x - centre, zero past D and
// past N. With fold (D < 64) column D carries the norm: 1 on the query side,
// |c|^2 on the candidate side (NaN past N: such candidates never pass), so
// the products give v = |c|^2 - 2 q.c directly.
__global__ void split_points_kernel(const float* __restrict__ X, int64_t N, int D, int64_t Np,
                                    const float* __restrict__ centre, const float* __restrict__ nrm, int fold,
                                    float* __restrict__ Qh, float* __restrict__ Ql, float* __restrict__ Ch,
                                    float* __restrict__ Cl) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < Np * kDp;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / kDp;
        const int d = (int)(e - i * kDp);
        float c = 0.0f, qv = 0.0f;
        if (d < D) {
            c = i < N ? X[i * D + d] - centre[d] : 0.0f;
            qv = -2.0f * c;  // exact
        } else if (fold && d == D) {
            c = i < N ? nrm[i] : __int_as_float(0x7FC00000);
            qv = 1.0f;
        }
        const float ch = tf32_head(c), qh = tf32_head(qv);
        Ch[e] = ch;
        Cl[e] = c - ch;
        Qh[e] = qh;
        Ql[e] = qv - qh;
    }
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

// An upper bound within 256 key units of the r-th smallest (0-based) key
// the warp holds: a bitwise radix select over the top 24 key bits (from the
// highest bit where the real keys differ), then the largest key with that
// prefix (empty slots hold 0xffffffff; r must be below the number of real
// keys). At least r + 1 keys are at or below it.
template <int kS>
__device__ __forceinline__ uint32_t warp_select_bound(const uint32_t (&key)[kS], int r) {
    // the bits all real keys share decide nothing: start below them
    uint32_t kmin = 0xFFFFFFFFu, kmax = 0u;
#pragma unroll
    for (int j = 0; j < kS; ++j)
        if (key[j] != 0xFFFFFFFFu) {
            kmin = min(kmin, key[j]);
            kmax = max(kmax, key[j]);
        }
    kmin = __reduce_min_sync(kFull, kmin);
    kmax = __reduce_max_sync(kFull, kmax);
    if (kmin >= kmax) return kmin | 0xFFu;
    const int h = 31 - __clz(kmin ^ kmax);  // the highest bit where real keys differ
    if (h < 8) return kmax | 0xFFu;
    uint32_t mask = ~((2u << h) - 1u);       // the shared bits (none when h = 31)
    uint32_t want = kmin & mask;
#pragma unroll 1
    for (int bit = h; bit >= 8; --bit) {
        const uint32_t m2 = mask | (1u << bit);
        unsigned c = 0u;
#pragma unroll
        for (int j = 0; j < kS; ++j) c += ((key[j] & m2) == want) ? 1u : 0u;
        c = __reduce_add_sync(kFull, c);
        if ((unsigned)r >= c) {
            r -= (int)c;
            want |= 1u << bit;
        }
        mask = m2;
    }
    return want | 0xFFu;
}

// One shortlist (n <= 32 kS entries at src) compacted by the whole warp:
// with r >= 0 the limit first drops to (a bound within 256 key units above
// the r-th smallest value) + band; the entries at or below the limit, other
// than the candidate `exclude`, are written packed, in order, to dst (which
// may be src), at most cap of them. Returns how many there are (possibly
// more than cap); lim is updated (both warp-uniform). Every entry is read
// into registers before the first write.
template <int kS>
__device__ int shortlist_compact(const float2* src, int n, int r, float band, float& lim, float2* dst, int cap,
                                 int exclude, int lane) {
    float v[kS];
    int id[kS];
    uint32_t key[kS];
#pragma unroll
    for (int j = 0; j < kS; ++j) {
        const int t = lane + 32 * j;
        v[j] = INFINITY;
        id[j] = 0;
        key[j] = 0xFFFFFFFFu;
        if (t < n) {
            const float2 e = src[t];
            v[j] = e.x;
            id[j] = __float_as_int(e.y);
            key[j] = order_key(e.x);
        }
    }
    if (r >= 0) lim = fminf(lim, key_value(warp_select_bound<kS>(key, r)) + band);
    int base = 0;
#pragma unroll
    for (int j = 0; j < kS; ++j) {
        const bool keep = lane + 32 * j < n && v[j] <= lim && id[j] != exclude;
        const unsigned bal = __ballot_sync(kFull, keep);
        const int pos = base + __popc(bal & ((1u << lane) - 1u));
        if (keep && pos < cap) dst[pos] = make_float2(v[j], __int_as_float(id[j]));
        base += __popc(bal);
    }
    __syncwarp();
    return base;
}

// The shortlist ranks candidates c of query q by v = |c|^2 - 2 q.c, the
// squared distance less the query's own |q|^2 (from the accumulator
// directly when the norm rides in a spare K column, else one FADD).
// |(v + |q|^2) - (exact FP32 difference-form distance)| <=
// kGamma (|q|^2 + |c|^2) (norms of the centred points) for D <= 64, summing
// worst cases: the norms' FP32 sums (64 u each), the 3xTF32 products (head
// x tail terms within 2^-21, the tail x tail term dropped), up to 24
// accumulations in the tensor cores' FP32 accumulator at a few units of
// rounding of partial sums bounded by |c|^2 + |q|^2 + |c|^2, the centring,
// and the difference form's own 65 u: about 3e-5; the constant keeps a
// factor 2 over it.
constexpr float kGamma = 6.0e-5f;

struct Args {
    const float* nrm;      // [Np] |x - centre|^2
    const unsigned* nmax;  // largest norm (float bits)
    int64_t N;
    int k;
    int ksteps;            // K-steps of 8 that cover D (and the norm column)
    int nqt, nct;          // query and candidate tiles
    float2* buf;           // [gridDim][kQ][kBuf] running shortlists (v, index bits)
    float2* lists;         // [N][S] final shortlists
    int32_t* counts;       // [N] final shortlist sizes, -1: left to the row kernel
    int S;
    int32_t* flagged;      // [N] queries left to the row kernel
    unsigned* nflagged;
    int* err;
    unsigned* pace;        // rounds finished, summed over the CTAs (zero at launch)
};

// Pacing between the CTAs of the (cooperative) launch: a CTA starts query
// round qn only when every CTA has finished round qn - 1, so that all CTAs
// sweep the candidates together and share them in L2. Thread 0 only; the
// wait is bounded (the error word is set and the pacing dropped when it
// gives up). No data passes between CTAs.
__device__ void pace_wait(const unsigned* pace, unsigned target, int nct, int* err) {
    // at most about 16 us per candidate tile of a round (a round takes about
    // 1.5 us per tile), and at least 2 s
    const uint64_t limit = std::max<uint64_t>(1ull << 23, (uint64_t)nct * 64ull);
    for (uint64_t it = 0; it < limit; ++it) {
        if (*(volatile const unsigned*)pace >= target) return;
        if ((it & 255u) == 255u && *(volatile int*)err) return;
        __nanosleep(256);
    }
    atomicExch(err, kErrTimeout);
}

// The MMAs of one (query tile, candidate tile) pair: KS K-steps of 8, each
// head x head + head x tail + tail x head into the accumulator. Unrolled with
// a compile-time count: a loop with a run-time count issued the MMAs at half
// the rate (65.4 ms against 80.8 ms for the kernel at N = 400k without
// filtering).
template <int KS>
__device__ __forceinline__ void tile_mmas(uint32_t acc, uint64_t qh, uint64_t ql, uint64_t ch, uint64_t cl) {
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
        // K-step ks: chunk ks / 4 (16 KB apart), 32 bytes = 2 address units per step
        const uint64_t o = (uint64_t)((ks >> 2) * (kHalf >> 4) + 2 * (ks & 3));
        mma_tf32(acc, qh + o, ch + o, kIdesc, ks ? 1u : 0u);
        mma_tf32(acc, qh + o, cl + o, kIdesc, 1u);
        mma_tf32(acc, ql + o, ch + o, kIdesc, 1u);
    }
}

// Shortlist bookkeeping: the self candidate (v = -|q|^2, the smallest) is
// kept while collecting and dropped at the end, so the limits use the
// (k + 1)-th smallest value (0-based rank k), which is at least the k-th
// smallest over the other candidates whether or not self was seen yet.
template <bool kFold>
__global__ void __launch_bounds__(kThreads, 1)
knn_tc_kernel(const __grid_constant__ CUtensorMap mapQH, const __grid_constant__ CUtensorMap mapQL,
              const __grid_constant__ CUtensorMap mapCH, const __grid_constant__ CUtensorMap mapCL, Args g) {
    extern __shared__ unsigned char smem_dyn[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t q_full, c_full[kStagesC], c_empty[kStagesC], tfull[kAcc], tempty[kAcc];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(16) float s_nc[4][kC];  // without fold: each epilogue warp's copy of the tile's norms
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&q_full), 1);
        for (int s = 0; s < kStagesC; ++s) {
            mbar_init(smem_u32(&c_full[s]), 1);
            mbar_init(smem_u32(&c_empty[s]), 1);
        }
        for (int b = 0; b < kAcc; ++b) {
            mbar_init(smem_u32(&tfull[b]), 1);
            mbar_init(smem_u32(&tempty[b]), 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_shared();
    }
    if (warp == 1) {  // kAcc 128-column FP32 accumulators
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&s_tmem)), "r"(kAcc * kC) : "memory");
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
        if (qn > 0 && threadIdx.x == 0) {
            atomicAdd(g.pace, 1u);  // round qn - 1 done
            pace_wait(g.pace, (unsigned)qn * gridDim.x, g.nct, g.err);
        }
        __syncthreads();
        tc_fence_after();
        if (warp == 0) {
            if (lane == 0 && !failed) {  // TMA producer
                const int nkc = g.ksteps > 4 ? 2 : 1;  // 32-column chunks the K-steps read
                const uint32_t qb = smem_u32(&q_full);
                mbar_expect_tx(qb, 2 * nkc * kHalf);
                for (int h = 0; h < 2; ++h)
                    for (int kc = 0; kc < nkc; ++kc)
                        tma_load_2d(smem_u32(smem + kSmQ + h * kTile + kc * kHalf), h ? &mapQL : &mapQH, kc * 32,
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
                    mbar_expect_tx(fb, 2 * nkc * kHalf);
                    for (int h = 0; h < 2; ++h)
                        for (int kc = 0; kc < nkc; ++kc)
                            tma_load_2d(smem_u32(st + h * kTile + kc * kHalf), h ? &mapCL : &mapCH, kc * 32,
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
                    const int s = (int)(it % kStagesC), b = (int)(it % kAcc);
                    if (!mbar_wait(smem_u32(&tempty[b]), ((uint32_t)(it / kAcc) & 1u) ^ 1u, g.err) ||
                        !mbar_wait(smem_u32(&c_full[s]), (uint32_t)(it / kStagesC) & 1u, g.err)) {
                        failed = true;
                        break;
                    }
                    tc_fence_after();
                    const unsigned char* st = smem + kSmC + s * 2 * kTile;
                    const uint64_t ch = sw128_desc(smem_u32(st));
                    const uint64_t cl = sw128_desc(smem_u32(st + kTile));
                    const uint32_t acc = tmem + (uint32_t)(b * kC);
                    switch (g.ksteps) {  // fully unrolled sequences issue back to back
                        case 1: tile_mmas<1>(acc, qh, ql, ch, cl); break;
                        case 2: tile_mmas<2>(acc, qh, ql, ch, cl); break;
                        case 3: tile_mmas<3>(acc, qh, ql, ch, cl); break;
                        case 4: tile_mmas<4>(acc, qh, ql, ch, cl); break;
                        case 5: tile_mmas<5>(acc, qh, ql, ch, cl); break;
                        case 6: tile_mmas<6>(acc, qh, ql, ch, cl); break;
                        case 7: tile_mmas<7>(acc, qh, ql, ch, cl); break;
                        default: tile_mmas<8>(acc, qh, ql, ch, cl); break;
                    }
                    mma_commit(smem_u32(&c_empty[s]));
                    mma_commit(smem_u32(&tfull[b]));
                    last = it;
                }
                if (last >= 0) mbar_wait_drain(smem_u32(&tfull[last % kAcc]), (uint32_t)(last / kAcc) & 1u);
            }
        } else if (warp >= kEpiWarpFirst) {
            // epilogue: thread = query (tensor-memory lane); shortlist in global memory
            const int ew = warp - kEpiWarpFirst, quarter = warp % 4;
            const int ql_ = 32 * quarter + lane;
            const int64_t q = (int64_t)qt * kQ + ql_;
            const bool live = q < g.N;
            const float nq = live ? g.nrm[q] : 0.0f;
            const float band = 2.0f * kGamma * (nq + ncmax);
            const bool finite = band <= 3.402823466e38f;
            float2* const warp_buf = g.buf + ((int64_t)blockIdx.x * kQ + 32 * quarter) * kBuf;
            float2* const bl = warp_buf + (int64_t)lane * kBuf;
            bool open = live && finite;  // still collecting (not overflowed)
            float lim = open ? INFINITY : -INFINITY;  // a closed list takes nothing
            int cnt = 0;
            const uint32_t lane_addr = tmem + ((uint32_t)(32 * quarter) << 16);
            // without fold: the candidate norms of the next tile, fetched one
            // tile ahead (each warp its own copy: the warps run decoupled)
            auto fetch = [&](int ct) -> float4 {
                const int64_t c = (int64_t)ct * kC + 4 * lane;
                float4 r = *reinterpret_cast<const float4*>(g.nrm + c);  // Np entries: in range
                if (c + 3 >= g.N) {
                    const float nan = __int_as_float(0x7FC00000);  // never kept
                    if (c + 0 >= g.N) r.x = nan;
                    if (c + 1 >= g.N) r.y = nan;
                    if (c + 2 >= g.N) r.z = nan;
                    if (c + 3 >= g.N) r.w = nan;
                }
                return r;
            };
            float4 nx = kFold ? make_float4(0.f, 0.f, 0.f, 0.f) : fetch(0);
            for (int ct = 0; ct < g.nct; ++ct) {
                const int64_t it = it0 + ct;
                const int b = (int)(it % kAcc);
                if (!kFold) {
                    __syncwarp();
                    reinterpret_cast<float4*>(s_nc[ew])[lane] = nx;
                    __syncwarp();
                    if (ct + 1 < g.nct) nx = fetch(ct + 1);
                }
                bool ok = failed || mbar_wait(smem_u32(&tfull[b]), (uint32_t)(it / kAcc) & 1u, g.err);
                failed = __any_sync(kFull, failed || !ok);
                if (!failed) {
                    // lists that might not take a whole tile are compacted first
                    unsigned need = __ballot_sync(kFull, open && cnt > kBuf - kC);
                    while (need) {
                        const int L = __ffs(need) - 1;
                        need &= need - 1;
                        float limL = __shfl_sync(kFull, lim, L);
                        float2* bL = warp_buf + (int64_t)L * kBuf;
                        const int n2 = shortlist_compact<kSlots>(bL, __shfl_sync(kFull, cnt, L), g.k,
                                                                 __shfl_sync(kFull, band, L), limL, bL, kBuf, -1, lane);
                        if (lane == L) {
                            cnt = n2;
                            lim = limL;
                            if (n2 > kBuf - kC) {  // too many near-ties: row kernel
                                open = false;
                                lim = -INFINITY;
                            }
                        }
                    }
                    tc_fence_after();
#pragma unroll 1
                    for (int cc = 0; cc < kC; cc += kChunk) {
                        float v[kChunk];
                        tmem_ld32(lane_addr + (uint32_t)(b * kC + cc), v);
                        if (!kFold) {
                            const float4* nc4 = reinterpret_cast<const float4*>(&s_nc[ew][cc]);
#pragma unroll
                            for (int j4 = 0; j4 < kChunk / 4; ++j4) {
                                const float4 n4 = nc4[j4];
                                // the query operand already carries the -2
                                v[4 * j4 + 0] += n4.x;
                                v[4 * j4 + 1] += n4.y;
                                v[4 * j4 + 2] += n4.z;
                                v[4 * j4 + 3] += n4.w;
                            }
                        }
                        const int c0 = ct * kC + cc;
                        // groups of 4 candidates: the warp votes on every
                        // group's minimum first (independent), then visits
                        // the groups some list takes from, candidate by candidate
                        bool hit[kChunk / 4];
#pragma unroll
                        for (int j4 = 0; j4 < kChunk / 4; ++j4) {
                            const float mn = fminf(fminf(v[4 * j4], v[4 * j4 + 1]), fminf(v[4 * j4 + 2], v[4 * j4 + 3]));
                            hit[j4] = __any_sync(kFull, mn <= lim);
                        }
#pragma unroll
                        for (int j4 = 0; j4 < kChunk / 4; ++j4) {
                            if (hit[j4]) {
#pragma unroll
                                for (int u = 0; u < 4; ++u) {
                                    const int j = 4 * j4 + u;
                                    const bool t = v[j] <= lim;
                                    if (__ballot_sync(kFull, t) && t)
                                        bl[cnt++] = make_float2(v[j], __int_as_float(c0 + j));
                                }
                            }
                        }
                    }
                    tc_fence_before();
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&tempty[b]));
            }
            // final limit (the (k+1)-th smallest + band; self dropped); the
            // list moves to its query's slot for the exact re-rank
            const bool done = open && !failed && cnt >= g.k + 1;
            __syncwarp();
            unsigned m = __ballot_sync(kFull, done);
            bool fits = false;
            while (m) {
                const int L = __ffs(m) - 1;
                m &= m - 1;
                float limL = __shfl_sync(kFull, lim, L);
                const int64_t qL = (int64_t)qt * kQ + 32 * quarter + L;
                const int n2 = shortlist_compact<kSlots>(warp_buf + (int64_t)L * kBuf, __shfl_sync(kFull, cnt, L), g.k,
                                                         __shfl_sync(kFull, band, L), limL, g.lists + qL * g.S, g.S,
                                                         (int)qL, lane);
                if (lane == L) {
                    fits = n2 >= g.k && n2 <= g.S;
                    g.counts[q] = fits ? n2 : -1;
                }
            }
            if (live && !(done && fits)) {
                g.counts[q] = -1;
                g.flagged[atomicAdd(g.nflagged, 1u)] = (int32_t)q;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && blockIdx.x < g.nqt) atomicAdd(g.pace, 1u);  // the last round done
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kAcc * kC) : "memory");
    }
}

// Exact re-rank, a warp per query: each shortlisted candidate gets the
// difference-form FP32 distance of knn_kernel (q_d - c_d, one FMA per d in
// order, a non-finite sum as +inf), then its rank in (distance, index)
// order among the shortlist; ranks below k are the query's list. kS: slots
// per lane (the shortlist capacity S = 32 kS).
template <int kS>
__global__ void __launch_bounds__(256)
knn_rerank_kernel(const float* __restrict__ X, int64_t N, int D, int k, const float2* __restrict__ lists,
                  const int32_t* __restrict__ counts, int32_t* __restrict__ out_idx, float* __restrict__ out_d2) {
    __shared__ float s_q[8][kDp];
    const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
    constexpr int S = 32 * kS;
    for (int64_t q = (int64_t)blockIdx.x * 8 + w; q < N; q += (int64_t)gridDim.x * 8) {
        const int n = counts[q];
        if (n < 0) continue;  // warp-uniform: the row kernel's query
        for (int d = lane; d < D; d += 32) s_q[w][d] = X[q * D + d];
        __syncwarp();
        const int nslots = (n + 31) / 32;
        float dv[kS];
        int id[kS], rank[kS];
#pragma unroll
        for (int j = 0; j < kS; ++j) {
            dv[j] = INFINITY;
            id[j] = INT_MAX;
            rank[j] = 0;
            if (lane + 32 * j < n) {
                id[j] = __float_as_int(lists[q * S + lane + 32 * j].y);
                const float* __restrict__ c = X + (int64_t)id[j] * D;
                float acc = 0.0f;
#pragma unroll 8
                for (int d = 0; d < D; ++d) {
                    const float t = s_q[w][d] - c[d];
                    acc = fmaf(t, t, acc);
                }
                dv[j] = (acc <= 3.402823466e38f) ? acc : INFINITY;
            }
        }
#pragma unroll
        for (int sj = 0; sj < kS; ++sj) {
            if (sj >= nslots) break;
            for (int sl = 0; sl < 32; ++sl) {
                const float od = __shfl_sync(kFull, dv[sj], sl);
                const int oi = __shfl_sync(kFull, id[sj], sl);
                if (sj * 32 + sl < n) {
#pragma unroll
                    for (int j = 0; j < kS; ++j) rank[j] += pair_less(od, oi, dv[j], id[j]) ? 1 : 0;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kS; ++j)
            if (lane + 32 * j < n && rank[j] < k) {
                out_idx[q * k + rank[j]] = id[j];
                out_d2[q * k + rank[j]] = dv[j];
            }
        __syncwarp();
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
    int fold = 0;              // D < 64: the norm rides in column D of the operands
    float* Qh = nullptr;       // [Np][64] query operand -2 (x - centre): heads
    float* Ql = nullptr;       //   tails
    float* Ch = nullptr;       // [Np][64] candidate operand x - centre: heads
    float* Cl = nullptr;       //   tails
    float* nrm = nullptr;      // [Np]
    float* centre = nullptr;   // [64]
    double* part = nullptr;    // [nparts][64]
    unsigned* ctl = nullptr;   // [0] leftover count, [1] error word, [2] largest norm, [3] pacing
    float2* buf = nullptr;     // [grid][kQ][kBuf]
    int S = 0;                 // final shortlist capacity (32 x 2, 4, 8 or 16)
    float2* lists = nullptr;   // [N][S]
    int32_t* counts = nullptr;    // [N]
    int32_t* leftover = nullptr;  // [N]
    CUtensorMap mapQH, mapQL, mapCH, mapCL;
};

bool knn_tc_supported(int D, int k) { return D >= 1 && D <= knntc::kDp && k >= 1 && k <= kBuf / 2; }

void knn_tc_destroy(KnnTc* w) {
    if (!w) return;
    void* ps[] = {w->Qh, w->Ql, w->Ch, w->Cl, w->nrm, w->centre, w->part, w->ctl, w->buf, w->lists, w->counts,
                  w->leftover};
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
    // final shortlists: room for 2 k + 32 entries (the k nearest and the
    // candidates within the band of the k-th), a power of two of 32-entry slots
    const int need = (2 * k + 32 + 31) / 32;
    w->S = 32 * (need <= 2 ? 2 : need <= 4 ? 4 : need <= 8 ? 8 : 16);
    w->fold = D < kDp ? 1 : 0;
    int rc = tc_alloc(&w->Qh, (size_t)(w->Np * kDp), "kNN query heads");
    if (!rc) rc = tc_alloc(&w->Ql, (size_t)(w->Np * kDp), "kNN query tails");
    if (!rc) rc = tc_alloc(&w->Ch, (size_t)(w->Np * kDp), "kNN candidate heads");
    if (!rc) rc = tc_alloc(&w->Cl, (size_t)(w->Np * kDp), "kNN candidate tails");
    if (!rc) rc = tc_alloc(&w->nrm, (size_t)w->Np, "kNN norms");
    if (!rc) rc = tc_alloc(&w->centre, (size_t)kDp, "kNN centre");
    if (!rc) rc = tc_alloc(&w->part, (size_t)w->nparts * kDp, "kNN column sums");
    if (!rc) rc = tc_alloc(&w->ctl, 4, "kNN control words");
    if (!rc) rc = tc_alloc(&w->buf, (size_t)w->grid * kQ * kBuf, "kNN shortlists");
    if (!rc) rc = tc_alloc(&w->lists, (size_t)N * w->S, "kNN final shortlists");
    if (!rc) rc = tc_alloc(&w->counts, (size_t)N, "kNN shortlist sizes");
    if (!rc) rc = tc_alloc(&w->leftover, (size_t)N, "kNN leftover queries");
    if (!rc) {
        // the maps cover the Kp columns the K-steps read (boxes past them
        // read zeros and move no data)
        const int64_t Kp = std::max<int64_t>(32, 8 * ((D + w->fold + 7) / 8));
        int r2 = encode_map_f32_2d(&w->mapQH, w->Qh, w->Np, Kp, kDp, 32, kQ);
        if (!r2) r2 = encode_map_f32_2d(&w->mapQL, w->Ql, w->Np, Kp, kDp, 32, kQ);
        if (!r2) r2 = encode_map_f32_2d(&w->mapCH, w->Ch, w->Np, Kp, kDp, 32, kC);
        if (!r2) r2 = encode_map_f32_2d(&w->mapCL, w->Cl, w->Np, Kp, kDp, 32, kC);
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
        norms_kernel<<<(int)std::min<int64_t>((w->Np + 255) / 256, 4096), 256, 0, st>>>(X, w->N, w->D, w->Np,
                                                                                       w->centre, w->nrm, w->ctl + 2);
        const int64_t total = w->Np * kDp;
        split_points_kernel<<<(int)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, st>>>(
            X, w->N, w->D, w->Np, w->centre, w->nrm, w->fold, w->Qh, w->Ql, w->Ch, w->Cl);
        e = cudaGetLastError();
    }
    const void* kern = w->fold ? (const void*)knn_tc_kernel<true> : (const void*)knn_tc_kernel<false>;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e == cudaSuccess) {
        Args g;
        g.nrm = w->nrm;
        g.nmax = w->ctl + 2;
        g.N = w->N;
        g.k = w->k;
        g.ksteps = (w->D + w->fold + 7) / 8;
        g.nqt = (int)(w->Np / kQ);
        g.nct = (int)(w->Np / kC);
        g.buf = w->buf;
        g.lists = w->lists;
        g.counts = w->counts;
        g.S = w->S;
        g.flagged = w->leftover;
        g.nflagged = w->ctl;
        g.err = reinterpret_cast<int*>(w->ctl + 1);
        g.pace = w->ctl + 3;
        // cooperative: the CTAs pace each other, so all must be resident
        void* params[] = {(void*)&w->mapQH, (void*)&w->mapQL, (void*)&w->mapCH, (void*)&w->mapCL, (void*)&g};
        e = cudaLaunchCooperativeKernel(kern, dim3(w->grid), dim3(kThreads), params, kSmem, st);
    }
    if (e == cudaSuccess) {
        const int grid = (int)std::min<int64_t>((w->N + 7) / 8, 4096);
        switch (w->S / 32) {
            case 2: knn_rerank_kernel<2><<<grid, 256, 0, st>>>(X, w->N, w->D, w->k, w->lists, w->counts, out_idx, out_d2); break;
            case 4: knn_rerank_kernel<4><<<grid, 256, 0, st>>>(X, w->N, w->D, w->k, w->lists, w->counts, out_idx, out_d2); break;
            case 8: knn_rerank_kernel<8><<<grid, 256, 0, st>>>(X, w->N, w->D, w->k, w->lists, w->counts, out_idx, out_d2); break;
            default: knn_rerank_kernel<16><<<grid, 256, 0, st>>>(X, w->N, w->D, w->k, w->lists, w->counts, out_idx, out_d2); break;
        }
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return set_error(TSNE_ERR_CUDA, "tensor-core kNN launch: %s", cudaGetErrorString(e));
    *launches += 6;
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
