// Out-of-core randomized PCA (Sec. 6, Algorithm oocPCA) on sm_103a.
//
// The only operations with the large matrix A (m x n, FP32, row-major, in
// device memory or, out of core, in host memory streamed block by block)
// are two products per pass over A:
//   G1  Y_blk = A_blk W          (b x l: A_blk times an n x l matrix)
//   G2  G    += A_blk* Y_blk     (n x l: the adjoint product, same pass)
// Carrying G = A* Y through the pass is what lets a power iteration load A
// only once (the fused AA* pass of the paper's implementation notes). The
// next right-hand side A* L_i of Algorithm oocPCA (L_i U_i = Y_i) is
// G_i U_i^-1, whose column space is that of G_i; the renormalization is
// therefore the LU factorization with partial pivoting of G_i itself,
// W_{i+1} = L(G_i): the same column space (so the same Y_{i+1} up to an
// invertible mix of its columns, which no later step sees), entries bounded
// by 1 even when Y_i is rank-deficient (forming G_i U_i^-1 would divide
// rounding noise by the vanishing pivots of such a Y_i), and an LU over the
// n rows of G instead of the m rows of Y.
//
// G1 and G2 are dense contractions and run on the fifth-generation tensor
// cores: tcgen05.mma (kind::tf32, 128 x 64 tiles, FP32 accumulator in
// tensor memory) fed by TMA loads with the 128-byte swizzle. To keep FP32
// accuracy, every operand is split into a TF32 head and tail (x = hi + lo,
// hi rounded to TF32, lo = x - hi exact in FP32) and a tile accumulates
// hi*hi + hi*lo + lo*hi (the lo*lo term is below 2^-22 of the product):
// three MMAs per step. The split of the A tiles happens in shared memory
// (converter warps) between the TMA load and the MMAs; for G2 the converter
// also transposes the tile, so both products read K-major operands.
//
// Warp roles of a GEMM CTA (384 threads): warp 0 issues the TMA loads, warp
// 1 owns the tensor memory and issues the MMAs (one thread), warps 2..7
// split (and transpose) the A tiles, warps 8..11 read the accumulators back
// (tcgen05.ld: warp w reads lanes 32 (w % 4) .. + 31) chain after chain and
// write the result. Stages and accumulators are handed over with mbarriers;
// every wait is bounded: a wait that gives up sets the error word, and the
// kernel finishes without further MMAs.
//
// The small steps (LU with partial pivoting of G, the QR of Y by shifted
// Cholesky QR, the SVD of the small matrix Q* A) run in FP64 in plain CUDA
// kernels below.
#include <cuda.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "fitsne_internal.cuh"
#include "fitsne_tc.cuh"
#include "oocpca_gb300.h"

namespace oocpca {

constexpr int kTileM = 128;  // rows of an MMA tile (tensor-memory lanes)
constexpr int kTileN = 64;   // columns of the accumulator (l <= 64)
constexpr int kStageK = 32;  // K of one pipeline stage: 32 FP32 = one 128-byte swizzle row
constexpr int kThreads = 384;
template <int MODE> struct Stages;  // pipeline depth per mode (shared memory: 192 KB each)
constexpr int kConvWarpFirst = 2;  // converter warps 2..7
constexpr int kConvWarps = 6;
constexpr int kEpiWarpFirst = 8;   // epilogue warps 8..11 (warp % 4 = tensor-memory lane quarter)
// The tensor cores' FP32 accumulator does not round each addition to
// nearest, so a long chain of MMAs into one accumulator drifts by up to
// about 2^-24 per added term (measured: 4e-4 of sigma_1 with K = 30,000).
// A chain therefore covers kChainStages stages (256 K-elements); the
// epilogue warps add every chain's accumulator into registers (FP32, round
// to nearest) while the next chain runs in the other of two accumulators.
constexpr int kChainStages = 8;

using namespace tc;

constexpr uint32_t kIdesc = idesc_tf32(kTileM, kTileN);

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
    tc::mma_tf32(tmem_d, a, b, kIdesc, accumulate);
}

}  // namespace oocpca

namespace oocpca {


enum : int { kModeAW = 0, kModeATY = 1 };

// One launch of G1 (mode kModeAW) or G2 (kModeATY) over a block of rows.
struct GemmArgs {
    int rows;            // rows of A in this block
    int cols;            // n
    int row_offset;      // index of the block's first row in Y (G1 output, G2 operand)
    int k_stages;        // G2: stages (32 rows each) per K split
    int n_tiles;         // G2: column tiles (ceil(n / 128))
    float* yt;           // G1: Y^T FP32, 64 x ldy (row j = column j of Y)
    float* yt_hi;        // G1: its TF32 head and tail
    float* yt_lo;
    int64_t ldy;
    const float* shift;  // G1: subtracted from column j of Y (centring; may be NULL)
    float* gpart;        // G2: partial products [split][n][64]
    int* err;            // error word (kErrTimeout)
};

template <> struct Stages<kModeAW> { static constexpr int value = 4; };   // 48 KB per stage
template <> struct Stages<kModeATY> { static constexpr int value = 3; };  // 64 KB per stage

template <int MODE>
struct StageLayout {
    // G1: raw A (TF32 head in place) | A tail | B head | B tail
    // G2: raw A (4 boxes of 32 rows) | A head | A tail | B head | B tail
    static constexpr uint32_t kA = kTileM * kStageK * 4;     // 16 KB
    static constexpr uint32_t kB = kTileN * kStageK * 4;     //  8 KB
    static constexpr uint32_t raw = 0;
    static constexpr uint32_t hi = (MODE == kModeAW) ? 0 : kA;
    static constexpr uint32_t lo = (MODE == kModeAW) ? kA : 2 * kA;
    static constexpr uint32_t bhi = lo + kA;
    static constexpr uint32_t blo = bhi + kB;
    static constexpr uint32_t bytes = blo + kB;
    static constexpr uint32_t tx = kA + 2 * kB;              // bytes the TMA delivers per stage
    static constexpr uint32_t smem = Stages<MODE>::value * bytes + 1024; // + alignment slack
};

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1)
pca_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapBh,
                const __grid_constant__ CUtensorMap mapBl, GemmArgs g) {
    using SL = StageLayout<MODE>;
    constexpr int kStages = Stages<MODE>::value;
    extern __shared__ unsigned char smem_dyn[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[4], conv_bar[4], empty_bar[4];
    __shared__ __align__(8) uint64_t tfull_bar[2], tempty_bar[2];
    __shared__ uint32_t s_tmem;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    // this CTA's tile and K range
    int m0, kbeg, nk, split = 0;
    if (MODE == kModeAW) {
        m0 = blockIdx.x * kTileM;                 // rows of A
        kbeg = 0;
        nk = (g.cols + kStageK - 1) / kStageK;    // K = n
    } else {
        m0 = (blockIdx.x % g.n_tiles) * kTileM;   // columns of A
        split = blockIdx.x / g.n_tiles;
        kbeg = split * g.k_stages * kStageK;      // K = rows of the block
        const int kend = min(g.rows, kbeg + g.k_stages * kStageK);
        nk = kend > kbeg ? (kend - kbeg + kStageK - 1) / kStageK : 0;
    }
    const int nchains = (nk + kChainStages - 1) / kChainStages;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&conv_bar[s]), kConvWarps);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&tfull_bar[b]), 1);
            mbar_init(smem_u32(&tempty_bar[b]), 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_shared();
    }
    if (warp == 1) {  // tensor memory: two accumulators of 64 columns x 128 lanes (FP32)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&s_tmem)), "r"(2 * kTileN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == 0) {
        if (lane == 0) {  // TMA producer
            int issued = 0;
            for (int i = 0; i < nk; ++i) {
                const int s = i % kStages;
                const uint32_t ph = (uint32_t)(i / kStages) & 1u;
                if (!mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1u, g.err)) break;
                unsigned char* st = smem + s * SL::bytes;
                const uint32_t fb = smem_u32(&full_bar[s]);
                mbar_expect_tx(fb, SL::tx);
                const int k0 = kbeg + i * kStageK;
                if (MODE == kModeAW) {
                    tma_load_2d(smem_u32(st + SL::raw), &mapA, k0, m0, fb);
                    tma_load_2d(smem_u32(st + SL::bhi), &mapBh, k0, 0, fb);
                    tma_load_2d(smem_u32(st + SL::blo), &mapBl, k0, 0, fb);
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        tma_load_2d(smem_u32(st + SL::raw + q * 4096), &mapA, m0 + 32 * q, k0, fb);
                    tma_load_2d(smem_u32(st + SL::bhi), &mapBh, g.row_offset + k0, 0, fb);
                    tma_load_2d(smem_u32(st + SL::blo), &mapBl, g.row_offset + k0, 0, fb);
                }
                issued = i + 1;
            }
            // every load issued must have landed before the CTA may leave
            for (int i = max(0, issued - kStages); i < issued; ++i)
                mbar_wait_drain(smem_u32(&full_bar[i % kStages]), (uint32_t)(i / kStages) & 1u);
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            int committed = -1;  // last chain committed
            for (int i = 0; i < nk; ++i) {
                const int s = i % kStages;
                const uint32_t ph = (uint32_t)(i / kStages) & 1u;
                const int c = i / kChainStages, b = c & 1;
                if (i % kChainStages == 0) {  // a new chain: its accumulator must have been read
                    if (!mbar_wait(smem_u32(&tempty_bar[b]), ((uint32_t)(c >> 1) & 1u) ^ 1u, g.err)) break;
                    tc_fence_after();
                }
                if (!mbar_wait(smem_u32(&conv_bar[s]), ph, g.err)) break;
                tc_fence_after();
                const unsigned char* st = smem + s * SL::bytes;
                const uint64_t ah = sw128_desc(smem_u32(st + SL::hi));
                const uint64_t al = sw128_desc(smem_u32(st + SL::lo));
                const uint64_t bh = sw128_desc(smem_u32(st + SL::bhi));
                const uint64_t bl = sw128_desc(smem_u32(st + SL::blo));
                const uint32_t acc = tmem + (uint32_t)(b * kTileN);
                const uint32_t first = (i % kChainStages) == 0;
#pragma unroll
                for (int kk = 0; kk < kStageK / 8; ++kk) {  // K = 8 per MMA: 32 bytes = 2 in the address field
                    const uint64_t o = (uint64_t)(2 * kk);
                    mma_tf32(acc, ah + o, bh + o, (first && kk == 0) ? 0u : 1u);
                    mma_tf32(acc, ah + o, bl + o, 1u);
                    mma_tf32(acc, al + o, bh + o, 1u);
                }
                mma_commit(smem_u32(&empty_bar[s]));  // the stage is free once these MMAs are done
                if (i % kChainStages == kChainStages - 1 || i == nk - 1) {
                    mma_commit(smem_u32(&tfull_bar[b]));  // the chain's accumulator is complete
                    committed = c;
                }
            }
            // the MMAs must be complete before the tensor memory is released
            if (committed >= 0)
                mbar_wait_drain(smem_u32(&tfull_bar[committed & 1]), (uint32_t)(committed >> 1) & 1u);
        }
    } else if (warp < kEpiWarpFirst) {
        // converters: TF32 head / tail of the A tile (G2: transposed to K-major)
        const int ct = threadIdx.x - kConvWarpFirst * 32;  // 0 .. 191
        for (int i = 0; i < nk; ++i) {
            const int s = i % kStages;
            const uint32_t ph = (uint32_t)(i / kStages) & 1u;
            if (!mbar_wait(smem_u32(&full_bar[s]), ph, g.err)) break;
            unsigned char* st = smem + s * SL::bytes;
            if (MODE == kModeAW) {
                float4* raw = reinterpret_cast<float4*>(st + SL::raw);
                float4* lo = reinterpret_cast<float4*>(st + SL::lo);
                for (int v = ct; v < kTileM * kStageK / 4; v += kConvWarps * 32) {
                    float4 x = raw[v], h, t;
                    h.x = tf32_head(x.x); t.x = x.x - h.x;
                    h.y = tf32_head(x.y); t.y = x.y - h.y;
                    h.z = tf32_head(x.z); t.z = x.z - h.z;
                    h.w = tf32_head(x.w); t.w = x.w - h.w;
                    raw[v] = h;
                    lo[v] = t;
                }
            } else {
                // raw box q holds A rows k = 0..31 (of this stage) x columns 32 q + c
                const unsigned char* raw = st + SL::raw;
                unsigned char* hi = st + SL::hi;
                unsigned char* lo = st + SL::lo;
                // a thread takes 4 consecutive rows k0..k0+3 of one column: 4 loads,
                // one 16-byte store of head and of tail (a chunk of the K-major row)
                for (int e = ct; e < kTileM * kStageK / 4; e += kConvWarps * 32) {
                    const int c = e % 32, k0 = ((e / 32) % 8) * 4, q = e / 256;
                    const unsigned char* box = raw + q * 4096;
                    float4 x, h, t;
                    x.x = *reinterpret_cast<const float*>(box + sw128_offset(k0, c));
                    x.y = *reinterpret_cast<const float*>(box + sw128_offset(k0 + 1, c));
                    x.z = *reinterpret_cast<const float*>(box + sw128_offset(k0 + 2, c));
                    x.w = *reinterpret_cast<const float*>(box + sw128_offset(k0 + 3, c));
                    h.x = tf32_head(x.x); t.x = x.x - h.x;
                    h.y = tf32_head(x.y); t.y = x.y - h.y;
                    h.z = tf32_head(x.z); t.z = x.z - h.z;
                    h.w = tf32_head(x.w); t.w = x.w - h.w;
                    const uint32_t o = sw128_offset(32 * q + c, k0);  // 16-byte aligned: k0 % 4 == 0
                    *reinterpret_cast<float4*>(hi + o) = h;
                    *reinterpret_cast<float4*>(lo + o) = t;
                }
            }
            fence_async_shared();  // generic-proxy writes become visible to the tensor cores
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&conv_bar[s]));
        }
    } else {
        // epilogue: add each chain's accumulator (FP32, round to nearest), then write
        const int q = warp % 4;                            // tensor-memory lanes 32 q .. 32 q + 31
        const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16);
        float v[kTileN];
#pragma unroll
        for (int c = 0; c < kTileN; ++c) v[c] = 0.0f;
        bool ok = true;
        for (int c = 0; c < nchains; ++c) {
            const int b = c & 1;
            if (!mbar_wait(smem_u32(&tfull_bar[b]), (uint32_t)(c >> 1) & 1u, g.err)) { ok = false; break; }
            tc_fence_after();
#pragma unroll
            for (int cc = 0; cc < kTileN; cc += 16) {
                float t[16];
                tmem_ld16(lane_addr + (uint32_t)(b * kTileN + cc), t);
#pragma unroll
                for (int u = 0; u < 16; ++u) v[cc + u] += t[u];
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&tempty_bar[b]));
        }
        const int r = m0 + 32 * q + lane;                  // G1: row of A; G2: column of A
        if (ok && MODE == kModeAW) {
            if (r < g.rows) {
                const int64_t col = (int64_t)g.row_offset + r;
#pragma unroll
                for (int j = 0; j < kTileN; ++j) {
                    const float y = g.shift ? v[j] - g.shift[j] : v[j];
                    const float h = tf32_head(y);
                    g.yt[j * g.ldy + col] = y;
                    g.yt_hi[j * g.ldy + col] = h;
                    g.yt_lo[j * g.ldy + col] = y - h;
                }
            }
        } else if (ok && r < g.cols) {
            float4* dst = reinterpret_cast<float4*>(g.gpart + ((int64_t)split * g.cols + r) * kTileN);
#pragma unroll
            for (int j = 0; j < kTileN / 4; ++j)
                dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTileN)
                     : "memory");
    }
}

}  // namespace oocpca

// ---------------------------------------------------------------------------
// FP64 small steps. Matrices with l <= 64 columns are kept "column-major":
// column j of an R x l matrix at X[j * ld + r] (rows contiguous), so that a
// thread per row reads and writes coalesced.
// ---------------------------------------------------------------------------
namespace oocpca {

constexpr int kSmallBlocks = 304;  // grid of the row-parallel small kernels (2 per SM)

// TF32 head and tail of the columns of X (R x l, column-major FP64, ldx) as
// the 64-row K-major operand: dst_hi / dst_lo [j * ldd + r], rows j >= l and
// columns r in [R, ldd) zero.
__global__ void split_operand_kernel(const double* __restrict__ X, int64_t ldx, int64_t R, int l,
                                     float* __restrict__ hi, float* __restrict__ lo, int64_t ldd) {
    const int64_t total = (int64_t)kTileN * ldd;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / ldd);
        const int64_t r = e - (int64_t)j * ldd;
        const float x = (j < l && r < R) ? (float)X[j * ldx + r] : 0.0f;
        const float h = tf32_head(x);
        hi[e] = h;
        lo[e] = x - h;
    }
}

// Gd[j * ld + c] (+)= sum over the splits of gpart[split][c][j] - mu[c] colsum[j]
// (FP64, splits in order): the pass's adjoint product A* Y, centred if mu.
__global__ void reduce_adjoint_kernel(const float* __restrict__ gpart, int nsplit, int64_t n, int l,
                                      const double* __restrict__ mu, const double* __restrict__ colsum,
                                      int accumulate, double* __restrict__ Gd, int64_t ld) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * l;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / l;
        const int j = (int)(e - c * l);
        double t = 0.0;
        for (int sp = 0; sp < nsplit; ++sp) t += (double)gpart[((int64_t)sp * n + c) * kTileN + j];
        if (mu) t -= mu[c] * colsum[j];
        double* d = &Gd[j * ld + c];
        *d = accumulate ? *d + t : t;
    }
}

// Y (FP32 transposed, 64 x ldy) to column-major FP64 (l x m).
__global__ void widen_kernel(const float* __restrict__ yt, int64_t ldy, int64_t m, int l,
                             double* __restrict__ Yd) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)l * m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / m);
        const int64_t r = e - (int64_t)j * m;
        Yd[e] = (double)yt[j * ldy + r];
    }
}

// Sums of the columns of a column-major R x l matrix (FP64, fixed order:
// per block, then by the last block): out[j]. Used for 1* Y (centring).
__global__ void __launch_bounds__(256)
colsum_kernel(const double* __restrict__ X, int64_t ld, int64_t R, int l, double* __restrict__ part,
              unsigned* __restrict__ ticket, double* __restrict__ out) {
    __shared__ double s[8];
    __shared__ bool s_last;
    const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
    for (int j = 0; j < l; ++j) {
        double t = 0.0;
        for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x)
            t += X[j * ld + r];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) s[wid] = t;
        __syncthreads();
        if (threadIdx.x == 0) {
            double u = 0.0;
            for (int w = 0; w < 8; ++w) u += s[w];
            part[(int64_t)blockIdx.x * kTileN + j] = u;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x < l) {
        double u = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) u += __ldcg(&part[(int64_t)b * kTileN + threadIdx.x]);
        out[threadIdx.x] = u;
    }
    if (threadIdx.x == 0) *ticket = 0u;
}

// LU with partial pivoting of X (column-major R x l, FP64, overwritten), one
// column per launch pair. Step j, pivot: the row with the largest |X[j][r]|
// among the rows not yet pivotal (ties: the smaller row) becomes pivot j
// (flag j + 1), and its entries j..l-1 become row j of U.
__global__ void __launch_bounds__(256)
lu_pivot_kernel(const double* __restrict__ Y, int64_t m, int l, int j,
                const unsigned char* __restrict__ used, double* __restrict__ part_v,
                int64_t* __restrict__ part_i, unsigned* __restrict__ ticket,
                unsigned char* __restrict__ used_out, int64_t* __restrict__ piv, double* __restrict__ U) {
    __shared__ double sv[8];
    __shared__ int64_t si[8];
    __shared__ bool s_last;
    const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
    double bv = -1.0;
    int64_t bi = INT64_MAX;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
        if (used[r]) continue;
        const double a = fabs(Y[(int64_t)j * m + r]);
        if (a > bv) { bv = a; bi = r; }  // r increases: the first of equal values is kept
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { sv[wid] = bv; si[wid] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w)
            if (sv[w] > bv || (sv[w] == bv && si[w] < bi)) { bv = sv[w]; bi = si[w]; }
        part_v[blockIdx.x] = bv;
        part_i[blockIdx.x] = bi;
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    bv = -1.0;
    bi = INT64_MAX;
    for (unsigned b = 0; b < gridDim.x; ++b) {
        const double v = __ldcg(&part_v[b]);
        const int64_t i = __ldcg(&part_i[b]);
        if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
    }
    *ticket = 0u;
    if (bi == INT64_MAX) bi = 0;  // cannot happen for l < m
    piv[j] = bi;
    used_out[bi] = (unsigned char)(j + 1);
    for (int c = j; c < l; ++c) U[j * kTileN + c] = Y[(int64_t)c * m + bi];
}

// Step j, elimination: every row not yet pivotal loses f times the pivot
// row, f = X[j][r] / U[j][j] (an exactly zero pivot eliminates nothing), and
// keeps f in column j: the multipliers are the entries of L.
__global__ void lu_elim_kernel(double* __restrict__ Y, int64_t m, int l, int j,
                               const unsigned char* __restrict__ used, const double* __restrict__ U) {
    const double d = U[j * kTileN + j];
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
        if (used[r]) continue;
        const double f = d != 0.0 ? Y[(int64_t)j * m + r] / d : 0.0;
        Y[(int64_t)j * m + r] = f;
        for (int c = j + 1; c < l; ++c) Y[(int64_t)c * m + r] -= f * U[j * kTileN + c];
    }
}

// L of the factorization in place: a row pivotal at step t holds 1 in column
// t and 0 after it (its multipliers before t stay), so that X = L with
// P X_in = L' U, |L| <= 1.
__global__ void lu_finalize_kernel(double* __restrict__ X, int64_t R, int l,
                                   const unsigned char* __restrict__ used) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        const int t = (int)used[r] - 1;
        if (t < 0) continue;
        X[(int64_t)t * R + r] = 1.0;
        for (int c = t + 1; c < l; ++c) X[(int64_t)c * R + r] = 0.0;
    }
}

// W = G U^-1 (n x l, column-major, FP64): forward substitution along each
// row, w_j = (g_j - sum_{i<j} w_i U[i][j]) / U[j][j]; a zero U[j][j] (an
// exactly rank-deficient Y) divides by 1 instead.
__global__ void right_solve_kernel(const double* __restrict__ G, int64_t ld, int64_t n, int l,
                                   const double* __restrict__ U, double* __restrict__ W) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        double w[kTileN];
        for (int j = 0; j < l; ++j) {
            double t = G[j * ld + c];
            for (int i = 0; i < j; ++i) t -= w[i] * U[i * kTileN + j];
            const double d = U[j * kTileN + j];
            w[j] = t / (d != 0.0 ? d : 1.0);
            W[j * ld + c] = w[j];
        }
    }
}

// Gram matrix C = X* X (l x l, FP64) of a column-major R x l matrix: each
// block sums the products over its rows in chunks staged in shared memory,
// the last block adds the blocks' partials in order (C[i * 64 + j], full).
__global__ void __launch_bounds__(256)
gram_kernel(const double* __restrict__ X, int64_t ld, int64_t R, int l, double* __restrict__ part,
            unsigned* __restrict__ ticket, double* __restrict__ C) {
    constexpr int kRows = 32;
    __shared__ double xs[kTileN][kRows + 1];
    __shared__ bool s_last;
    const int npair = l * (l + 1) / 2;
    double acc[9];
    int pi[9], pj[9];
    int np = 0;
    for (int p = threadIdx.x; p < npair && np < 9; p += blockDim.x, ++np) {
        int i = 0, rem = p;
        while (rem >= l - i) { rem -= l - i; ++i; }
        pi[np] = i;
        pj[np] = i + rem;
        acc[np] = 0.0;
    }
    const int64_t chunks = (R + kRows - 1) / kRows;
    for (int64_t ch = blockIdx.x; ch < chunks; ch += gridDim.x) {
        const int64_t r0 = ch * kRows;
        __syncthreads();
        for (int e = threadIdx.x; e < l * kRows; e += blockDim.x) {
            const int j = e / kRows, rr = e % kRows;
            xs[j][rr] = (r0 + rr < R) ? X[j * ld + r0 + rr] : 0.0;
        }
        __syncthreads();
        for (int q = 0; q < np; ++q) {
            double t = 0.0;
            for (int rr = 0; rr < kRows; ++rr) t += xs[pi[q]][rr] * xs[pj[q]][rr];
            acc[q] += t;
        }
    }
    for (int q = 0; q < np; ++q) part[(int64_t)blockIdx.x * (kTileN * kTileN) + pi[q] * kTileN + pj[q]] = acc[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int p = threadIdx.x; p < npair; p += blockDim.x) {
        int i = 0, rem = p;
        while (rem >= l - i) { rem -= l - i; ++i; }
        const int j = i + rem;
        double t = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) t += __ldcg(&part[(int64_t)b * (kTileN * kTileN) + i * kTileN + j]);
        C[i * kTileN + j] = t;
        C[j * kTileN + i] = t;
    }
    if (threadIdx.x == 0) *ticket = 0u;
}

// Cholesky C + shift I = R* R (R upper, l x l in a 64 x 64 array), one CTA.
// shift_scale > 0 adds the shift of shifted Cholesky QR (Fukaya, Kannan,
// Nakatsukasa, Yamamoto and Yanagisawa, SIAM J. Sci. Comput. 2020):
// s = shift_scale * u * ||X||_F^2 with ||X||_F^2 = trace(C), u = 2^-53. A
// pivot that is not positive (rounding on a rank-deficient X) is replaced by
// the largest of the shift and 2^-40 trace(C), so that R stays invertible.
__global__ void cholesky_kernel(const double* __restrict__ Cin, int l, double shift_scale,
                                double* __restrict__ R) {
    __shared__ double A[kTileN][kTileN + 1];
    __shared__ double s_tr;
    for (int e = threadIdx.x; e < kTileN * kTileN; e += blockDim.x) {
        const int i = e / kTileN, j = e % kTileN;
        A[i][j] = (i < l && j < l) ? Cin[i * kTileN + j] : 0.0;
        R[e] = 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < l; ++i) t += A[i][i];
        s_tr = t;
    }
    __syncthreads();
    const double tr = s_tr;
    const double shift = shift_scale * 0x1p-53 * tr;
    const double floor_p = fmax(shift, 0x1p-40 * tr);
    if (threadIdx.x < l) A[threadIdx.x][threadIdx.x] += shift;
    __syncthreads();
    for (int k = 0; k < l; ++k) {
        __shared__ double s_d;
        if (threadIdx.x == 0) {
            double d = A[k][k];
            if (!(d > 0.0)) d = floor_p > 0.0 ? floor_p : 1.0;
            s_d = sqrt(d);
            R[k * kTileN + k] = s_d;
        }
        __syncthreads();
        const double d = s_d;
        for (int j = k + 1 + threadIdx.x; j < l; j += blockDim.x) R[k * kTileN + j] = A[k][j] / d;
        __syncthreads();
        for (int e = threadIdx.x; e < (l - k - 1) * (l - k - 1); e += blockDim.x) {
            const int i = k + 1 + e / (l - k - 1), j = k + 1 + e % (l - k - 1);
            if (j >= i) A[i][j] -= R[k * kTileN + i] * R[k * kTileN + j];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < (l - k - 1) * (l - k - 1); e += blockDim.x) {
            const int i = k + 1 + e / (l - k - 1), j = k + 1 + e % (l - k - 1);
            if (j < i) A[i][j] = A[j][i];
        }
        __syncthreads();
    }
}

// Symmetric eigendecomposition H = V diag(lambda) V* (l x l, FP64) by cyclic
// Jacobi rotations in the round-robin order (each round rotates l / 2
// disjoint pairs at once), until every off-diagonal entry is below 1e-15 of
// the largest diagonal one or 40 sweeps; then sigma_j = sqrt(max(lambda_j,
// 0)) in decreasing order, with the matching columns of V (each column's
// largest entry made positive). One CTA of 256 threads.
__global__ void jacobi_svd_kernel(const double* __restrict__ Hin, int l, double* __restrict__ Vout,
                                  double* __restrict__ sigma) {
    __shared__ double H[kTileN][kTileN + 1];
    __shared__ double V[kTileN][kTileN + 1];
    __shared__ double cs[kTileN / 2], sn[kTileN / 2];
    __shared__ int pp[kTileN / 2], qq[kTileN / 2];
    __shared__ double s_off, s_diag;
    __shared__ int order[kTileN];
    const int L = (l + 1) & ~1;  // even number of players (a dummy one when l is odd)
    for (int e = threadIdx.x; e < kTileN * kTileN; e += blockDim.x) {
        const int i = e / kTileN, j = e % kTileN;
        H[i][j] = (i < l && j < l) ? Hin[i * kTileN + j] : 0.0;
        V[i][j] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int sweep = 0; sweep < 40; ++sweep) {
        if (threadIdx.x == 0) {
            double off = 0.0, dg = 0.0;
            for (int i = 0; i < l; ++i) {
                dg = fmax(dg, fabs(H[i][i]));
                for (int j = i + 1; j < l; ++j) off = fmax(off, fabs(H[i][j]));
            }
            s_off = off;
            s_diag = dg;
        }
        __syncthreads();
        if (!(s_off > 1e-15 * s_diag)) break;
        for (int r = 0; r < L - 1; ++r) {
            if (threadIdx.x < L / 2) {
                const int k = threadIdx.x;
                auto player = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + r) % (L - 1); };
                int p = player(k), q = player(L - 1 - k);
                if (p > q) { const int t = p; p = q; q = t; }
                double c = 1.0, s = 0.0;
                if (q < l && H[p][q] != 0.0) {
                    const double th = (H[q][q] - H[p][p]) / (2.0 * H[p][q]);
                    const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                    c = 1.0 / sqrt(t * t + 1.0);
                    s = t * c;
                }
                pp[k] = p;
                qq[k] = q < l ? q : p;
                cs[k] = c;
                sn[k] = (q < l) ? s : 0.0;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < (L / 2) * l; e += blockDim.x) {  // rows p, q
                const int k = e / l, x = e % l, p = pp[k], q = qq[k];
                if (p == q) continue;
                const double a = H[p][x], b = H[q][x];
                H[p][x] = cs[k] * a - sn[k] * b;
                H[q][x] = sn[k] * a + cs[k] * b;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < (L / 2) * l; e += blockDim.x) {  // columns p, q
                const int k = e / l, x = e % l, p = pp[k], q = qq[k];
                if (p == q) continue;
                const double a = H[x][p], b = H[x][q];
                H[x][p] = cs[k] * a - sn[k] * b;
                H[x][q] = sn[k] * a + cs[k] * b;
                const double va = V[x][p], vb = V[x][q];
                V[x][p] = cs[k] * va - sn[k] * vb;
                V[x][q] = sn[k] * va + cs[k] * vb;
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < l; ++i) order[i] = i;
        for (int i = 1; i < l; ++i)  // insertion sort, decreasing eigenvalue (ties by index)
            for (int j = i; j > 0 && H[order[j]][order[j]] > H[order[j - 1]][order[j - 1]]; --j) {
                const int t = order[j]; order[j] = order[j - 1]; order[j - 1] = t;
            }
        for (int j = 0; j < l; ++j) sigma[j] = sqrt(fmax(H[order[j]][order[j]], 0.0));
    }
    __syncthreads();
    for (int j = threadIdx.x; j < l; j += blockDim.x) {
        const int c = order[j];
        int arg = 0;
        for (int i = 1; i < l; ++i)
            if (fabs(V[i][c]) > fabs(V[arg][c])) arg = i;
        const double sg = V[arg][c] < 0.0 ? -1.0 : 1.0;
        for (int i = 0; i < kTileN; ++i) Vout[i * kTileN + j] = (i < l) ? sg * V[i][c] : 0.0;
    }
}

// out (R x k, row-major FP32) = X (R x l, column-major FP64) * M[:, 0..k)
// (l x k in a 64 x 64 array), each column scaled by 1 / scale[j] if scale
// (0 where scale[j] is 0).
__global__ void small_product_kernel(const double* __restrict__ X, int64_t ld, int64_t R, int l, int k,
                                     const double* __restrict__ M, const double* __restrict__ scale,
                                     float* __restrict__ out) {
    __shared__ double Ms[kTileN * kTileN];
    for (int e = threadIdx.x; e < kTileN * kTileN; e += blockDim.x) Ms[e] = M[e];
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        double x[kTileN];
        for (int i = 0; i < l; ++i) x[i] = X[i * ld + r];
        for (int j = 0; j < k; ++j) {
            double t = 0.0;
            for (int i = 0; i < l; ++i) t += x[i] * Ms[i * kTileN + j];
            if (scale) t = scale[j] > 0.0 ? t / scale[j] : 0.0;
            out[r * k + j] = (float)t;
        }
    }
}

// Per-block FP64 column sums of rows [0, rows) of a row-major FP32 block
// (lda): part[blockIdx.y][c], the block's rows split over gridDim.y.
__global__ void colsum_rows_kernel(const float* __restrict__ A, int64_t rows, int64_t n, int64_t lda,
                                   double* __restrict__ part) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int64_t per = (rows + gridDim.y - 1) / gridDim.y;
    const int64_t r0 = (int64_t)blockIdx.y * per, r1 = min(rows, r0 + per);
    double t = 0.0;
    for (int64_t r = r0; r < r1; ++r) t += (double)A[r * lda + c];
    part[(int64_t)blockIdx.y * n + c] += t;
}

// mu[c] = sum over the gridDim.y partial rows / m.
__global__ void mean_finish_kernel(const double* __restrict__ part, int ny, int64_t n, int64_t m,
                                   double* __restrict__ mu) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int y = 0; y < ny; ++y) t += part[(int64_t)y * n + c];
        mu[c] = t / (double)m;
    }
}

// shift[j] = sum_c mu[c] W[c][j] (FP32 out: G1 subtracts it from column j of
// Y, which centres A W), one block per column j.
__global__ void __launch_bounds__(256)
mean_shift_kernel(const double* __restrict__ mu, const double* __restrict__ W, int64_t ld, int64_t n,
                  float* __restrict__ shift) {
    __shared__ double s[8];
    const int j = blockIdx.x;
    double t = 0.0;
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) t += mu[c] * W[j * ld + c];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x % 32 == 0) s[threadIdx.x / 32] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int w = 0; w < 8; ++w) u += s[w];
        shift[j] = (float)u;
    }
}

// Gd[j][c] -= mu[c] colsum[j]: the adjoint product of the centred matrix.
__global__ void center_adjoint_kernel(double* __restrict__ Gd, int64_t ld, int64_t n, int l,
                                      const double* __restrict__ mu, const double* __restrict__ colsum) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * l;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / n);
        const int64_t c = e - (int64_t)j * n;
        Gd[j * ld + c] -= mu[c] * colsum[j];
    }
}

// W (n x l, column-major FP64) from a row-major FP32 n x l matrix (Omega).
__global__ void omega_kernel(const float* __restrict__ Om, int64_t n, int l, double* __restrict__ W,
                             int64_t ld) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * l;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / l;
        const int j = (int)(e - c * l);
        W[j * ld + c] = (double)Om[e];
    }
}

}  // namespace oocpca

// ---------------------------------------------------------------------------
// Host side: the plan, the passes over A, the ABI.
// ---------------------------------------------------------------------------
namespace {

using namespace oocpca;
using fitsne::set_error;

int cuda_fail(cudaError_t e, const char* what) {
    return set_error(TSNE_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CU(call, what)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);  \
    } while (0)

// 2-D FP32 tensor map over rows x cols (row stride ld elements) with a box of
// box_cols x box_rows and the 128-byte swizzle; out-of-range boxes read zeros.
int make_map(CUtensorMap* map, const float* base, int64_t rows, int64_t cols, int64_t ld, int box_cols,
             int box_rows) {
    const int r = encode_map_f32_2d(map, base, rows, cols, ld, box_cols, box_rows);
    if (r < 0) return set_error(TSNE_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    if (r != 0) return set_error(TSNE_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", r);
    return TSNE_OK;
}

template <typename T>
int dalloc(T** p, size_t count, const char* what) {
    *p = nullptr;
    const cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(1, count) * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return set_error(e == cudaErrorMemoryAllocation ? TSNE_ERR_OOM : TSNE_ERR_CUDA,
                         "cudaMalloc of %s (%zu bytes): %s", what, count * sizeof(T), cudaGetErrorString(e));
    }
    return TSNE_OK;
}

int grid_of(int64_t items, int per) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(kSmallBlocks * 4, (items + per - 1) / per));
}

}  // namespace

struct tsne_oocpca {
    int64_t m, n;
    int k, l, its, center;
    int64_t block_rows;
    cudaStream_t st;
    cudaStream_t copy_st;
    cudaEvent_t copied[2], used[2];
    int sm_count;
    int64_t ldy, ldw;       // columns of the 64-row operands (m, n rounded up to 32)
    int nsplit_max;
    int64_t launches;
    int ran;
    int passes;
    double ms[4];
    // device workspace
    float *yt, *yt_hi, *yt_lo;  // 64 x ldy
    float *w_hi, *w_lo;         // 64 x ldw
    float* gpart;               // [nsplit_max][n][64]
    double *Gd, *Wd;            // column-major n x 64
    double* Yd;                 // column-major m x 64 (LU and QR workspace)
    double *Y0d, *G0d;          // first pass, for the test hook
    unsigned char* used_rows;   // [max(m, n)] pivot step + 1 of each row (0: not pivotal)
    int64_t* piv;               // [64]
    double *Um, *Cm, *Rm, *Vm, *sig;  // 64 x 64 (U of the LU, Gram, Cholesky R, eigenvectors), [64]
    double* part;               // Gram partials [kSmallBlocks][64][64]
    double* part_v;             // [4 kSmallBlocks]
    int64_t* part_i;            // [4 kSmallBlocks]
    double *mu, *colsum, *mu_part;  // [n], [64], [64][n]
    float* shiftf;              // [64]
    unsigned* ticket;           // self-resetting completion counter
    int* err;
    float* blk[2];              // device block buffers (host-resident A)
    CUtensorMap mapYh, mapYl, mapWh, mapWl;
};

namespace {

void free_plan(tsne_oocpca* p) {
    void* ptrs[] = {p->yt, p->yt_hi, p->yt_lo, p->w_hi, p->w_lo, p->gpart, p->Gd, p->Wd, p->Yd, p->Y0d,
                    p->G0d, p->used_rows, p->piv, p->Um, p->Cm, p->Rm, p->Vm, p->sig, p->part,
                    p->part_v, p->part_i, p->mu, p->colsum, p->mu_part, p->shiftf, p->ticket, p->err,
                    p->blk[0], p->blk[1]};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    for (int i = 0; i < 2; ++i) {
        if (p->copied[i]) cudaEventDestroy(p->copied[i]);
        if (p->used[i]) cudaEventDestroy(p->used[i]);
    }
    if (p->copy_st) cudaStreamDestroy(p->copy_st);
    delete p;
}

// The G1 / G2 launches of one block (rows [r0, r0 + rows) of A at Ablk).
int block_products(tsne_oocpca* p, const float* Ablk, int64_t lda, int64_t r0, int64_t rows, bool with_g1,
                   bool accumulate) {
    CUtensorMap mA1, mA2;
    if (with_g1)
        if (int rc = make_map(&mA1, Ablk, rows, p->n, lda, 32, kTileM)) return rc;
    if (int rc = make_map(&mA2, Ablk, rows, p->n, lda, 32, 32)) return rc;
    GemmArgs g{};
    g.rows = (int)rows;
    g.cols = (int)p->n;
    g.row_offset = (int)r0;
    g.yt = p->yt;
    g.yt_hi = p->yt_hi;
    g.yt_lo = p->yt_lo;
    g.ldy = p->ldy;
    g.shift = p->center ? p->shiftf : nullptr;
    g.gpart = p->gpart;
    g.err = p->err;
    if (with_g1) {
        const int grid = (int)((rows + kTileM - 1) / kTileM);
        pca_gemm_kernel<kModeAW><<<grid, kThreads, StageLayout<kModeAW>::smem, p->st>>>(mA1, p->mapWh,
                                                                                      p->mapWl, g);
        p->launches += 1;
        CU(cudaGetLastError(), "G1 launch");
    }
    // G2: column tiles x K splits (each split a whole number of 32-row stages)
    g.n_tiles = (int)((p->n + kTileM - 1) / kTileM);
    const int64_t stages = (rows + kStageK - 1) / kStageK;
    int nsplit = (int)std::min<int64_t>(p->nsplit_max, std::max<int64_t>(1, (4LL * p->sm_count + g.n_tiles - 1) / g.n_tiles));
    nsplit = (int)std::min<int64_t>(nsplit, stages);
    g.k_stages = (int)((stages + nsplit - 1) / nsplit);
    nsplit = (int)((stages + g.k_stages - 1) / g.k_stages);  // every split has at least one stage
    pca_gemm_kernel<kModeATY><<<g.n_tiles * nsplit, kThreads, StageLayout<kModeATY>::smem, p->st>>>(
        mA2, p->mapYh, p->mapYl, g);
    reduce_adjoint_kernel<<<grid_of(p->n * p->l, 256), 256, 0, p->st>>>(p->gpart, nsplit, p->n, p->l, nullptr,
                                                                       nullptr, accumulate ? 1 : 0, p->Gd, p->n);
    p->launches += 2;
    CU(cudaGetLastError(), "G2 launch");
    return TSNE_OK;
}

// One pass over A: Y = A W (unless !with_g1: Y^T hi / lo already hold the
// operand, e.g. Q) and Gd = A* Y. Host-resident A streams through the two
// block buffers on the copy stream.
int pass(tsne_oocpca* p, const float* A, int64_t lda, int on_host, bool with_g1) {
    const int64_t b = p->block_rows;
    int blk = 0;
    for (int64_t r0 = 0; r0 < p->m; r0 += b, ++blk) {
        const int64_t rows = std::min<int64_t>(b, p->m - r0);
        const float* Ablk = A + r0 * lda;
        if (on_host) {
            const int s = blk & 1;
            // the buffer is free once the products of two blocks ago are done
            CU(cudaStreamWaitEvent(p->copy_st, p->used[s], 0), "copy wait");
            CU(cudaMemcpyAsync(p->blk[s], Ablk, sizeof(float) * rows * lda, cudaMemcpyHostToDevice, p->copy_st),
               "block copy");
            CU(cudaEventRecord(p->copied[s], p->copy_st), "copy event");
            CU(cudaStreamWaitEvent(p->st, p->copied[s], 0), "compute wait");
            Ablk = p->blk[s];
        }
        if (int rc = block_products(p, Ablk, lda, r0, rows, with_g1, blk > 0)) return rc;
        if (on_host) CU(cudaEventRecord(p->used[blk & 1], p->st), "use event");
    }
    p->passes += 1;
    return TSNE_OK;
}

// Column sums of Yd (m x l) into colsum; then Gd -= mu colsum* (centring).
int center_adjoint(tsne_oocpca* p) {
    colsum_kernel<<<kSmallBlocks, 256, 0, p->st>>>(p->Yd, p->m, p->m, p->l, p->part, p->ticket, p->colsum);
    center_adjoint_kernel<<<grid_of(p->n * p->l, 256), 256, 0, p->st>>>(p->Gd, p->n, p->n, p->l, p->mu,
                                                                        p->colsum);
    p->launches += 2;
    CU(cudaGetLastError(), "centring launch");
    return TSNE_OK;
}

// W (column-major n x l) to the G1 operand (and, when centring, the shift).
int set_w(tsne_oocpca* p, const double* W) {
    split_operand_kernel<<<grid_of(kTileN * p->ldw, 256), 256, 0, p->st>>>(W, p->n, p->n, p->l, p->w_hi,
                                                                           p->w_lo, p->ldw);
    p->launches += 1;
    if (p->center) {
        CU(cudaMemsetAsync(p->shiftf, 0, sizeof(float) * kTileN, p->st), "shift reset");
        mean_shift_kernel<<<p->l, 256, 0, p->st>>>(p->mu, W, p->n, p->n, p->shiftf);
        p->launches += 1;
    }
    CU(cudaGetLastError(), "operand launch");
    return TSNE_OK;
}

}  // namespace

namespace {

struct PhaseTimer {
    cudaStream_t st;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> rec;
    int cur = -1;
    cudaEvent_t start = nullptr;
    explicit PhaseTimer(cudaStream_t s) : st(s) {}
    void begin(int phase) {
        cur = phase;
        cudaEventCreate(&start);
        cudaEventRecord(start, st);
    }
    void end() {
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, st);
        rec.push_back({cur, {start, e}});
    }
    void read(double* ms) {
        for (auto& r : rec) {
            float t = 0.0f;
            if (cudaEventElapsedTime(&t, r.second.first, r.second.second) == cudaSuccess) ms[r.first] += t;
        }
    }
    ~PhaseTimer() {
        for (auto& r : rec) {
            cudaEventDestroy(r.second.first);
            cudaEventDestroy(r.second.second);
        }
    }
};

// LU with partial pivoting of X (column-major R x l, FP64): X becomes L.
int lu(tsne_oocpca* p, double* X, int64_t R) {
    CU(cudaMemsetAsync(p->used_rows, 0, (size_t)R, p->st), "pivot flags reset");
    CU(cudaMemsetAsync(p->Um, 0, sizeof(double) * kTileN * kTileN, p->st), "U reset");
    const int g = (int)std::min<int64_t>(4 * kSmallBlocks, (R + 255) / 256);
    for (int j = 0; j < p->l; ++j) {
        lu_pivot_kernel<<<g, 256, 0, p->st>>>(X, R, p->l, j, p->used_rows, p->part_v, p->part_i, p->ticket,
                                             p->used_rows, p->piv, p->Um);
        lu_elim_kernel<<<g, 256, 0, p->st>>>(X, R, p->l, j, p->used_rows, p->Um);
        p->launches += 2;
    }
    lu_finalize_kernel<<<g, 256, 0, p->st>>>(X, R, p->l, p->used_rows);
    p->launches += 1;
    CU(cudaGetLastError(), "LU launch");
    return TSNE_OK;
}

// Shifted Cholesky QR, three rounds: Yd (m x l) becomes Q.
int cholesky_qr3(tsne_oocpca* p) {
    const double shift_scale = 11.0 * ((double)p->m * p->l + (double)p->l * (p->l + 1));
    for (int round = 0; round < 3; ++round) {
        gram_kernel<<<kSmallBlocks, 256, 0, p->st>>>(p->Yd, p->m, p->m, p->l, p->part, p->ticket, p->Cm);
        cholesky_kernel<<<1, 256, 0, p->st>>>(p->Cm, p->l, round == 0 ? shift_scale : 0.0, p->Rm);
        right_solve_kernel<<<grid_of(p->m, 256), 256, 0, p->st>>>(p->Yd, p->m, p->m, p->l, p->Rm, p->Yd);
        p->launches += 3;
    }
    CU(cudaGetLastError(), "QR launch");
    return TSNE_OK;
}

int widen(tsne_oocpca* p) {
    widen_kernel<<<grid_of(p->m * p->l, 256), 256, 0, p->st>>>(p->yt, p->ldy, p->m, p->l, p->Yd);
    p->launches += 1;
    CU(cudaGetLastError(), "widen launch");
    return TSNE_OK;
}

int column_means(tsne_oocpca* p, const float* A, int64_t lda, int on_host) {
    const int ny = 64;
    CU(cudaMemsetAsync(p->mu_part, 0, sizeof(double) * ny * p->n, p->st), "mean reset");
    const dim3 grid((unsigned)((p->n + 255) / 256), ny);
    int blk = 0;
    for (int64_t r0 = 0; r0 < p->m; r0 += p->block_rows, ++blk) {
        const int64_t rows = std::min<int64_t>(p->block_rows, p->m - r0);
        const float* Ablk = A + r0 * lda;
        if (on_host) {
            const int s = blk & 1;
            CU(cudaStreamWaitEvent(p->copy_st, p->used[s], 0), "copy wait");
            CU(cudaMemcpyAsync(p->blk[s], Ablk, sizeof(float) * rows * lda, cudaMemcpyHostToDevice, p->copy_st),
               "block copy");
            CU(cudaEventRecord(p->copied[s], p->copy_st), "copy event");
            CU(cudaStreamWaitEvent(p->st, p->copied[s], 0), "compute wait");
            Ablk = p->blk[s];
        }
        colsum_rows_kernel<<<grid, 256, 0, p->st>>>(Ablk, rows, p->n, lda, p->mu_part);
        p->launches += 1;
        if (on_host) CU(cudaEventRecord(p->used[blk & 1], p->st), "use event");
    }
    mean_finish_kernel<<<grid_of(p->n, 256), 256, 0, p->st>>>(p->mu_part, ny, p->n, p->m, p->mu);
    p->launches += 1;
    p->passes += 1;
    CU(cudaGetLastError(), "mean launch");
    return TSNE_OK;
}

}  // namespace

extern "C" {

int tsne_oocpca_create(int64_t m, int64_t n, int32_t k, int32_t l, const tsne_oocpca_opts* opts,
                       tsne_oocpca** out) {
    fitsne::clear_error();
    if (!out) return set_error(TSNE_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (m < 2 || n < 2 || m >= INT32_MAX || n >= INT32_MAX)
        return set_error(TSNE_ERR_INVALID_ARG, "m, n must be in [2, 2^31 - 1)");
    if (n % 4 != 0) return set_error(TSNE_ERR_INVALID_ARG, "n must be a multiple of 4 (got %lld)", (long long)n);
    if (k < 1 || l < k || l > kTileN || l >= std::min(m, n))
        return set_error(TSNE_ERR_INVALID_ARG, "need 1 <= k <= l <= 64 and l < min(m, n) (k %d, l %d)", k, l);
    tsne_oocpca_opts o{};
    if (opts) o = *opts;
    tsne_oocpca* p = new tsne_oocpca();
    memset(p, 0, sizeof(*p));
    p->m = m;
    p->n = n;
    p->k = k;
    p->l = l;
    p->its = o.its == 0 ? 2 : (o.its < 0 ? 0 : o.its);
    p->center = o.center ? 1 : 0;
    p->block_rows = o.block_rows;
    if (p->block_rows < 0) {
        free_plan(p);
        return set_error(TSNE_ERR_INVALID_ARG, "block_rows must be >= 0");
    }
    p->st = (cudaStream_t)o.stream;
    p->ldy = (m + 31) / 32 * 32;
    p->ldw = (n + 31) / 32 * 32;
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (ce != cudaSuccess) { free_plan(p); return cuda_fail(ce, "device query"); }
    // K splits of G2: enough CTAs for about four per SM over the column tiles
    const int64_t n_tiles = (n + kTileM - 1) / kTileM;
    p->nsplit_max = (int)std::max<int64_t>(1, (4LL * p->sm_count + n_tiles - 1) / n_tiles);
    int rc = TSNE_OK;
#define ALLOC(ptr, count) \
    if (rc == TSNE_OK) rc = dalloc(&p->ptr, (size_t)(count), #ptr)
    ALLOC(yt, kTileN * p->ldy);
    ALLOC(yt_hi, kTileN * p->ldy);
    ALLOC(yt_lo, kTileN * p->ldy);
    ALLOC(w_hi, kTileN * p->ldw);
    ALLOC(w_lo, kTileN * p->ldw);
    ALLOC(gpart, (int64_t)p->nsplit_max * n * kTileN);
    ALLOC(Gd, kTileN * n);
    ALLOC(Wd, kTileN * n);
    ALLOC(Yd, kTileN * m);
    ALLOC(Y0d, kTileN * m);
    ALLOC(G0d, kTileN * n);
    ALLOC(used_rows, std::max(m, n));
    ALLOC(piv, kTileN);
    ALLOC(Um, kTileN * kTileN);
    ALLOC(Cm, kTileN * kTileN);
    ALLOC(Rm, kTileN * kTileN);
    ALLOC(Vm, kTileN * kTileN);
    ALLOC(sig, kTileN);
    ALLOC(part, (int64_t)kSmallBlocks * kTileN * kTileN);
    ALLOC(part_v, 4 * kSmallBlocks);
    ALLOC(part_i, 4 * kSmallBlocks);
    ALLOC(mu, n);
    ALLOC(colsum, kTileN);
    ALLOC(mu_part, 64 * n);
    ALLOC(shiftf, kTileN);
    ALLOC(ticket, 1);
    ALLOC(err, 1);
#undef ALLOC
    if (rc != TSNE_OK) { free_plan(p); return rc; }
    ce = cudaMemsetAsync(p->yt, 0, sizeof(float) * kTileN * p->ldy, p->st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(p->ticket, 0, sizeof(unsigned), p->st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(p->Gd, 0, sizeof(double) * kTileN * n, p->st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(p->Wd, 0, sizeof(double) * kTileN * n, p->st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(p->Yd, 0, sizeof(double) * kTileN * m, p->st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(p->shiftf, 0, sizeof(float) * kTileN, p->st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(p->st);
    if (ce != cudaSuccess) { free_plan(p); return cuda_fail(ce, "plan initialisation"); }
    if ((rc = make_map(&p->mapYh, p->yt_hi, kTileN, p->ldy, p->ldy, 32, kTileN)) ||
        (rc = make_map(&p->mapYl, p->yt_lo, kTileN, p->ldy, p->ldy, 32, kTileN)) ||
        (rc = make_map(&p->mapWh, p->w_hi, kTileN, p->ldw, p->ldw, 32, kTileN)) ||
        (rc = make_map(&p->mapWl, p->w_lo, kTileN, p->ldw, p->ldw, 32, kTileN))) {
        free_plan(p);
        return rc;
    }
    ce = cudaFuncSetAttribute(pca_gemm_kernel<kModeAW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              StageLayout<kModeAW>::smem);
    if (ce == cudaSuccess)
        ce = cudaFuncSetAttribute(pca_gemm_kernel<kModeATY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  StageLayout<kModeATY>::smem);
    if (ce != cudaSuccess) { free_plan(p); return cuda_fail(ce, "shared memory limit"); }
    *out = p;
    return TSNE_OK;
}

int tsne_oocpca_destroy(tsne_oocpca* plan) {
    if (!plan) return TSNE_OK;
    cudaStreamSynchronize(plan->st);
    if (plan->copy_st) cudaStreamSynchronize(plan->copy_st);
    free_plan(plan);
    return TSNE_OK;
}

int tsne_oocpca_run(tsne_oocpca* p, const float* A, int64_t lda, int32_t a_on_host, const float* Omega,
                    float* U, double* sigma, float* V) {
    fitsne::clear_error();
    if (!p) return set_error(TSNE_ERR_INVALID_ARG, "plan is NULL");
    if (!A || !Omega || !U || !sigma || !V) return set_error(TSNE_ERR_INVALID_ARG, "NULL pointer");
    if (lda < p->n || lda % 4 != 0 || (reinterpret_cast<uintptr_t>(A) & 15) != 0)
        return set_error(TSNE_ERR_INVALID_ARG, "lda must be >= n and a multiple of 4, A 16-byte aligned");
    const int on_host = a_on_host ? 1 : 0;
    // block size: all rows for device A, else rows filling 1 GiB per buffer
    int64_t b = p->block_rows;
    if (b == 0) b = on_host ? ((int64_t)1 << 30) / (lda * 4) : p->m;
    // blocks start on multiples of 128 rows: every TMA coordinate along the
    // rows of Y (block start + stage offset) is then a multiple of 32
    if (b < p->m) b = std::max<int64_t>(kTileM, b / kTileM * kTileM);
    b = std::min<int64_t>(b, p->m);
    if (on_host) {
        if (!p->copy_st) {
            CU(cudaStreamCreateWithFlags(&p->copy_st, cudaStreamNonBlocking), "copy stream");
            for (int i = 0; i < 2; ++i) {
                CU(cudaEventCreateWithFlags(&p->copied[i], cudaEventDisableTiming), "event");
                CU(cudaEventCreateWithFlags(&p->used[i], cudaEventDisableTiming), "event");
            }
        }
        if (p->block_rows != b || !p->blk[0]) {
            for (int i = 0; i < 2; ++i) {
                if (p->blk[i]) cudaFree(p->blk[i]);
                p->blk[i] = nullptr;
            }
            for (int i = 0; i < 2; ++i)
                if (int rc = dalloc(&p->blk[i], (size_t)(b * lda), "block buffer")) return rc;
        }
    }
    p->block_rows = b;
    p->ran = 0;
    p->passes = 0;
    for (double& x : p->ms) x = 0.0;
    CU(cudaMemsetAsync(p->err, 0, sizeof(int), p->st), "error reset");
    PhaseTimer tm(p->st);
    if (p->center) {
        tm.begin(3);
        if (int rc = column_means(p, A, lda, on_host)) return rc;
        tm.end();
    }
    // W = Omega; pass 0: Y_0 = A Omega, G_0 = A* Y_0
    omega_kernel<<<grid_of(p->n * p->l, 256), 256, 0, p->st>>>(Omega, p->n, p->l, p->Wd, p->n);
    p->launches += 1;
    if (int rc = set_w(p, p->Wd)) return rc;
    tm.begin(0);
    if (int rc = pass(p, A, lda, on_host, true)) return rc;
    if (int rc = widen(p)) return rc;
    if (p->center)
        if (int rc = center_adjoint(p)) return rc;
    tm.end();
    CU(cudaMemcpyAsync(p->Y0d, p->Yd, sizeof(double) * p->l * p->m, cudaMemcpyDeviceToDevice, p->st), "copy");
    CU(cudaMemcpyAsync(p->G0d, p->Gd, sizeof(double) * p->l * p->n, cudaMemcpyDeviceToDevice, p->st), "copy");
    for (int i = 1; i <= p->its; ++i) {
        // W = L(G_{i-1}): the column space of A* L_{i-1} = G_{i-1} U_{i-1}^-1
        tm.begin(1);
        if (int rc = lu(p, p->Gd, p->n)) return rc;
        if (int rc = set_w(p, p->Gd)) return rc;
        tm.end();
        tm.begin(0);
        if (int rc = pass(p, A, lda, on_host, true)) return rc;  // Y_i = A W, G_i = A* Y_i
        if (int rc = widen(p)) return rc;
        if (p->center)
            if (int rc = center_adjoint(p)) return rc;
        tm.end();
    }
    // Q R = Y_its; Q* A by one more pass (as the G2 operand); SVD of Q* A
    tm.begin(2);
    if (int rc = cholesky_qr3(p)) return rc;
    split_operand_kernel<<<grid_of(kTileN * p->ldy, 256), 256, 0, p->st>>>(p->Yd, p->m, p->m, p->l, p->yt_hi,
                                                                           p->yt_lo, p->ldy);
    p->launches += 1;
    tm.end();
    tm.begin(0);
    if (int rc = pass(p, A, lda, on_host, false)) return rc;  // Gd = A* Q = (Q* A)*
    if (p->center)
        if (int rc = center_adjoint(p)) return rc;
    tm.end();
    tm.begin(2);
    gram_kernel<<<kSmallBlocks, 256, 0, p->st>>>(p->Gd, p->n, p->n, p->l, p->part, p->ticket, p->Cm);
    jacobi_svd_kernel<<<1, 256, 0, p->st>>>(p->Cm, p->l, p->Vm, p->sig);
    small_product_kernel<<<grid_of(p->m, 256), 256, 0, p->st>>>(p->Yd, p->m, p->m, p->l, p->k, p->Vm, nullptr, U);
    small_product_kernel<<<grid_of(p->n, 256), 256, 0, p->st>>>(p->Gd, p->n, p->n, p->l, p->k, p->Vm, p->sig, V);
    p->launches += 4;
    CU(cudaGetLastError(), "SVD launch");
    CU(cudaMemcpyAsync(sigma, p->sig, sizeof(double) * p->k, cudaMemcpyDeviceToDevice, p->st), "sigma copy");
    tm.end();
    int err = 0;
    CU(cudaMemcpyAsync(&err, p->err, sizeof(int), cudaMemcpyDeviceToHost, p->st), "error read-back");
    CU(cudaStreamSynchronize(p->st), "run synchronise");
    tm.read(p->ms);
    p->ran = 1;
    if (err) return set_error(TSNE_ERR_TIMEOUT, "a tensor-core pipeline wait gave up");
    return TSNE_OK;
}

int tsne_oocpca_debug_copy(tsne_oocpca* p, int32_t which, double* host_dst, size_t bytes) {
    if (!p || !host_dst) return set_error(TSNE_ERR_INVALID_ARG, "NULL pointer");
    if (!p->ran) return set_error(TSNE_ERR_INVALID_ARG, "no run yet");
    const double* src;
    int64_t R;
    if (which == 0) { src = p->Y0d; R = p->m; }
    else if (which == 1) { src = p->G0d; R = p->n; }
    else if (which == 2) { src = p->Yd; R = p->m; }
    else return set_error(TSNE_ERR_INVALID_ARG, "which must be 0, 1 or 2");
    const size_t need = sizeof(double) * (size_t)R * p->l;
    if (bytes < need) return set_error(TSNE_ERR_INVALID_ARG, "buffer too small (%zu bytes needed)", need);
    std::vector<double> cm((size_t)R * p->l);
    CU(cudaMemcpy(cm.data(), src, need, cudaMemcpyDeviceToHost), "debug copy");
    for (int64_t r = 0; r < R; ++r)
        for (int j = 0; j < p->l; ++j) host_dst[r * p->l + j] = cm[(size_t)j * R + r];
    return TSNE_OK;
}

int tsne_oocpca_phase_ms(const tsne_oocpca* p, double* ms_out, int32_t* passes_out) {
    if (!p || !ms_out) return set_error(TSNE_ERR_INVALID_ARG, "NULL pointer");
    for (int i = 0; i < 4; ++i) ms_out[i] = p->ms[i];
    if (passes_out) *passes_out = p->passes;
    return TSNE_OK;
}

int64_t tsne_oocpca_launch_count(const tsne_oocpca* p) { return p ? p->launches : 0; }

}  // extern "C"
