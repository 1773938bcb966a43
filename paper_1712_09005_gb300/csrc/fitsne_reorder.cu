// Locality relabelling of the points for the attraction gathers.
//
// The attraction reads y_j for every stored p_ij: ~150 random 8-byte reads
// per point per iteration, each one L1TEX request. Relabelling the points so
// that neighbours in P get nearby labels turns most of these reads into
// cache hits of the CTA's working set. Two sources of labels:
//   * the graph order (at the start of a run): P alone decides. Two
//     pseudo-random coordinates per point are averaged over the point's row
//     of P for a few rounds, z_i <- sum_j p_ij z_j / sum_j p_ij (a random
//     walk on the kNN graph, the power iteration that early exaggeration
//     also performs on the embedding): every component but the slow,
//     cluster-level ones dies out, so points of one cluster of the graph
//     collapse onto nearby values. The labels follow a Hilbert curve over
//     those values. This gives the gathers their locality from iteration 0,
//     before the embedding has formed any structure;
//   * the embedding order (during a run): neighbours in P are close in the
//     embedding once the clusters have formed, so the labels follow a
//     Hilbert curve over a 1024 x 1024 grid on the current box (1-D: 2^20
//     cells).
// Ties are broken by the original label: every permutation is deterministic.
// P is relabelled once per relabelling: row k of the new matrix is row
// perm[k] of the caller's P with its columns mapped through inv and its
// entries kept in their order. The gradient is equivariant under relabelling
// and each row's attraction sum keeps its order, so results do not change.
#include <algorithm>

#include "fitsne_internal.cuh"

namespace fitsne {

namespace {

// Position along a Hilbert curve of order 10 of the cell (x, y), x, y in
// [0, 1024): at each scale s the quadrant (rx, ry) adds s^2 times its rank in
// the curve's visiting order, and the coordinates are turned into the
// quadrant's own frame (a transpose, with a reflection in one quadrant), so
// that consecutive positions are always adjacent cells (a Z-order curve jumps
// across the grid at quadrant boundaries; Hilbert labels measured about 1 %
// faster per iteration at N = 1M).
__device__ __forceinline__ unsigned hilbert_index10(unsigned x, unsigned y) {
    unsigned d = 0;
    for (unsigned s = 512; s > 0; s >>= 1) {
        const unsigned rx = (x & s) ? 1u : 0u;
        const unsigned ry = (y & s) ? 1u : 0u;
        d += s * s * ((3u * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) {
                x = 1023u - x;
                y = 1023u - y;
            }
            const unsigned t = x;
            x = y;
            y = t;
        }
    }
    return d;
}

// (key << 32) | original label for the point at current position c.
template <int S>
__global__ void relabel_keys_kernel(const float* __restrict__ Y, const int32_t* __restrict__ perm_cur,
                                    int reordered, int64_t N, int64_t M,
                                    const Params* __restrict__ params,
                                    unsigned long long* __restrict__ keys) {
    const Params P = *params;
    const float inv_w = 1.0f / P.width;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < M;
         c += (int64_t)gridDim.x * blockDim.x) {
        if (c >= N) {
            keys[c] = ~0ull;
            continue;
        }
        unsigned key;
        if (S == 2) {
            const float2 y = reinterpret_cast<const float2*>(Y)[c];
            const int cx = min(1023, max(0, (int)((y.x - P.y_min) * inv_w * 1024.0f)));
            const int cy = min(1023, max(0, (int)((y.y - P.y_min) * inv_w * 1024.0f)));
            key = hilbert_index10((unsigned)cx, (unsigned)cy);
        } else {
            key = (unsigned)min(1048575, max(0, (int)((Y[c] - P.y_min) * inv_w * 1048576.0f)));
        }
        const unsigned orig = reordered ? (unsigned)perm_cur[c] : (unsigned)c;
        keys[c] = ((unsigned long long)key << 32) | orig;
    }
}

// One compare-exchange stage (k, j) of a bitonic sort of M = 2^m keys.
__global__ void bitonic_kernel(unsigned long long* __restrict__ a, int64_t M, int64_t k, int64_t j) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = i ^ j;
        if (l <= i) continue;
        const unsigned long long x = a[i], y = a[l];
        const bool up = (i & k) == 0;
        if ((x > y) == up) {
            a[i] = y;
            a[l] = x;
        }
    }
}

// perm[k] = original label at sorted position k (low half of the key).
__global__ void keys_to_perm_kernel(const unsigned long long* __restrict__ keys, int64_t N,
                                    int32_t* __restrict__ perm) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x)
        perm[k] = (int32_t)(keys[k] & 0xffffffffu);
}

// inv[perm[k]] = k; row lengths of the relabelled matrix; cur_of[k] =
// current position of that point (to move the run state).
__global__ void relabel_perm_kernel(const int32_t* __restrict__ perm,
                                    const int32_t* __restrict__ inv_cur, int reordered, int64_t N,
                                    const int32_t* __restrict__ row_ptr, int32_t* __restrict__ inv,
                                    int32_t* __restrict__ len, int32_t* __restrict__ cur_of) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = perm[k];
        inv[o] = (int32_t)k;
        len[k] = row_ptr[o + 1] - row_ptr[o];
        cur_of[k] = reordered ? inv_cur[o] : o;
    }
}

// Moves an N x s state array to the new labels: dst[k] = src[cur_of[k]].
template <int S>
__global__ void gather_rows_kernel(const float* __restrict__ src, const int32_t* __restrict__ idx,
                                   int64_t N, float* __restrict__ dst) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        if (S == 2)
            reinterpret_cast<float2*>(dst)[k] = reinterpret_cast<const float2*>(src)[idx[k]];
        else
            dst[k] = src[idx[k]];
    }
}

// dst[idx[k]] = src[k] (back to the caller's labels).
template <int S>
__global__ void scatter_rows_kernel(const float* __restrict__ src, const int32_t* __restrict__ idx,
                                    int64_t N, float* __restrict__ dst) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        if (S == 2)
            reinterpret_cast<float2*>(dst)[idx[k]] = reinterpret_cast<const float2*>(src)[k];
        else
            dst[idx[k]] = src[k];
    }
}

// Exclusive scan of len[0..N) into out[0..N], 2048 per block; block totals
// in bsum, turned into offsets by the last block (in order, any count).
__device__ __forceinline__ int scan_warp_incl(int x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

__device__ int block_scan_excl(int v, int* sw, int& total) {
    const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
    const int x = scan_warp_incl(v, lane);
    if (lane == 31) sw[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = lane < (int)(blockDim.x / 32) ? sw[lane] : 0;
        t = scan_warp_incl(t, lane);
        sw[lane] = t;
    }
    __syncthreads();
    total = sw[blockDim.x / 32 - 1];
    const int e = x - v + (wid ? sw[wid - 1] : 0);
    __syncthreads();
    return e;
}

__global__ void __launch_bounds__(1024)
scan_pass1_kernel(const int32_t* __restrict__ len, int64_t N, int32_t* __restrict__ out,
                  int32_t* __restrict__ bsum, unsigned* __restrict__ ticket) {
    __shared__ int sw[32];
    __shared__ bool s_last;
    const int64_t i0 = (int64_t)blockIdx.x * 2048 + threadIdx.x * 2;
    const int a = i0 < N ? len[i0] : 0, b = i0 + 1 < N ? len[i0 + 1] : 0;
    int tot;
    const int e = block_scan_excl(a + b, sw, tot);
    if (i0 < N) out[i0] = e;
    if (i0 + 1 < N) out[i0 + 1] = e + a;
    if (threadIdx.x == 0) {
        bsum[blockIdx.x] = tot;
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    int carry = 0;
    for (unsigned s = 0; s < gridDim.x; s += blockDim.x) {
        const unsigned i = s + threadIdx.x;
        const int v = i < gridDim.x ? __ldcg(&bsum[i]) : 0;
        int t;
        const int ex = block_scan_excl(v, sw, t);
        if (i < gridDim.x) bsum[i] = carry + ex;
        carry += t;
    }
    if (threadIdx.x == 0) {
        out[N] = carry;
        *ticket = 0u;
    }
}

__global__ void scan_pass2_kernel(int32_t* __restrict__ out, int64_t N,
                                  const int32_t* __restrict__ bsum) {
    const int64_t i = (int64_t)blockIdx.x * 2048 + threadIdx.x * 2;
    const int add = bsum[blockIdx.x];
    if (i < N) out[i] += add;
    if (i + 1 < N) out[i + 1] += add;
}

// Relabelled rows: warp per new row k copies row perm[k] of P, columns mapped
// through inv.
__global__ void __launch_bounds__(256)
relabel_csr_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                   const float* __restrict__ val, const int32_t* __restrict__ perm,
                   const int32_t* __restrict__ inv, const int32_t* __restrict__ rp2, int64_t N,
                   int32_t* __restrict__ col2, float* __restrict__ val2) {
    const int lane = threadIdx.x % 32;
    const int64_t nwarp = (int64_t)gridDim.x * blockDim.x / 32;
    for (int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; k < N; k += nwarp) {
        const int o = perm[k];
        const int s0 = row_ptr[o], s1 = row_ptr[o + 1], d0 = rp2[k];
        for (int t = lane; t < s1 - s0; t += 32) {
            col2[d0 + t] = inv[col[s0 + t]];
            val2[d0 + t] = val[s0 + t];
        }
    }
}

// ---------------------------------------------------------------------------
// Graph order from P alone.
// ---------------------------------------------------------------------------

// SplitMix64 output function (Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014): a counter-based source of
// the starting coordinates.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

// z_i: two uniforms in [-1, 1) drawn from the label (24 bits each); a row
// without entries starts (and stays) at 0.
__global__ void order_init_kernel(const int32_t* __restrict__ row_ptr, int64_t N,
                                  float2* __restrict__ Z) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long h = splitmix64((unsigned long long)i);
        float a = (float)(unsigned)(h >> 40) * (1.0f / 8388608.0f) - 1.0f;
        float b = (float)(unsigned)((h >> 8) & 0xffffffu) * (1.0f / 8388608.0f) - 1.0f;
        if (row_ptr[i + 1] == row_ptr[i]) a = b = 0.0f;
        Z[i] = make_float2(a, b);
    }
}

// One averaging round, a warp per row: Zout_i = sum_j p_ij Zin_j / sum_j p_ij
// (Zin_i where the row is empty or sums to 0). Lane l takes entries l, l + 32,
// ... and the lanes' sums meet in an xor tree: the result does not depend on
// the launch, so the order is deterministic.
__global__ void __launch_bounds__(256)
order_smooth_kernel(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                    const float* __restrict__ val, int64_t N, const float2* __restrict__ Zin,
                    float2* __restrict__ Zout) {
    const int lane = threadIdx.x % 32;
    const int64_t nwarp = (int64_t)gridDim.x * blockDim.x / 32;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; i < N; i += nwarp) {
        const int beg = row_ptr[i], end = row_ptr[i + 1];
        float ax = 0.0f, ay = 0.0f, w = 0.0f;
        for (int e = beg + lane; e < end; e += 32) {
            const float v = __ldg(val + e);
            const float2 z = __ldg(Zin + __ldg(col + e));
            ax += v * z.x;
            ay += v * z.y;
            w += v;
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            ax += __shfl_xor_sync(0xffffffffu, ax, o);
            ay += __shfl_xor_sync(0xffffffffu, ay, o);
            w += __shfl_xor_sync(0xffffffffu, w, o);
        }
        if (lane == 0) Zout[i] = (w > 0.0f) ? make_float2(ax / w, ay / w) : Zin[i];
    }
}

constexpr int kOrderStatBlocks = 256;

// Mean and standard deviation of each coordinate of Z (FP64 sums in a fixed
// order: per block, then by the last block), turned into the key window
// window = (lo_x, lo_y, sc_x, sc_y): cell = (z - lo) sc over mean +- 3 sd.
__global__ void __launch_bounds__(256)
order_stats_kernel(const float2* __restrict__ Z, int64_t N, double* __restrict__ partial,
                   unsigned* __restrict__ ticket, float* __restrict__ window) {
    __shared__ double s_v[4][8];
    __shared__ bool s_last;
    const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 z = Z[i];
        a[0] += z.x;
        a[1] += z.y;
        a[2] += (double)z.x * z.x;
        a[3] += (double)z.y * z.y;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) a[k] += __shfl_xor_sync(0xffffffffu, a[k], o);
        if (lane == 0) s_v[k][wid] = a[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < 4; ++k) {
            double t = 0.0;
            for (int q = 0; q < (int)(blockDim.x / 32); ++q) t += s_v[k][q];
            partial[4 * blockIdx.x + k] = t;
        }
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    for (unsigned b = 0; b < gridDim.x; ++b)
        for (int k = 0; k < 4; ++k) t[k] += __ldcg(&partial[4 * b + k]);
    *ticket = 0u;
    const double n = (double)(N > 0 ? N : 1);
    for (int d = 0; d < 2; ++d) {
        const double mean = t[d] / n;
        const double var = fmax(t[2 + d] / n - mean * mean, 0.0);
        const double sd = sqrt(var);
        const bool ok = sd > 0.0 && isfinite(sd);
        window[d] = ok ? (float)(mean - 3.0 * sd) : 0.0f;
        window[2 + d] = ok ? (float)(1024.0 / (6.0 * sd)) : 0.0f;
    }
}

// (Hilbert position of z_c's cell << 32) | c; keys past N sort last.
__global__ void order_keys_kernel(const float2* __restrict__ Z, int64_t N, int64_t M,
                                  const float* __restrict__ window,
                                  unsigned long long* __restrict__ keys) {
    const float lx = window[0], ly = window[1], sx = window[2], sy = window[3];
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < M;
         c += (int64_t)gridDim.x * blockDim.x) {
        if (c >= N) {
            keys[c] = ~0ull;
            continue;
        }
        const float2 z = Z[c];
        // fmaxf first: a NaN coordinate lands in cell 0
        const float fx = fminf(fmaxf((z.x - lx) * sx, 0.0f), 1023.0f);
        const float fy = fminf(fmaxf((z.y - ly) * sy, 0.0f), 1023.0f);
        const unsigned key = hilbert_index10((unsigned)fx, (unsigned)fy);
        keys[c] = ((unsigned long long)key << 32) | (unsigned long long)c;
    }
}

// inv[perm[k]] = k.
__global__ void invert_perm_kernel(const int32_t* __restrict__ perm, int64_t N,
                                   int32_t* __restrict__ inv) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x)
        inv[perm[k]] = (int32_t)k;
}

// len[k] = length of row perm[k] of P.
__global__ void perm_row_len_kernel(const int32_t* __restrict__ perm, int64_t N,
                                    const int32_t* __restrict__ row_ptr, int32_t* __restrict__ len) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = perm[k];
        len[k] = row_ptr[o + 1] - row_ptr[o];
    }
}

int grid_for_n(const tsne_plan* pl, int64_t n, int per_block) {
    int64_t b = (n + per_block - 1) / per_block;
    const int64_t cap = 8LL * pl->sm_count;
    return (int)std::max<int64_t>(1, std::min(b, cap));
}

}  // namespace

namespace {

// Sorts the M keys in pl->sort_keys (bitonic) and writes their low halves,
// the labels in key order, to perm_out[0..N).
void sort_keys_to_perm(tsne_plan* pl, int64_t M, int32_t* perm_out) {
    cudaStream_t st = pl->stream;
    const int g = grid_for_n(pl, M, 256);
    for (int64_t k = 2; k <= M; k <<= 1)
        for (int64_t j = k >> 1; j > 0; j >>= 1) {
            bitonic_kernel<<<g, 256, 0, st>>>(pl->sort_keys, M, k, j);
            pl->launches += 1;
        }
    keys_to_perm_kernel<<<grid_for_n(pl, pl->N, 256), 256, 0, st>>>(pl->sort_keys, pl->N, perm_out);
    pl->launches += 1;
}

int64_t pow2_at_least(int64_t n) {
    int64_t M = 1;
    while (M < n) M <<= 1;
    return M;
}

// rp2/col2/val2 = P with row k taken from row perm[k] and columns mapped
// through inv (entry order kept).
void relabel_csr(tsne_plan* pl, const tsne_csr& P, const int32_t* perm, const int32_t* inv) {
    cudaStream_t st = pl->stream;
    const int64_t N = pl->N;
    perm_row_len_kernel<<<grid_for_n(pl, N, 256), 256, 0, st>>>(perm, N, P.row_ptr, pl->row_len);
    const int nb = (int)((N + 2047) / 2048);
    scan_pass1_kernel<<<nb, 1024, 0, st>>>(pl->row_len, N, pl->rp2, pl->scan_bsum, pl->relabel_ticket);
    scan_pass2_kernel<<<nb, 1024, 0, st>>>(pl->rp2, N, pl->scan_bsum);
    relabel_csr_kernel<<<grid_for_n(pl, N * 32, 256), 256, 0, st>>>(
        P.row_ptr, P.col, P.val, perm, inv, pl->rp2, N, pl->col2, pl->val2);
    pl->launches += 4;
}

// Moves the run to the labels in pl->perm_next (new label -> caller's
// label): perm/inv become the new order, Y_cur (current labels) is gathered
// into Y_out, uY and gains are moved in place; with copy_P the relabelled P
// is rebuilt.
void apply_perm_next(tsne_plan* pl, const tsne_csr& P, int copy_P, const float* Y_cur,
                     float* uY_cur, float* gains_cur, float* Y_out) {
    cudaStream_t st = pl->stream;
    const int64_t N = pl->N;
    const int gn = grid_for_n(pl, N, 256);
    // the new inverse; cur_of from the current inverse (read before the swap)
    relabel_perm_kernel<<<gn, 256, 0, st>>>(pl->perm_next, pl->inv, pl->reordered, N, P.row_ptr,
                                            pl->inv_next, pl->row_len, pl->cur_of);
    pl->launches += 1;
    std::swap(pl->perm, pl->perm_next);
    std::swap(pl->inv, pl->inv_next);
    if (copy_P) relabel_csr(pl, P, pl->perm, pl->inv);
    const int64_t ns = N * pl->s;
    if (pl->s == 2) {
        gather_rows_kernel<2><<<gn, 256, 0, st>>>(Y_cur, pl->cur_of, N, Y_out);
        gather_rows_kernel<2><<<gn, 256, 0, st>>>(uY_cur, pl->cur_of, N, pl->tmp_state);
        cudaMemcpyAsync(uY_cur, pl->tmp_state, sizeof(float) * ns, cudaMemcpyDeviceToDevice, st);
        gather_rows_kernel<2><<<gn, 256, 0, st>>>(gains_cur, pl->cur_of, N, pl->tmp_state);
        cudaMemcpyAsync(gains_cur, pl->tmp_state, sizeof(float) * ns, cudaMemcpyDeviceToDevice, st);
    } else {
        gather_rows_kernel<1><<<gn, 256, 0, st>>>(Y_cur, pl->cur_of, N, Y_out);
        gather_rows_kernel<1><<<gn, 256, 0, st>>>(uY_cur, pl->cur_of, N, pl->tmp_state);
        cudaMemcpyAsync(uY_cur, pl->tmp_state, sizeof(float) * ns, cudaMemcpyDeviceToDevice, st);
        gather_rows_kernel<1><<<gn, 256, 0, st>>>(gains_cur, pl->cur_of, N, pl->tmp_state);
        cudaMemcpyAsync(gains_cur, pl->tmp_state, sizeof(float) * ns, cudaMemcpyDeviceToDevice, st);
    }
    pl->launches += 3;
    pl->reordered = 1;
}

}  // namespace

cudaError_t launch_relabel(tsne_plan* pl, const tsne_csr& P, const float* Y_cur, float* uY_cur,
                           float* gains_cur, float* Y_out) {
    cudaStream_t st = pl->stream;
    const int64_t N = pl->N;
    const int64_t M = pow2_at_least(N);
    const int g = grid_for_n(pl, M, 256);
    if (pl->s == 2)
        relabel_keys_kernel<2><<<g, 256, 0, st>>>(Y_cur, pl->perm, pl->reordered, N, M, pl->host_job.params, pl->sort_keys);
    else
        relabel_keys_kernel<1><<<g, 256, 0, st>>>(Y_cur, pl->perm, pl->reordered, N, M, pl->host_job.params, pl->sort_keys);
    pl->launches += 1;
    sort_keys_to_perm(pl, M, pl->perm_next);
    apply_perm_next(pl, P, 1, Y_cur, uY_cur, gains_cur, Y_out);
    return cudaGetLastError();
}

cudaError_t launch_graph_order(tsne_plan* pl, const tsne_csr& P, int rounds, int32_t* perm_out,
                               int32_t* inv_out) {
    cudaStream_t st = pl->stream;
    const int64_t N = pl->N;
    const int64_t M = pow2_at_least(N);
    float2* Z[2] = {reinterpret_cast<float2*>(pl->order_z), reinterpret_cast<float2*>(pl->order_z) + N};
    const int gn = grid_for_n(pl, N, 256);
    order_init_kernel<<<gn, 256, 0, st>>>(P.row_ptr, N, Z[0]);
    pl->launches += 1;
    const int gw = grid_for_n(pl, N * 32, 256);
    for (int r = 0; r < rounds; ++r) {
        order_smooth_kernel<<<gw, 256, 0, st>>>(P.row_ptr, P.col, P.val, N, Z[r & 1], Z[(r + 1) & 1]);
        pl->launches += 1;
    }
    const float2* Zf = Z[rounds & 1];
    order_stats_kernel<<<kOrderStatBlocks, 256, 0, st>>>(Zf, N, pl->order_stats, pl->relabel_ticket,
                                                         reinterpret_cast<float*>(pl->order_stats + 4 * kOrderStatBlocks));
    order_keys_kernel<<<grid_for_n(pl, M, 256), 256, 0, st>>>(
        Zf, N, M, reinterpret_cast<const float*>(pl->order_stats + 4 * kOrderStatBlocks), pl->sort_keys);
    pl->launches += 2;
    sort_keys_to_perm(pl, M, perm_out);
    invert_perm_kernel<<<gn, 256, 0, st>>>(perm_out, N, inv_out);
    pl->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_order_copy(tsne_plan* pl, const tsne_csr& P, const int32_t* perm,
                              const int32_t* inv) {
    relabel_csr(pl, P, perm, inv);
    return cudaGetLastError();
}

cudaError_t launch_apply_order(tsne_plan* pl, const tsne_csr& P, const int32_t* perm, int copy_P,
                               const float* Y_cur, float* uY_cur, float* gains_cur, float* Y_out) {
    cudaError_t e = cudaMemcpyAsync(pl->perm_next, perm, sizeof(int32_t) * pl->N,
                                    cudaMemcpyDeviceToDevice, pl->stream);
    if (e != cudaSuccess) return e;
    apply_perm_next(pl, P, copy_P, Y_cur, uY_cur, gains_cur, Y_out);
    return cudaGetLastError();
}

cudaError_t launch_to_labels(tsne_plan* pl, const float* src, int to_caller, float* dst) {
    const int gn = grid_for_n(pl, pl->N, 256);
    if (to_caller) {
        if (pl->s == 2) scatter_rows_kernel<2><<<gn, 256, 0, pl->stream>>>(src, pl->perm, pl->N, dst);
        else scatter_rows_kernel<1><<<gn, 256, 0, pl->stream>>>(src, pl->perm, pl->N, dst);
    } else {
        if (pl->s == 2) gather_rows_kernel<2><<<gn, 256, 0, pl->stream>>>(src, pl->perm, pl->N, dst);
        else gather_rows_kernel<1><<<gn, 256, 0, pl->stream>>>(src, pl->perm, pl->N, dst);
    }
    pl->launches += 1;
    return cudaGetLastError();
}

}  // namespace fitsne
