// Locality relabelling of the points for the attraction gathers.
//
// The attraction reads y_j for every stored p_ij: ~150 random 8-byte reads
// per point per iteration, each one L1TEX request. Relabelling the points so
// that neighbours in P get nearby labels turns most of these reads into
// cache hits of the CTA's working set. Neighbours in P are
// close in the embedding once the clusters have formed, so the new labels
// follow a Hilbert curve over a 1024 x 1024 grid on the current
// box (1-D: 2^20 cells), ties broken by the original label: a deterministic
// permutation. P is relabelled once per relabelling: row k of the new matrix
// is row perm[k] of the caller's P with its columns mapped through inv.
// The gradient is equivariant under relabelling; only the order of the
// attraction sum inside a row changes.
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

// perm[k] = original label at sorted position k; inv[perm[k]] = k; row
// lengths of the relabelled matrix; cur_of[k] = current position of that
// point (to move the run state).
__global__ void relabel_perm_kernel(const unsigned long long* __restrict__ keys,
                                    const int32_t* __restrict__ inv_cur, int reordered, int64_t N,
                                    const int32_t* __restrict__ row_ptr, int32_t* __restrict__ perm,
                                    int32_t* __restrict__ inv, int32_t* __restrict__ len,
                                    int32_t* __restrict__ cur_of) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = (int32_t)(keys[k] & 0xffffffffu);
        perm[k] = o;
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

int grid_for_n(const tsne_plan* pl, int64_t n, int per_block) {
    int64_t b = (n + per_block - 1) / per_block;
    const int64_t cap = 8LL * pl->sm_count;
    return (int)std::max<int64_t>(1, std::min(b, cap));
}

}  // namespace

cudaError_t launch_relabel(tsne_plan* pl, const tsne_csr& P, const float* Y_cur, float* uY_cur,
                           float* gains_cur, float* Y_out) {
    cudaStream_t st = pl->stream;
    const int64_t N = pl->N;
    int64_t M = 1;
    while (M < N) M <<= 1;
    const int g = grid_for_n(pl, M, 256);
    if (pl->s == 2)
        relabel_keys_kernel<2><<<g, 256, 0, st>>>(Y_cur, pl->perm, pl->reordered, N, M, pl->host_job.params, pl->sort_keys);
    else
        relabel_keys_kernel<1><<<g, 256, 0, st>>>(Y_cur, pl->perm, pl->reordered, N, M, pl->host_job.params, pl->sort_keys);
    pl->launches += 1;
    for (int64_t k = 2; k <= M; k <<= 1)
        for (int64_t j = k >> 1; j > 0; j >>= 1) {
            bitonic_kernel<<<g, 256, 0, st>>>(pl->sort_keys, M, k, j);
            pl->launches += 1;
        }
    // the new labels; perm/inv are overwritten, so the current ones are read first
    const int gn = grid_for_n(pl, N, 256);
    relabel_perm_kernel<<<gn, 256, 0, st>>>(pl->sort_keys, pl->inv, pl->reordered, N, P.row_ptr,
                                            pl->perm_next, pl->inv_next, pl->row_len, pl->cur_of);
    pl->launches += 1;
    std::swap(pl->perm, pl->perm_next);
    std::swap(pl->inv, pl->inv_next);
    // relabelled P
    const int nb = (int)((N + 2047) / 2048);
    scan_pass1_kernel<<<nb, 1024, 0, st>>>(pl->row_len, N, pl->rp2, pl->scan_bsum, pl->relabel_ticket);
    scan_pass2_kernel<<<nb, 1024, 0, st>>>(pl->rp2, N, pl->scan_bsum);
    relabel_csr_kernel<<<grid_for_n(pl, N * 32, 256), 256, 0, st>>>(
        P.row_ptr, P.col, P.val, pl->perm, pl->inv, pl->rp2, N, pl->col2, pl->val2);
    pl->launches += 3;
    // run state to the new labels
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
