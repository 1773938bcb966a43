/*
 * oocpca_gb300.h - C ABI of the out-of-core randomized PCA of Linderman et
 * al., "Efficient Algorithms for t-distributed Stochastic Neighborhood
 * Embedding" (arXiv 1712.09005), Sec. 6, Algorithm oocPCA, on one GB300
 * (sm_103a). Part of libfitsne_gb300.so.
 *
 * Given A (m x n) and k <= l < min(m, n), the algorithm returns U (m x k,
 * orthonormal columns), sigma (k, non-negative, decreasing) and V (n x k,
 * orthonormal columns) with A ~ U diag(sigma) V*:
 *   Omega (n x l) random; Y_0 = A Omega; L_0 U_0 = Y_0 (LU, partial pivoting);
 *   for i = 1 .. its: Y_i = A A* L_{i-1}; L_i U_i = Y_i if i < its;
 *   Q R = Y_its; U' Sigma V* = Q* A (small SVD); U = Q U'.
 * A is read block by block ("b rows at a time"), from device memory or, out
 * of core, from host memory, and each power iteration reads it once: the
 * pass that forms Y_i = A W also accumulates G_i = A* Y_i, and the next W
 * is the L factor of the LU factorization (partial pivoting) of G_i, which
 * spans the column space of A* L_i = G_i U_i^-1 (the renormalization moves
 * from Y_i to G_i: the same subspace, bounded entries when Y_i is
 * rank-deficient). The final Q* A takes one more pass, so a run reads A
 * its + 2 times.
 *
 * Precision: A, Omega, U and V are FP32. The products with A run on the
 * tensor cores (tcgen05, TF32 inputs split into head and tail, three MMAs
 * per step, FP32 accumulation): FP32-level products (relative error about
 * 1e-6). The renormalizations, the QR (shifted Cholesky QR, three rounds)
 * and the small SVD (Jacobi on the l x l Gram matrix of Q* A) are FP64; sigma
 * is returned in FP64.
 *
 * Conventions: pointers are DEVICE pointers owned by the caller unless a
 * comment says HOST; calls enqueue their work on the plan's stream and
 * tsne_oocpca_run synchronises it before returning. Return values are
 * TSNE_OK (0) or a negative TSNE_ERR_* code of fitsne_gb300.h;
 * tsne_last_error_string() describes the last failure of the calling thread.
 */
#ifndef OOCPCA_GB300_H
#define OOCPCA_GB300_H

#include <stdint.h>

#include "fitsne_gb300.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tsne_oocpca tsne_oocpca;

/* Options; zero-initialised fields take the defaults in brackets. */
typedef struct {
    int32_t its;        /* power iterations [2]; < 0: none */
    int32_t center;     /* 1: decompose the column-centred matrix A - 1 mu* (mu = column
                           means, one extra pass over A; the centring is applied to the
                           products, A itself is not modified) [0] */
    int64_t block_rows; /* b, rows of A per block, rounded down to a multiple of 128 (at
                           least 128) [all rows when A is on the device; rows filling
                           1 GiB per block buffer when A is in host memory] */
    void* stream;       /* cudaStream_t for all work; NULL = the legacy default stream */
} tsne_oocpca_opts;

/*
 * Plan for A of m x n (2 <= m, n < 2^31, n a multiple of 4), k components
 * and l = k + (oversampling) random vectors, 1 <= k <= l <= 64,
 * l < min(m, n) (the paper's default is l = k + 2). Allocates the device
 * workspace (about 12 m l + 40 n l bytes plus, for host-resident A, two
 * block buffers). INVALID_ARG on bad sizes, OOM.
 */
int tsne_oocpca_create(int64_t m, int64_t n, int32_t k, int32_t l, const tsne_oocpca_opts* opts,
                       tsne_oocpca** out);
int tsne_oocpca_destroy(tsne_oocpca* plan);

/*
 * One decomposition. A: m x n FP32 row-major with leading dimension lda
 * (elements, >= n, a multiple of 4, 16-byte aligned base); a_on_host = 1
 * when A is HOST memory (pinned memory lets the block copies overlap the
 * products), 0 for device memory. Omega: n x l FP32 row-major, device (the
 * random matrix of the algorithm; the caller draws it, e.g. uniform on
 * [-1, 1)). Outputs (device): U m x k FP32 row-major, sigma k FP64
 * (decreasing), V n x k FP32 row-major; the sign of each pair (U_j, V_j) is
 * chosen so that the largest entry of the j-th singular vector of the small
 * matrix Q* A is positive. Synchronises the stream. INVALID_ARG on bad
 * pointers or lda, TIMEOUT if a pipeline wait of the tensor-core kernels
 * gave up (the outputs are then invalid), CUDA on a runtime failure.
 */
int tsne_oocpca_run(tsne_oocpca* plan, const float* A, int64_t lda, int32_t a_on_host,
                    const float* Omega, float* U, double* sigma, float* V);

/*
 * Test hook: copies an intermediate of the last run to HOST memory (FP64):
 *   0  Y of the first pass (= A Omega, centred if requested), m x l row-major
 *   1  G of the first pass (= A* Y_0), n x l row-major
 *   2  Q of the final QR, m x l row-major
 * bytes must be at least the size; INVALID_ARG otherwise or before a run.
 */
int tsne_oocpca_debug_copy(tsne_oocpca* plan, int32_t which, double* host_dst, size_t bytes);

/* Device time (CUDA events) of the last run's phases: ms_out[0] passes over
 * A (tensor-core products and block copies), [1] renormalizations, [2] QR
 * and small SVD, [3] column means (centring). Also the number of passes over
 * A in *passes_out (may be NULL). */
int tsne_oocpca_phase_ms(const tsne_oocpca* plan, double* ms_out, int32_t* passes_out);

/* Kernels the plan has launched (host-side count). */
int64_t tsne_oocpca_launch_count(const tsne_oocpca* plan);

#ifdef __cplusplus
}
#endif

#endif /* OOCPCA_GB300_H */
