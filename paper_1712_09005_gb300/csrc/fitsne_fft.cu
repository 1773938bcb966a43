// Step 2 of the interpolation scheme: the Toeplitz (2-D: block-Toeplitz)
// product v = K~ w on the equispaced nodes (Sec. 2.2, Eq. equikereval2;
// Sec. 2.4), done as a circular convolution on an L^s torus, L >= 2n, with a
// hand-written shared-memory FFT (mixed-radix 2/3/4/5 Stockham, FP32,
// twiddles rounded from FP64).
//
// Inputs (node units, offsets o in units of delta): the charge grid w0 and
// the dipole grids d_m = sum L_g(y)(t_m - j_m - 1/2) from the spread. The
// Appendix needs h1 = K1 * w0, v_{m+1} = K2 * w_{y(m)} and v_{s+2} = K2 * w0;
// with w_{y(m)} = delta d_m + y~(m) w0 the combination the gradient uses,
//   u_m[g] = v_{m+1}[g] - y~_g(m) v_{s+2}[g] = delta (K2 * d_m - G_m * w0)[g],
// G_m(o) = o_m K2(o), follows by expanding y~_g'(m) = y~_g(m) - delta (g - g')_m
// (exact). The transforms therefore produce, per node,
//   (h1, u'_1, u'_2, v_{s+2}) = (K1 * w0, K2 * d_1 - G_1 * w0, K2 * d_2 - G_2 * w0, K2 * w0)
// with u_m = delta u'_m; no output is a small difference of large values.
// h1 is not formed: Z + N = sum_g w0[g] (K1 * w0)[g] = L^-s sum_k |W0^(k)|^2 K1^(k)
// (Parseval; K1^ is real), summed in FP64 from the forward spectra.
//
// Real signals are packed in pairs into complex transforms:
//   C0 = w0 + i d_1, C1 = d_2 (+ i 0), CK = K1 + i K2, CG = G_1 + i G_2.
// K1, K2 are even in every offset (real, even spectra: Re / Im of one
// transform); G_m is odd in offset m and even in the other (imaginary
// spectrum i S_m), so the spectrum of CG is i S_1 - S_2. Outputs are packed
// the same way: D0 = U1 + i U2 -> (u'_1, u'_2), D1 = V -> v.
//
// 2-D passes (one CTA per work item; the items of every job of the table are
// shared out over a grid-stride loop):
//   rows_fwd_kernel  FFT along dimension 2 of the n rows of C0, C1, and of
//                    the rows o1 = 0..n-1 of CK and CG (the rows o1 < 0
//                    follow by symmetry)
//   cols_kernel      per column pair (k2, L-k2): FFT along dimension 1,
//                    split the packed spectra, the Parseval sums of Z,
//                    multiply, pack, inverse FFT
//   rows_inv_kernel  inverse FFT of the n needed rows, node values
// 1-D: conv1d_kernel does a job's whole convolution in one CTA.
#include <math.h>

#include <algorithm>

#include "fitsne_internal.cuh"

namespace fitsne {

namespace {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * (s i)
__device__ __forceinline__ float2 mul_si(float2 a, float s) { return make_float2(-s * a.y, s * a.x); }
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// R-point DFT in registers, X_k = sum_j x_j exp(s 2 pi i jk / R), s = -1 forward.
template <int R>
struct Dft;

template <>
struct Dft<2> {
    __device__ __forceinline__ static void run(float2 (&v)[2], float) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <>
struct Dft<3> {
    __device__ __forceinline__ static void run(float2 (&v)[3], float s) {
        const float h = 0.866025403784438647f;  // sqrt(3)/2
        float2 t = cadd(v[1], v[2]);
        float2 m = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
        float2 d = mul_si(csub(v[1], v[2]), s * h);
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, d);
        v[2] = csub(m, d);
    }
};

template <>
struct Dft<4> {
    __device__ __forceinline__ static void run(float2 (&v)[4], float s) {
        float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        float2 t2 = cadd(v[1], v[3]), t3 = mul_si(csub(v[1], v[3]), s);
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    }
};

template <>
struct Dft<5> {
    __device__ __forceinline__ static void run(float2 (&v)[5], float s) {
        const float c1 = 0.309016994374947424f;   // cos(2 pi / 5)
        const float c2 = -0.809016994374947424f;  // cos(4 pi / 5)
        const float s1 = 0.951056516295153572f;   // sin(2 pi / 5)
        const float s2 = 0.587785252292473129f;   // sin(4 pi / 5)
        float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
        float2 t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
        float2 a1 = make_float2(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
        float2 a2 = make_float2(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
        float2 b1 = mul_si(make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y), s);
        float2 b2 = mul_si(make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y), s);
        v[0] = cadd(v[0], cadd(t1, t2));
        v[1] = cadd(a1, b1);
        v[4] = csub(a1, b1);
        v[2] = cadd(a2, b2);
        v[3] = csub(a2, b2);
    }
};

// One Stockham stage of radix R for B transforms of length L stored
// contiguously (x + b L -> y + b L); Ns = product of the earlier radices.
template <int R>
__device__ __forceinline__ void stage(const float2* __restrict__ x, float2* __restrict__ y, int L,
                                      int Ns, int B, const float2* __restrict__ tw, float s) {
    const int M = L / R;
    const int stride = L / (Ns * R);
    const int total = B * M;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int bi = t / M;
        const int j = t - bi * M;
        const float2* xb = x + bi * L;
        float2* yb = y + bi * L;
        const int k = j % Ns;
        float2 v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = xb[j + q * M];
        if (Ns > 1) {
#pragma unroll
            for (int q = 1; q < R; ++q) {
                float2 w = __ldg(&tw[q * k * stride]);
                if (s > 0.0f) w.y = -w.y;
                v[q] = cmul(v[q], w);
            }
        }
        Dft<R>::run(v, s);
        const int out = (j - k) * R + k;
#pragma unroll
        for (int q = 0; q < R; ++q) yb[out + q * Ns] = v[q];
    }
}

// B in-shared-memory FFTs of length e.L, ping-ponging between x and y.
// Callers synchronise before; returns the buffer holding the result.
__device__ float2* fft_batch(float2* x, float2* y, const FftEntry& e, int B,
                             const float2* __restrict__ tw, float s) {
    int Ns = 1;
    for (int st = 0; st < e.nst; ++st) {
        const int R = e.radix[st];
        switch (R) {
            case 2: stage<2>(x, y, e.L, Ns, B, tw, s); break;
            case 3: stage<3>(x, y, e.L, Ns, B, tw, s); break;
            case 4: stage<4>(x, y, e.L, Ns, B, tw, s); break;
            default: stage<5>(x, y, e.L, Ns, B, tw, s); break;
        }
        __syncthreads();
        float2* t = x;
        x = y;
        y = t;
        Ns *= R;
    }
    return x;
}

// Kernel pair (K1, K2) at squared node distance d2 (in units of delta^2).
__device__ __forceinline__ float2 kernel_pair(float delta2, int d2) {
    const float k1 = __frcp_rn(1.0f + delta2 * (float)d2);
    return make_float2(k1, k1 * k1);
}

// Fixed-point spread value to FP32.
__device__ __forceinline__ float fx(long long v, float inv) { return __ll2float_rn(v) * inv; }

// Signed node offset represented by circulant index i (|offset| < n), or -1
// for the gap that outputs in [0, n) never reach.
__device__ __forceinline__ int circ_offset(int i, int n, int L) {
    return i < n ? i : (i > L - n ? L - i : -1);
}

}  // namespace

namespace {

__device__ __forceinline__ int fft_rows_items(const Job& J) {
    const Params* P = J.params;
    return job_live(*P) ? 4 * P->n : 0;
}
__device__ __forceinline__ int fft_cols_items(const Job& J) {
    const Params* P = J.params;
    return job_live(*P) ? P->L / 2 + 1 : 0;
}
__device__ __forceinline__ int fft_inv_items(const Job& J) {
    const Params* P = J.params;
    return job_live(*P) ? P->n : 0;
}
__device__ __forceinline__ int fft_1d_items(const Job& J) {
    const Params* P = J.params;
    return job_live(*P) ? 1 : 0;
}

}  // namespace

// ----------------------------------------------------------------------------
// Rows per work item of a row pass: as many rows of length L as the launch's
// shared memory holds (per_row float2 each), but no more than keeps about
// 4 items per SM over the whole table.
// ----------------------------------------------------------------------------
__device__ __forceinline__ int rows_per_item(int L, int per_row, int smem_floats2, int total_rows,
                                             int sm_count) {
    int rp = smem_floats2 / (per_row * L);
    int want = total_rows / (4 * sm_count);
    if (want < 1) want = 1;
    if (rp > want) rp = want;
    if (rp > 16) rp = 16;
    return rp < 1 ? 1 : rp;
}

// ----------------------------------------------------------------------------
// 2-D, pass 1: row FFTs. Row m < 4n of a job: type m / n (0: C0, 1: C1,
// 2: CK, 3: CG), row r = m % n (for CK and CG the offset o1 = r >= 0). Output
// rows of length L, row-major, at spec + type n L. A work item takes rp
// consecutive rows (one batched FFT).
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
rows_fwd_kernel(const Job* __restrict__ jobs, int njobs, Tables tab, int smem_floats2,
                int sm_count) {
    extern __shared__ float2 sm[];
    __shared__ int32_t s_start[kMaxJobs + 1];
    __shared__ FftEntry e;
    const int total_rows = split_jobs(jobs, njobs, s_start, [](const Job& J) { return fft_rows_items(J); });
    const int total = split_jobs(jobs, njobs, s_start, [&](const Job& J) {
        const int rows = fft_rows_items(J);
        if (!rows) return 0;
        const int rp = rows_per_item(J.params->L, 2, smem_floats2, total_rows, sm_count);
        return (rows + rp - 1) / rp;
    });
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int j = job_of(s_start, njobs, item);
        const Job& J = jobs[j];
        const Params P = *J.params;
        if (threadIdx.x == 0) e = tab.fft[P.fft_idx];
        __syncthreads();
        const int n = P.n, L = P.L;
        const int rpj = rows_per_item(L, 2, smem_floats2, total_rows, sm_count);
        const int m0 = (item - s_start[j]) * rpj;
        const int rp = min(rpj, 4 * n - m0);
        const int64_t G = (int64_t)n * n;
        const long long* __restrict__ w = J.w;
        const float2* tw = tab.tw + e.tw_off;
        const float inv = P.fx_inv;
        float2* A = sm;
        float2* B = sm + rp * L;
        for (int idx = threadIdx.x; idx < rp * L; idx += blockDim.x) {
            const int q = idx / L, c = idx - q * L;
            const int m = m0 + q;
            const int type = m / n, r = m - type * n;
            float2 v = make_float2(0.0f, 0.0f);
            if (type == 0) {
                if (c < n) v = make_float2(fx(w[(int64_t)r * n + c], inv), fx(w[G + (int64_t)r * n + c], inv));
            } else if (type == 1) {
                if (c < n) v = make_float2(fx(w[2 * G + (int64_t)r * n + c], inv), 0.0f);
            } else {
                const int o = circ_offset(c, n, L);
                if (o >= 0) {
                    const float2 k = kernel_pair(P.delta2, r * r + o * o);
                    if (type == 2) {
                        v = k;
                    } else {
                        const int o2 = (c < n) ? c : c - L;  // signed offset
                        v = make_float2((float)r * k.y, (float)o2 * k.y);
                    }
                }
            }
            A[idx] = v;
        }
        __syncthreads();
        const float2* res = fft_batch(A, B, e, rp, tw, -1.0f);
        for (int idx = threadIdx.x; idx < rp * L; idx += blockDim.x) {
            const int q = idx / L, c = idx - q * L;
            const int m = m0 + q;
            const int type = m / n, r = m - type * n;
            J.spec[(int64_t)type * n * L + (int64_t)r * L + c] = res[idx];
        }
        __syncthreads();
    }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sum of one double per thread (blockDim.x <= 1024); result in thread 0.
__device__ __forceinline__ double block_sum_d(double v, double* sred) {
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
    __syncthreads();
    if (lane == 0) sred[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x / 32); ++k) t += sred[k];
    return t;
}

// Publishes Z = sum_i h1(y_i) - N given S = sum_i h1(y_i) = w0 . (K1 * w0)
// (equal: both are the sum of L_g(y_i) v1[g] over points and nodes).
__device__ void publish_Z(double S, const Job& J) {
    const double Z = S - (double)J.N;
    J.params->Z = Z;
    J.params->inv_Z = (float)(1.0 / Z);
    if (J.Z_out) *J.Z_out = Z;
}

// ----------------------------------------------------------------------------
// 2-D, pass 2: column pairs (k2, L - k2), k2 = 0 .. L/2 of a job. Forward FFT
// of six columns per pair (C0 and C1 at k2 and L - k2, CK and CG at k2),
// spectra products, inverse FFT of the four packed results, which overwrite
// the first n rows of columns k2 and L - k2 of C0 and C1.
// A work item takes cp adjacent pairs: its loads and stores of a row then
// touch cp consecutive values (whole sectors rather than one value in four),
// and each FFT stage has 6 cp transforms' butterflies for the CTA's threads.
// cp is as large as the launch's shared memory allows for the job's L, and
// no larger than keeps about 4 items per SM over the whole table (a lone
// small grid keeps one pair per item).
// Each pair's Parseval terms of Z are summed in an order fixed by L alone
// (lane l of one warp adds k1 = l, l + 32, ...; then an xor tree), so Z does
// not depend on cp or on the CTA size; the last item of a job adds the pairs'
// sums in pair order.
// Rows o1 < 0 of the kernels: CK row -r = CK row r (even); the CG row
// spectrum is real with X_{-r}[k2] = -X_r[L - k2] (G_1 odd, G_2 even in o1).
// At column L - k2 the kernel spectra are K^(k1, k2), S_1(k1, k2) and
// -S_2(k1, k2) (G_2 is odd in o2).
// ----------------------------------------------------------------------------
__device__ __forceinline__ int cols_per_item(int L, int smem_floats2, int total_pairs, int sm_count) {
    int cp = smem_floats2 / (12 * L);
    int want = total_pairs / (4 * sm_count);
    if (want < 1) want = 1;
    if (cp > want) cp = want;
    if (cp > 8) cp = 8;
    return cp < 1 ? 1 : cp;
}

__global__ void __launch_bounds__(1024)
cols_kernel(const Job* __restrict__ jobs, int njobs, Tables tab, int smem_floats2, int sm_count) {
    extern __shared__ float2 sm[];
    __shared__ int32_t s_start[kMaxJobs + 1];
    __shared__ FftEntry e;
    __shared__ bool s_last;
    // column pairs of the whole table, then items per job
    const int total_pairs = split_jobs(jobs, njobs, s_start, [](const Job& J) { return fft_cols_items(J); });
    const int total = split_jobs(jobs, njobs, s_start, [&](const Job& J) {
        const int pairs = fft_cols_items(J);
        if (!pairs) return 0;
        const int cp = cols_per_item(J.params->L, smem_floats2, total_pairs, sm_count);
        return (pairs + cp - 1) / cp;
    });
    const int lane = threadIdx.x % 32, wid = threadIdx.x / 32, nwarps = blockDim.x / 32;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int j = job_of(s_start, njobs, item);
        const Job& J = jobs[j];
        const int it = item - s_start[j], nk = s_start[j + 1] - s_start[j];
        const Params P = *J.params;
        if (threadIdx.x == 0) e = tab.fft[P.fft_idx];
        __syncthreads();
        const int n = P.n, L = P.L;
        const int cpj = cols_per_item(L, smem_floats2, total_pairs, sm_count);
        const int k2_0 = it * cpj;
        const int cp = min(cpj, L / 2 + 1 - k2_0);
        const float2* tw = tab.tw + e.tw_off;
        float2* C0 = J.spec;
        float2* C1 = J.spec + (int64_t)n * L;
        const float2* CK = J.spec + 2 * (int64_t)n * L;
        const float2* CG = J.spec + 3 * (int64_t)n * L;
        float2* X = sm;
        float2* Yb = sm + 6 * cp * L;
        const float2 z = make_float2(0.0f, 0.0f);
        for (int idx = threadIdx.x; idx < L * cp; idx += blockDim.x) {
            const int i = idx / cp, pq = idx - i * cp;
            const int k2 = k2_0 + pq, k2b = (L - k2) % L;
            float2* Xp = X + 6 * pq * L;
            const bool in = i < n;
            Xp[i] = in ? C0[(int64_t)i * L + k2] : z;
            Xp[L + i] = in ? C0[(int64_t)i * L + k2b] : z;
            Xp[2 * L + i] = in ? C1[(int64_t)i * L + k2] : z;
            Xp[3 * L + i] = in ? C1[(int64_t)i * L + k2b] : z;
            float2 ck = z, cg = z;
            if (in) {
                ck = CK[(int64_t)i * L + k2];
                cg = CG[(int64_t)i * L + k2];
            } else if (i > L - n) {
                ck = CK[(int64_t)(L - i) * L + k2];
                const float2 t = CG[(int64_t)(L - i) * L + k2b];
                cg = make_float2(-t.x, -t.y);
            }
            Xp[4 * L + i] = ck;
            Xp[5 * L + i] = cg;
        }
        __syncthreads();
        float2* F = fft_batch(X, Yb, e, 6 * cp, tw, -1.0f);
        float2* O = (F == X) ? Yb : X;
        double* zt = reinterpret_cast<double*>(O + 4 * cp * L);  // the buffer's unused tail
        for (int idx = threadIdx.x; idx < L * cp; idx += blockDim.x) {
            const int pq = idx / L, k1 = idx - pq * L;
            const int k2 = k2_0 + pq, k2b = (L - k2) % L;
            const float2* Fp = F + 6 * pq * L;
            float2* Op = O + 4 * pq * L;
            const int k1n = (L - k1) % L;
            const float2 xa = Fp[k1], xb = Fp[L + k1];
            const float2 xa_m = Fp[k1n], xb_m = Fp[L + k1n];
            // C0 = w0 + i d_1 split at (k1, k2) [a] and (k1, L - k2) [b]
            const float2 w0a = cscale(cadd(xa, conjf2(xb_m)), 0.5f);
            const float2 ta = csub(xa, conjf2(xb_m));
            const float2 d1a = make_float2(0.5f * ta.y, -0.5f * ta.x);
            const float2 w0b = cscale(cadd(xb, conjf2(xa_m)), 0.5f);
            const float2 tb = csub(xb, conjf2(xa_m));
            const float2 d1b = make_float2(0.5f * tb.y, -0.5f * tb.x);
            const float2 d2a = Fp[2 * L + k1], d2b = Fp[3 * L + k1];
            const float2 ck = Fp[4 * L + k1];      // (K1^, K2^)
            const float2 cg = Fp[5 * L + k1];      // i S1 - S2
            const float K1 = ck.x, K2 = ck.y, S1 = cg.y, S2 = -cg.x;
            // Parseval terms of Z + N at (k1, k2) and (k1, L - k2)
            double zp = ((double)w0a.x * w0a.x + (double)w0a.y * w0a.y) * (double)K1;
            if (k2b != k2) zp += ((double)w0b.x * w0b.x + (double)w0b.y * w0b.y) * (double)K1;
            // U1 = d1 K2 - i S1 w0, U2 = d2 K2 - i S2 w0, V = w0 K2 (S2 flips sign at L - k2)
            const float2 va = cscale(w0a, K2), vb = cscale(w0b, K2);
            const float2 u1a = csub(cscale(d1a, K2), mul_si(w0a, S1));
            const float2 u2a = csub(cscale(d2a, K2), mul_si(w0a, S2));
            const float2 u1b = csub(cscale(d1b, K2), mul_si(w0b, S1));
            const float2 u2b = cadd(cscale(d2b, K2), mul_si(w0b, S2));
            Op[k1] = cadd(u1a, mul_si(u2a, 1.0f));
            Op[L + k1] = cadd(u1b, mul_si(u2b, 1.0f));
            Op[2 * L + k1] = va;
            Op[3 * L + k1] = vb;
            zt[pq * L + k1] = zp;
        }
        __syncthreads();
        for (int pq = wid; pq < cp; pq += nwarps) {
            double zs = 0.0;
            for (int k1 = lane; k1 < L; k1 += 32) zs += zt[pq * L + k1];
            zs = warp_sum_d(zs);
            if (lane == 0) J.z_partial[k2_0 + pq] = zs;
        }
        __syncthreads();
        const float2* R = fft_batch(O, F, e, 4 * cp, tw, 1.0f);
        for (int idx = threadIdx.x; idx < n * cp; idx += blockDim.x) {
            const int i = idx / cp, pq = idx - i * cp;
            const int k2 = k2_0 + pq, k2b = (L - k2) % L;
            const float2* Rp = R + 4 * pq * L;
            C0[(int64_t)i * L + k2] = Rp[i];
            C1[(int64_t)i * L + k2] = Rp[2 * L + i];
            if (k2b != k2) {
                C0[(int64_t)i * L + k2b] = Rp[L + i];
                C1[(int64_t)i * L + k2b] = Rp[3 * L + i];
            }
        }
        if (threadIdx.x == 0) {
            __threadfence();
            s_last = (atomicAdd(&J.tickets[2], 1u) == (unsigned)nk - 1);
        }
        __syncthreads();
        if (s_last && threadIdx.x == 0) {
            __threadfence();
            J.tickets[2] = 0u;
            double S = 0.0;
            for (int q = 0; q <= L / 2; ++q) S += __ldcg(&J.z_partial[q]);
            publish_Z(S / ((double)L * (double)L), J);
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------
// 2-D, pass 3: inverse row FFTs of the first n rows of D0 and D1; node
// values (0, u'_1, u'_2, v) / L^2 for columns < n. A work item takes rp
// consecutive rows (2 rp transforms in one batch).
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
rows_inv_kernel(const Job* __restrict__ jobs, int njobs, Tables tab, int smem_floats2,
                int sm_count) {
    extern __shared__ float2 sm[];
    __shared__ int32_t s_start[kMaxJobs + 1];
    __shared__ FftEntry e;
    const int total_rows = split_jobs(jobs, njobs, s_start, [](const Job& J) { return fft_inv_items(J); });
    const int total = split_jobs(jobs, njobs, s_start, [&](const Job& J) {
        const int rows = fft_inv_items(J);
        if (!rows) return 0;
        const int rp = rows_per_item(J.params->L, 4, smem_floats2, total_rows, sm_count);
        return (rows + rp - 1) / rp;
    });
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int j = job_of(s_start, njobs, item);
        const Job& J = jobs[j];
        const Params P = *J.params;
        if (threadIdx.x == 0) e = tab.fft[P.fft_idx];
        __syncthreads();
        const int n = P.n, L = P.L;
        const int rpj = rows_per_item(L, 4, smem_floats2, total_rows, sm_count);
        const int r0 = (item - s_start[j]) * rpj;
        const int rp = min(rpj, n - r0);
        const float2* tw = tab.tw + e.tw_off;
        const float2* D0 = J.spec;
        const float2* D1 = J.spec + (int64_t)n * L;
        float4* __restrict__ hgrid = J.hgrid;
        float2* X = sm;
        float2* Yb = sm + 2 * rp * L;
        const float scale = 1.0f / ((float)L * (float)L);
        for (int idx = threadIdx.x; idx < rp * L; idx += blockDim.x) {
            const int q = idx / L, c = idx - q * L;
            X[2 * q * L + c] = D0[(int64_t)(r0 + q) * L + c];
            X[(2 * q + 1) * L + c] = D1[(int64_t)(r0 + q) * L + c];
        }
        __syncthreads();
        const float2* R = fft_batch(X, Yb, e, 2 * rp, tw, 1.0f);
        for (int idx = threadIdx.x; idx < rp * n; idx += blockDim.x) {
            const int q = idx / n, c = idx - q * n;
            const float2 a = R[2 * q * L + c], b = R[(2 * q + 1) * L + c];
            hgrid[(int64_t)(r0 + q) * n + c] = make_float4(0.0f, a.x * scale, a.y * scale, b.x * scale);
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------
// 1-D: the whole convolution of a job in one work item. Forward: C0 = w0 + i d_1 and
// CK' = (K1 + lam G_1) + i K2, lam a power of two (exact) that brings the
// largest |G_1(o)| = max o / (1 + delta^2 o^2)^2 near 1 (the maximum is
// 3 sqrt(3) / (16 delta) at o = 1 / (delta sqrt 3), or at o = n - 1), so the
// three kernels share a transform at comparable magnitudes and the parity
// split loses no accuracy.
// Spectrum of CK': K1^ + i (lam S_1 + K2^); K2^ is the even and lam S_1 the
// odd part of the imaginary part in k. Z from the Parseval sum; inverse:
// D0 = U1 + i V -> (u'_1, v). Node values (0, u'_1, 0, v) / L.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
conv1d_kernel(const Job* __restrict__ jobs, int njobs, Tables tab) {
    extern __shared__ float2 sm[];
    __shared__ int32_t s_start[kMaxJobs + 1];
    __shared__ FftEntry e;
    __shared__ double sred[32];
    const int total = split_jobs(jobs, njobs, s_start, [](const Job& J) { return fft_1d_items(J); });
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int j = job_of(s_start, njobs, item);
        const Job& J = jobs[j];
        const Params P = *J.params;
        if (threadIdx.x == 0) e = tab.fft[P.fft_idx];
        __syncthreads();
        const int n = P.n, L = P.L;
        const float2* tw = tab.tw + e.tw_off;
        const long long* __restrict__ w = J.w;
        const float inv = P.fx_inv;
        const float o_star = 1.0f / (P.delta * 1.7320508f);
        const float o_max = (float)(n - 1);
        const float om = fminf(o_star, o_max);
        const float den = 1.0f + P.delta2 * om * om;
        const float g_max = fmaxf(om / (den * den), 1.0f);
        const int lg = (int)rintf(log2f(g_max));
        const float lam = ldexpf(1.0f, -lg), inv_lam = ldexpf(1.0f, lg);
        float2* X = sm;
        float2* Yb = sm + 2 * L;
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            X[i] = i < n ? make_float2(fx(w[i], inv), fx(w[n + i], inv)) : make_float2(0.0f, 0.0f);
            const int o = circ_offset(i, n, L);
            float2 kv = make_float2(0.0f, 0.0f);
            if (o >= 0) {
                const float2 k = kernel_pair(P.delta2, o * o);
                const int so = (i < n) ? i : i - L;  // signed offset
                kv = make_float2(k.x + lam * (float)so * k.y, k.y);
            }
            X[L + i] = kv;
        }
        __syncthreads();
        float2* F = fft_batch(X, Yb, e, 2, tw, -1.0f);
        float2* O = (F == X) ? Yb : X;
        double zp = 0.0;
        for (int k = threadIdx.x; k < L; k += blockDim.x) {
            const int kn = (L - k) % L;
            const float2 x = F[k], xm = conjf2(F[kn]);
            const float2 w0 = cscale(cadd(x, xm), 0.5f);
            const float2 t = csub(x, xm);
            const float2 d1 = make_float2(0.5f * t.y, -0.5f * t.x);
            const float2 ck = F[L + k], ckn = F[L + kn];
            const float K1 = ck.x, K2 = 0.5f * (ck.y + ckn.y), S1 = 0.5f * (ck.y - ckn.y) * inv_lam;
            zp += ((double)w0.x * w0.x + (double)w0.y * w0.y) * (double)K1;
            const float2 u1 = csub(cscale(d1, K2), mul_si(w0, S1));
            O[k] = cadd(u1, mul_si(cscale(w0, K2), 1.0f));
        }
        const double zt = block_sum_d(zp, sred);
        if (threadIdx.x == 0) publish_Z(zt / (double)L, J);
        __syncthreads();
        const float2* R = fft_batch(O, F, e, 1, tw, 1.0f);
        const float scale = 1.0f / (float)L;
        float4* __restrict__ hgrid = J.hgrid;
        for (int g = threadIdx.x; g < n; g += blockDim.x)
            hgrid[g] = make_float4(0.0f, R[g].x * scale, 0.0f, R[g].y * scale);
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------
// Launch geometry depends only on the table's capacities, so one enqueued
// sequence (or a captured graph of it) serves every iteration whatever N_int
// the box rule picks.
// ----------------------------------------------------------------------------
static size_t smem_rows_fwd(int L_max) { return sizeof(float2) * std::max(2 * L_max, 8192); }
static size_t smem_cols(int L_max) { return sizeof(float2) * 12 * L_max; }
static size_t smem_rows_inv(int L_max) { return sizeof(float2) * std::max(4 * L_max, 8192); }
static size_t smem_1d(int L_max) { return sizeof(float2) * 4 * L_max; }

cudaError_t fft_configure(int s, int L_max) {
    cudaError_t e = cudaSuccess;
    if (s == 2) {
        e = cudaFuncSetAttribute(rows_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_rows_fwd(L_max));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_cols(L_max));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(rows_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_rows_inv(L_max));
    } else {
        e = cudaFuncSetAttribute(conv1d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_1d(L_max));
    }
    return e;
}

static int cap_grid(int64_t items, int64_t cap) {
    if (items > cap) items = cap;
    return (int)(items < 1 ? 1 : items);
}

cudaError_t launch_convolution(const Job* jobs, const TableCaps& c, const Tables& t,
                               cudaStream_t st) {
    const int64_t J = c.njobs;
    if (c.s == 2) {
        const int tr = c.fft_threads > 0 ? c.fft_threads : 256;
        const int tc = c.fft_threads > 0 ? c.fft_threads : 512;
        const int g1 = cap_grid(4 * (int64_t)c.max_n * J, 4LL * c.sm_count);
        // a lone job's grid already gives more rows than SMs: one row per item, and
        // the smaller shared-memory request keeps more CTAs resident
        const size_t sf = c.njobs > 1 ? smem_rows_fwd(c.max_L) : sizeof(float2) * 2 * c.max_L;
        rows_fwd_kernel<<<g1, tr, sf, st>>>(jobs, c.njobs, t, (int)(sf / sizeof(float2)), c.sm_count);
        const int g2 = cap_grid((int64_t)(c.max_L / 2 + 1) * J, 2LL * c.sm_count);
        cols_kernel<<<g2, tc, smem_cols(c.max_L), st>>>(jobs, c.njobs, t,
                                                       (int)(smem_cols(c.max_L) / sizeof(float2)),
                                                       c.sm_count);
        const int g3 = cap_grid((int64_t)c.max_n * J, 4LL * c.sm_count);
        const size_t si = c.njobs > 1 ? smem_rows_inv(c.max_L) : sizeof(float2) * 4 * c.max_L;
        rows_inv_kernel<<<g3, tr, si, st>>>(jobs, c.njobs, t, (int)(si / sizeof(float2)), c.sm_count);
    } else {
        const int g = cap_grid(J, c.sm_count);
        conv1d_kernel<<<g, 1024, smem_1d(c.max_L), st>>>(jobs, c.njobs, t);
    }
    return cudaGetLastError();
}

}  // namespace fitsne
