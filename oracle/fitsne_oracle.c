/*
 * FIt-SNE oracle: a plain, slow, FP64 CPU implementation of the t-SNE
 * gradient and of its interpolation/FFT approximation, written from
 * Linderman, Rachh, Hoskins, Steinerberger, Kluger, "Efficient Algorithms for
 * t-distributed Stochastic Neighborhood Embedding" (arXiv 1712.09005).
 *
 * TEST INFRASTRUCTURE. This file is the checker, not the product. Only the
 * test suite, the package smoke check and the CPU-baseline leg of the
 * benchmark may load it. It shares no code, header, table or helper with the
 * CUDA library, and it never consumes anything the CUDA library produced.
 *
 * Precision: every quantity is FP64, except the few decisions the method
 * takes on the FP32 embedding coordinates (bounding box, interval count and
 * the interval a point falls in). Those are evaluated in FP32 with IEEE
 * round-to-nearest and no contraction (build with -ffp-contract=off), so
 * that any implementation that follows the same rule lands every point in
 * the same interval.
 *
 * Contents, each citing the passage it follows:
 *   orc_exact_gradient  Sec. 1.1 (gradient, Z) and Sec. 1.2 (exaggeration),
 *                       split into attraction and Eq. (frep) repulsion.
 *   orc_kl              Sec. 1.1 (KL divergence C(Y)).
 *   orc_box             Sec. 2.2 / 2.4 (box, intervals) and Sec. 2.5 (N_int rule).
 *   orc_interp_gradient Sec. 2.1-2.4 (Steps 1-3, Eq. (equinodes),
 *                       Eq. (equikereval2), Algorithm 1, 2-D tensor version)
 *                       and the Appendix (h sums, F_rep = (h - y h)/Z).
 *   orc_fft             the radix-2 FFT used for the Toeplitz product (Sec. 2.2).
 *   orc_step / orc_run  gradient descent with exaggeration (Sec. 1.2, Sec. 4);
 *                       the momentum/gain constants are not in the paper.
 *
 * Readings where the paper is silent or inconsistent (also listed in the
 * design notes): sign of F_rep follows the gradient of Sec. 1.1; the self
 * term K(y_i, y_i) that the grid cannot exclude is kept in every h sum and
 * Z = sum_i h1(y_i) - N; a degenerate box (all coordinates equal) has width
 * 1; points on the upper edge belong to the last interval.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2

/* ------------------------------------------------------------------------ */
/* Kernels of Eq. (kers): K1 = (1+r^2)^-1, K2 = K1^2.                       */
/* ------------------------------------------------------------------------ */
static double kernel1(double r2) { return 1.0 / (1.0 + r2); }
static double kernel2(double r2) { double k = 1.0 / (1.0 + r2); return k * k; }

/* ------------------------------------------------------------------------ */
/* Exact gradient, Sec. 1.1:                                                */
/*   dC/dy_i = 4 sum_j (alpha p_ij - q_ij) q_ij Z (y_i - y_j)                */
/* written as 4 (alpha * attr_i + rep_i) with                               */
/*   attr_i = sum_j p_ij (y_i - y_j) / (1 + |y_i - y_j|^2)        (Sec. 3)  */
/*   rep_i  = sum_{l != i} (y_l - y_i) / (1 + |y_l - y_i|^2)^2 / Z (Eq. frep)*/
/*   Z      = sum_{k != l} 1 / (1 + |y_k - y_l|^2).                         */
/* O(N^2); Y is N x s row-major.                                            */
/* ------------------------------------------------------------------------ */
static double sqdist(const double* Y, int s, int64_t i, int64_t j) {
    double d2 = 0.0;
    for (int m = 0; m < s; ++m) {
        double d = Y[i * s + m] - Y[j * s + m];
        d2 += d * d;
    }
    return d2;
}

int orc_exact_gradient(int64_t N, int s, const double* Y, const int32_t* row_ptr,
                       const int32_t* col, const float* val, double alpha,
                       double* dY, double* Z_out, double* attr, double* rep) {
    if (N < 1 || s < 1 || s > 3) return ORC_EINVAL;
    double Z = 0.0;
#pragma omp parallel for reduction(+ : Z) schedule(static)
    for (int64_t k = 0; k < N; ++k) {
        double zk = 0.0;
        for (int64_t l = 0; l < N; ++l)
            if (l != k) zk += kernel1(sqdist(Y, s, k, l));
        Z += zk;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double a[3] = {0, 0, 0}, r[3] = {0, 0, 0};
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int64_t j = col[e];
            double w = (double)val[e] * kernel1(sqdist(Y, s, i, j));
            for (int m = 0; m < s; ++m) a[m] += w * (Y[i * s + m] - Y[j * s + m]);
        }
        for (int64_t l = 0; l < N; ++l) {
            if (l == i) continue;
            double k2 = kernel2(sqdist(Y, s, i, l));
            for (int m = 0; m < s; ++m) r[m] += k2 * (Y[l * s + m] - Y[i * s + m]);
        }
        for (int m = 0; m < s; ++m) {
            r[m] /= Z;
            if (attr) attr[i * s + m] = a[m];
            if (rep) rep[i * s + m] = r[m];
            dY[i * s + m] = 4.0 * (alpha * a[m] + r[m]);
        }
    }
    if (Z_out) *Z_out = Z;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* KL divergence, Sec. 1.1: C = sum_{ij} p_ij log(p_ij / q_ij) over the      */
/* stored entries of P, with q_ij = (1+|y_i-y_j|^2)^-1 / Z. Entries with     */
/* p_ij = 0 contribute 0.                                                    */
/* ------------------------------------------------------------------------ */
double orc_kl(int64_t N, int s, const double* Y, const int32_t* row_ptr,
              const int32_t* col, const float* val, double Z) {
    double C = 0.0;
#pragma omp parallel for reduction(+ : C) schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            double p = (double)val[e];
            if (p <= 0.0) continue;
            double q = kernel1(sqdist(Y, s, i, col[e])) / Z;
            C += p * log(p / q);
        }
    }
    return C;
}

/* ------------------------------------------------------------------------ */
/* Box and intervals (Sec. 2.2, Sec. 2.4, Sec. 2.5).                         */
/* All points lie in [y_min, y_max] (the square [y_min, y_max]^2 in 2-D);    */
/* it is cut into N_int equal intervals per dimension of width b, each       */
/* carrying p equispaced nodes of spacing delta = b / p.                     */
/* N_int rule (Sec. 2.5): the larger of a floor and the box width, here      */
/* max(n_min, ceil(width)), capped at n_int_max; or a fixed count.           */
/* The FP32 values below are the decisions an implementation must share.    */
/* ------------------------------------------------------------------------ */
typedef struct {
    float y_min;    /* lower corner of the box, every dimension */
    float width;    /* y_max - y_min (1 if all coordinates are equal) */
    float b;        /* interval width, width / N_int, FP32 */
    float inv_b;    /* 1 / b, FP32 */
    int32_t n_int;  /* intervals per dimension */
    int32_t p;      /* nodes per interval */
    double delta;   /* node spacing b / p (FP64) */
} orc_box_t;

typedef struct {
    int32_t p;            /* interpolation nodes per interval */
    int32_t n_int_fixed;  /* > 0: this many intervals per dimension */
    int32_t n_min;        /* floor of the automatic rule */
    int32_t n_int_max;    /* cap of the automatic rule */
    int32_t use_fft;      /* 0: literal Toeplitz sum; 1: FFT of the circulant embedding */
    int32_t force_box;    /* 1: take box_y_min / box_width instead of the bounding box */
    float box_y_min;
    float box_width;
} orc_opts_t;

static void finish_box(orc_box_t* bx, float y_min, float width, int n_int, int p) {
    bx->y_min = y_min;
    bx->width = width;
    bx->n_int = n_int;
    bx->p = p;
    bx->b = width / (float)n_int;
    bx->inv_b = 1.0f / bx->b;
    bx->delta = (double)bx->b / (double)p;
}

int orc_box(int64_t N, int s, const double* Y, const orc_opts_t* o, orc_box_t* bx) {
    if (N < 1 || s < 1 || o->p < 2) return ORC_EINVAL;
    if (o->force_box) {
        if (o->n_int_fixed < 1 || !(o->box_width > 0.0f)) return ORC_EINVAL;
        finish_box(bx, o->box_y_min, o->box_width, o->n_int_fixed, o->p);
        return ORC_OK;
    }
    float lo = (float)Y[0], hi = (float)Y[0];
    for (int64_t k = 0; k < N * s; ++k) {
        float v = (float)Y[k];
        if (v < lo) lo = v;
        if (v > hi) hi = v;
    }
    float width = hi - lo;
    if (!(width > 0.0f)) width = 1.0f;
    int n_int;
    if (o->n_int_fixed > 0) {
        n_int = o->n_int_fixed;
    } else {
        float c = ceilf(width);
        if (c > (float)o->n_int_max) c = (float)o->n_int_max;
        n_int = (int)c;
        if (n_int < o->n_min) n_int = o->n_min;
        if (n_int > o->n_int_max) n_int = o->n_int_max;
    }
    finish_box(bx, lo, width, n_int, o->p);
    return ORC_OK;
}

/* Interval holding coordinate y: floor((y - y_min) * inv_b) in FP32, clamped
 * to [0, N_int - 1] (points on the upper edge go to the last interval). */
static int interval_of(float y, const orc_box_t* bx) {
    float u = y - bx->y_min;
    float f = u * bx->inv_b;
    if (!(f >= 0.0f)) return 0;
    if (f >= (float)bx->n_int) return bx->n_int - 1;
    int l = (int)floorf(f);
    return l > bx->n_int - 1 ? bx->n_int - 1 : l;
}

/* Lagrange basis on the p equispaced nodes of one interval (Sec. 2.1,
 * Eq. (kerinterp)). In units of delta, measured from the interval's left
 * end, node j sits at j + 1/2 (Eq. (equinodes) scaled to the interval). */
static void lagrange(int p, double t, double* L) {
    for (int j = 0; j < p; ++j) {
        double num = 1.0, den = 1.0;
        for (int k = 0; k < p; ++k) {
            if (k == j) continue;
            num *= t - ((double)k + 0.5);
            den *= (double)(j - k);
        }
        L[j] = num / den;
    }
}

/* For point coordinate y (dimension-free): its interval l, the local
 * coordinate t = (y - (y_min + l b)) / delta and the p Lagrange weights. */
static int point_weights(double y, const orc_box_t* bx, double* L) {
    int l = interval_of((float)y, bx);
    double left = (double)bx->y_min + (double)l * (double)bx->b;
    double t = (y - left) / bx->delta;
    lagrange(bx->p, t, L);
    return l;
}

/* ------------------------------------------------------------------------ */
/* Radix-2 complex FFT (iterative Cooley-Tukey, bit reversal first).         */
/* sign = -1: forward, X_k = sum_j x_j e^{-2 pi i jk/n}; sign = +1: inverse  */
/* without the 1/n factor. n must be a power of two.                          */
/* ------------------------------------------------------------------------ */
int orc_fft(int64_t n, double* re, double* im, int sign) {
    if (n < 1 || (n & (n - 1))) return ORC_EINVAL;
    for (int64_t i = 1, j = 0; i < n; ++i) {
        int64_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    const double pi = 3.14159265358979323846;
    for (int64_t len = 2; len <= n; len <<= 1) {
        for (int64_t k = 0; k < len / 2; ++k) {
            double ang = (double)sign * 2.0 * pi * (double)k / (double)len;
            double wr = cos(ang), wi = sin(ang);
            for (int64_t i = 0; i < n; i += len) {
                int64_t a = i + k, b = i + k + len / 2;
                double xr = re[b] * wr - im[b] * wi;
                double xi = re[b] * wi + im[b] * wr;
                re[b] = re[a] - xr; im[b] = im[a] - xi;
                re[a] += xr; im[a] += xi;
            }
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Step 2 on the node grid (Eq. (equikereval2)): v_g = sum_g' K(g - g') w_g'  */
/* over the n^s nodes, K evaluated at the node offset (g - g') * delta.      */
/* ------------------------------------------------------------------------ */
typedef double (*kernel_fn)(double);

static void toeplitz_direct(int s, int64_t n, double delta, kernel_fn K,
                            const double* w, double* v) {
    int64_t G = (s == 1) ? n : n * n;
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < G; ++g) {
        int64_t g1 = (s == 1) ? g : g / n, g2 = (s == 1) ? 0 : g % n;
        double acc = 0.0;
        for (int64_t h = 0; h < G; ++h) {
            int64_t h1 = (s == 1) ? h : h / n, h2 = (s == 1) ? 0 : h % n;
            double d1 = (double)(g1 - h1) * delta, d2 = (double)(g2 - h2) * delta;
            acc += K(d1 * d1 + d2 * d2) * w[h];
        }
        v[g] = acc;
    }
}

/* The same product through the FFT (Sec. 2.2; Sec. 2.4 in 2-D): the Toeplitz
 * matrix is embedded in a circulant of length L >= 2n per dimension
 * (L a power of two). Offset index i stands for the signed offset i (i < n)
 * or i - L (i > L - n); the remaining entries are never reached by outputs
 * in [0, n) and are set to 0. */
static int64_t next_pow2(int64_t x) { int64_t L = 1; while (L < x) L <<= 1; return L; }

static void fft_2d(int64_t L, double* re, double* im, int sign, int s) {
    if (s == 1) { orc_fft(L, re, im, sign); return; }
#pragma omp parallel
    {
        double* cr = (double*)malloc(sizeof(double) * L);
        double* ci = (double*)malloc(sizeof(double) * L);
#pragma omp for schedule(static)
        for (int64_t r = 0; r < L; ++r) orc_fft(L, re + r * L, im + r * L, sign);
#pragma omp for schedule(static)
        for (int64_t c = 0; c < L; ++c) {
            for (int64_t r = 0; r < L; ++r) { cr[r] = re[r * L + c]; ci[r] = im[r * L + c]; }
            orc_fft(L, cr, ci, sign);
            for (int64_t r = 0; r < L; ++r) { re[r * L + c] = cr[r]; im[r * L + c] = ci[r]; }
        }
        free(cr);
        free(ci);
    }
}

/* Spectrum of the circulant embedding of kernel K on the node offsets. */
static int kernel_spectrum(int s, int64_t n, int64_t L, double delta, kernel_fn K,
                           double* kr, double* ki) {
    int64_t T = (s == 1) ? L : L * L;
    memset(kr, 0, sizeof(double) * T);
    memset(ki, 0, sizeof(double) * T);
    for (int64_t i1 = 0; i1 < ((s == 1) ? 1 : L); ++i1) {
        for (int64_t i2 = 0; i2 < L; ++i2) {
            int64_t a = (s == 1) ? i2 : i1, c = (s == 1) ? 0 : i2;
            int64_t oa = a < n ? a : (a > L - n ? a - L : INT64_MIN);
            int64_t oc = c < n ? c : (c > L - n ? c - L : INT64_MIN);
            if (oa == INT64_MIN || oc == INT64_MIN) continue;
            double d1 = (double)oa * delta, d2 = (double)oc * delta;
            kr[i1 * L + i2] = K(d1 * d1 + d2 * d2);
        }
    }
    fft_2d(L, kr, ki, -1, s);
    return ORC_OK;
}

/* Zero-padded spectrum of a node grid w (n^s values) on the L^s torus. */
static void grid_spectrum(int s, int64_t n, int64_t L, const double* w, double* xr, double* xi) {
    int64_t T = (s == 1) ? L : L * L;
    memset(xr, 0, sizeof(double) * T);
    memset(xi, 0, sizeof(double) * T);
    int64_t G = (s == 1) ? n : n * n;
    for (int64_t g = 0; g < G; ++g) {
        int64_t g1 = (s == 1) ? g : g / n, g2 = (s == 1) ? 0 : g % n;
        xr[(s == 1) ? g1 : g1 * L + g2] = w[g];
    }
    fft_2d(L, xr, xi, -1, s);
}

/* v = inverse FFT of (grid spectrum x kernel spectrum), read on [0, n)^s. */
static void apply_spectrum(int s, int64_t n, int64_t L, const double* xr, const double* xi,
                           const double* kr, const double* ki, double* tr, double* ti,
                           double* v) {
    int64_t T = (s == 1) ? L : L * L;
    for (int64_t t = 0; t < T; ++t) {
        tr[t] = xr[t] * kr[t] - xi[t] * ki[t];
        ti[t] = xr[t] * ki[t] + xi[t] * kr[t];
    }
    fft_2d(L, tr, ti, +1, s);
    int64_t G = (s == 1) ? n : n * n;
    for (int64_t g = 0; g < G; ++g) {
        int64_t g1 = (s == 1) ? g : g / n, g2 = (s == 1) ? 0 : g % n;
        v[g] = tr[(s == 1) ? g1 : g1 * L + g2] / (double)T;
    }
}

/* ------------------------------------------------------------------------ */
/* Interpolated gradient (Sec. 2.1-2.4 and the Appendix).                     */
/*                                                                           */
/* Step 1 (spread): w_c[g] = sum_i W_g(y_i) q_c(i) for the charges           */
/*   q_0 = 1 and q_m = y_i(m), m = 1..s, where W_g(y) is the product over    */
/*   dimensions of the Lagrange weight of node g in y's interval (zero for   */
/*   nodes of other intervals).                                              */
/* Step 2: v = Ktilde w on the node grid for the pairs (K1, q_0) -> h_1,     */
/*   (K2, q_m) -> h_{m+1}, (K2, q_0) -> h_{s+2} (Appendix).                  */
/* Step 3 (interpolate back): h_k(y_i) = sum_g W_g(y_i) v_k[g].              */
/* Then Z = sum_i h_1(y_i) - N, F_rep,i(m) = (h_{m+1} - y_i(m) h_{s+2}) / Z  */
/* (Appendix), attr_i exact over P (Sec. 3), dY = 4 (alpha attr + F_rep).    */
/*                                                                           */
/* Optional outputs: h (N x (s+2), the potentials at the points), w          */
/* ((s+1) x n^s node grids), attr and rep (N x s), the box.                  */
/* ------------------------------------------------------------------------ */
int orc_interp_gradient(int64_t N, int s, const double* Y, const int32_t* row_ptr,
                        const int32_t* col, const float* val, double alpha,
                        const orc_opts_t* o, double* dY, double* Z_out, double* h_out,
                        double* w_out, double* attr_out, double* rep_out,
                        orc_box_t* box_out) {
    if (N < 1 || (s != 1 && s != 2) || o->p < 2 || o->p > 16) return ORC_EINVAL;
    orc_box_t bx;
    int rc = orc_box(N, s, Y, o, &bx);
    if (rc) return rc;
    if (box_out) *box_out = bx;
    const int p = bx.p;
    const int64_t n = (int64_t)bx.n_int * p;
    const int64_t G = (s == 1) ? n : n * n;
    const int nch = s + 1;

    double* w = (double*)calloc((size_t)(nch * G), sizeof(double));
    double* v = (double*)calloc((size_t)((s + 2) * G), sizeof(double));
    double* h = (double*)calloc((size_t)(N * (s + 2)), sizeof(double));
    if (!w || !v || !h) { free(w); free(v); free(h); return ORC_ENOMEM; }

    /* Step 1: spread the charges onto the nodes of each point's interval. */
    for (int64_t i = 0; i < N; ++i) {
        double L0[16], L1[16];
        int l0 = point_weights(Y[i * s + 0], &bx, L0);
        int l1 = 0;
        if (s == 2) l1 = point_weights(Y[i * s + 1], &bx, L1);
        for (int j0 = 0; j0 < p; ++j0) {
            for (int j1 = 0; j1 < (s == 2 ? p : 1); ++j1) {
                double W = (s == 2) ? L0[j0] * L1[j1] : L0[j0];
                int64_t g = (s == 2) ? ((int64_t)(l0 * p + j0) * n + (l1 * p + j1))
                                     : (int64_t)(l0 * p + j0);
                w[0 * G + g] += W;
                for (int m = 0; m < s; ++m) w[(1 + m) * G + g] += W * Y[i * s + m];
            }
        }
    }
    if (w_out) memcpy(w_out, w, sizeof(double) * nch * G);

    /* Step 2: node-to-node interactions (Toeplitz / block-Toeplitz product). */
    struct { kernel_fn K; int ch; } pairs[4];
    int npair = 0;
    pairs[npair].K = kernel1; pairs[npair++].ch = 0;                      /* h_1 */
    for (int m = 0; m < s; ++m) { pairs[npair].K = kernel2; pairs[npair++].ch = 1 + m; } /* h_{m+1} */
    pairs[npair].K = kernel2; pairs[npair++].ch = 0;                      /* h_{s+2} */
    if (o->use_fft) {
        int64_t L = next_pow2(2 * n);
        int64_t T = (s == 1) ? L : L * L;
        double* buf = (double*)malloc(sizeof(double) * T * 2 * (2 + nch + 1));
        if (!buf) { free(w); free(v); free(h); return ORC_ENOMEM; }
        double *k1r = buf, *k1i = buf + T, *k2r = buf + 2 * T, *k2i = buf + 3 * T;
        double *tr = buf + 4 * T, *ti = buf + 5 * T;
        double* chr = buf + 6 * T; /* nch spectra, re and im interleaved per channel */
        kernel_spectrum(s, n, L, bx.delta, kernel1, k1r, k1i);
        kernel_spectrum(s, n, L, bx.delta, kernel2, k2r, k2i);
        for (int c = 0; c < nch; ++c)
            grid_spectrum(s, n, L, w + c * G, chr + 2 * c * T, chr + (2 * c + 1) * T);
        for (int k = 0; k < npair; ++k) {
            const double* kr = pairs[k].K == kernel1 ? k1r : k2r;
            const double* ki = pairs[k].K == kernel1 ? k1i : k2i;
            int c = pairs[k].ch;
            apply_spectrum(s, n, L, chr + 2 * c * T, chr + (2 * c + 1) * T, kr, ki, tr, ti,
                           v + k * G);
        }
        free(buf);
    } else {
        for (int k = 0; k < npair; ++k)
            toeplitz_direct(s, n, bx.delta, pairs[k].K, w + pairs[k].ch * G, v + k * G);
    }

    /* Step 3: interpolate the node values back to the points. */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double L0[16], L1[16];
        int l0 = point_weights(Y[i * s + 0], &bx, L0);
        int l1 = 0;
        if (s == 2) l1 = point_weights(Y[i * s + 1], &bx, L1);
        for (int k = 0; k < s + 2; ++k) {
            double acc = 0.0;
            for (int j0 = 0; j0 < p; ++j0) {
                for (int j1 = 0; j1 < (s == 2 ? p : 1); ++j1) {
                    double W = (s == 2) ? L0[j0] * L1[j1] : L0[j0];
                    int64_t g = (s == 2) ? ((int64_t)(l0 * p + j0) * n + (l1 * p + j1))
                                         : (int64_t)(l0 * p + j0);
                    acc += W * v[k * G + g];
                }
            }
            h[i * (s + 2) + k] = acc;
        }
    }

    /* Z and the forces. */
    double Zs = 0.0;
    for (int64_t i = 0; i < N; ++i) Zs += h[i * (s + 2) + 0];
    double Z = Zs - (double)N;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double a[2] = {0, 0};
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int64_t j = col[e];
            double q = (double)val[e] * kernel1(sqdist(Y, s, i, j));
            for (int m = 0; m < s; ++m) a[m] += q * (Y[i * s + m] - Y[j * s + m]);
        }
        for (int m = 0; m < s; ++m) {
            double frep = (h[i * (s + 2) + 1 + m] - Y[i * s + m] * h[i * (s + 2) + s + 1]) / Z;
            dY[i * s + m] = 4.0 * (alpha * a[m] + frep);
            if (attr_out) attr_out[i * s + m] = a[m];
            if (rep_out) rep_out[i * s + m] = frep;
        }
    }
    if (Z_out) *Z_out = Z;
    if (h_out) memcpy(h_out, h, sizeof(double) * N * (s + 2));
    free(w); free(v); free(h);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Gradient descent with exaggeration (Sec. 1.2, Sec. 4).                     */
/* alpha(iter) = early_alpha for iter < early_iters, late_alpha for the last  */
/* late_iters iterations of n_iter, 1 otherwise. The update itself is not     */
/* given by the paper; this is the usual t-SNE rule with per-coordinate       */
/* gains and momentum:                                                        */
/*   gain <- gain + gain_inc   if sign(dY) != sign(uY), else gain * gain_dec  */
/*   gain <- max(gain, min_gain)                                               */
/*   uY   <- mu * uY - lr * gain * dY;   Y <- Y + uY                           */
/* with mu = momentum_early before mom_switch_iter, momentum_late after.      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t n_iter;
    int32_t early_iters;
    int32_t late_iters;
    int32_t mom_switch_iter;
    double early_alpha;
    double late_alpha;
    double lr;
    double momentum_early;
    double momentum_late;
    double min_gain;
    double gain_inc;
    double gain_dec;
} orc_sched_t;

double orc_alpha(const orc_sched_t* sp, int iter) {
    if (iter < sp->early_iters) return sp->early_alpha;
    if (sp->late_iters > 0 && iter >= sp->n_iter - sp->late_iters) return sp->late_alpha;
    return 1.0;
}

static int sgn(double x) { return (x > 0.0) - (x < 0.0); }

int orc_step(int64_t N, int s, double* Y, double* uY, double* gains, const double* dY,
             const orc_sched_t* sp, int iter) {
    double mu = iter < sp->mom_switch_iter ? sp->momentum_early : sp->momentum_late;
    for (int64_t k = 0; k < N * s; ++k) {
        double g = gains[k];
        g = (sgn(dY[k]) != sgn(uY[k])) ? g + sp->gain_inc : g * sp->gain_dec;
        if (g < sp->min_gain) g = sp->min_gain;
        gains[k] = g;
        uY[k] = mu * uY[k] - sp->lr * g * dY[k];
        Y[k] += uY[k];
    }
    return ORC_OK;
}

/* Full run: n_iter iterations of interpolated gradient + step, starting with
 * uY = 0 and gains = 1; returns the KL divergence of the final embedding
 * (interpolated Z) in *kl_out. Y is updated in place. */
int orc_run(int64_t N, int s, double* Y, const int32_t* row_ptr, const int32_t* col,
            const float* val, const orc_opts_t* o, const orc_sched_t* sp, double* kl_out) {
    double* uY = (double*)calloc((size_t)(N * s), sizeof(double));
    double* gains = (double*)malloc(sizeof(double) * N * s);
    double* dY = (double*)malloc(sizeof(double) * N * s);
    if (!uY || !gains || !dY) { free(uY); free(gains); free(dY); return ORC_ENOMEM; }
    for (int64_t k = 0; k < N * s; ++k) gains[k] = 1.0;
    int rc = ORC_OK;
    double Z = 0.0;
    for (int it = 0; it < sp->n_iter && rc == ORC_OK; ++it) {
        rc = orc_interp_gradient(N, s, Y, row_ptr, col, val, orc_alpha(sp, it), o, dY, &Z,
                                 NULL, NULL, NULL, NULL, NULL);
        if (rc == ORC_OK) rc = orc_step(N, s, Y, uY, gains, dY, sp, it);
    }
    if (rc == ORC_OK && kl_out) {
        rc = orc_interp_gradient(N, s, Y, row_ptr, col, val, 1.0, o, dY, &Z,
                                 NULL, NULL, NULL, NULL, NULL);
        if (rc == ORC_OK) *kl_out = orc_kl(N, s, Y, row_ptr, col, val, Z);
    }
    free(uY); free(gains); free(dY);
    return rc;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
