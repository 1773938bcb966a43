// C ABI of the GB300 FIt-SNE library (declared in include/fitsne_gb300.h):
// plan construction (a one-row job table with scratch sized for the largest
// grid the plan allows, the FFT length table and its twiddles), argument
// validation, and the per-iteration launch sequence
//   box -> count/scan/scatter/spread -> rows/cols/rows FFT (+ Z) -> forces
//   (-> advance, in a run).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <vector>

#include "fitsne_internal.cuh"

using fitsne::FftEntry;
using fitsne::Job;
using fitsne::JobDyn;
using fitsne::Params;

namespace fitsne {

namespace {
thread_local char g_err[512] = "";
}

int set_error(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

void clear_error() { g_err[0] = 0; }

const char* last_error() { return g_err; }

// Binary point of the fixed-point spread: every spread value is a sum over
// at most N points of W (t - j - 1/2) or W, |W| <= lmax^s with lmax the
// largest Lagrange basis value on [0, p], |t - j - 1/2| <= p - 1/2. The shift
// keeps N times twice that bound below 2^62.
int fixed_point_shift(int64_t N, int s, int p) {
    double lmax = 0.0;
    for (int k = 0; k <= 4000; ++k) {
        const double t = p * (double)k / 4000.0;
        for (int j = 0; j < p; ++j) {
            double num = 1.0, den = 1.0;
            for (int m = 0; m < p; ++m) {
                if (m == j) continue;
                num *= t - (m + 0.5);
                den *= (double)(j - m);
            }
            lmax = std::max(lmax, fabs(num / den));
        }
    }
    const double C = pow(lmax, s) * std::max(1.0, p - 0.5) * 2.0;
    int shift = (int)floor(62.0 - log2((double)N * C));
    return std::min(shift, 60);
}

namespace {

bool smooth5(int L) {
    int x = L;
    for (int f : {2, 3, 5})
        while (x % f == 0) x /= f;
    return x == 1;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

int fft_set_create(int n_max, cudaStream_t st, FftSet* out) {
    std::vector<FftEntry> tab;
    int off = 0;
    for (int L = 4;; L += 2) {
        if (!smooth5(L)) continue;
        FftEntry e{};
        e.L = L;
        e.tw_off = off;
        int x = L, k = 0;
        while (x % 4 == 0) { e.radix[k++] = 4; x /= 4; }
        while (x % 2 == 0) { e.radix[k++] = 2; x /= 2; }
        while (x % 3 == 0) { e.radix[k++] = 3; x /= 3; }
        while (x % 5 == 0) { e.radix[k++] = 5; x /= 5; }
        e.nst = k;
        tab.push_back(e);
        off += L;
        if (L >= 2 * n_max) break;
    }
    std::vector<float2> tw(off);
    for (const FftEntry& e : tab)
        for (int j = 0; j < e.L; ++j) {
            const double a = -2.0 * M_PI * (double)j / (double)e.L;
            tw[e.tw_off + j] = make_float2((float)cos(a), (float)sin(a));
        }
    std::vector<int32_t> of_n(n_max + 1);
    for (int nn = 0, idx = 0; nn <= n_max; ++nn) {
        while (tab[idx].L < 2 * nn) ++idx;
        of_n[nn] = idx;
    }
    FftSet f;
    f.n_fft = (int)tab.size();
    f.L_max = tab.back().L;
    const size_t b0 = align256(sizeof(FftEntry) * tab.size());
    const size_t b1 = align256(sizeof(float2) * tw.size());
    const size_t b2 = align256(sizeof(int32_t) * of_n.size());
    void* base = nullptr;
    cudaError_t e = cudaMalloc(&base, b0 + b1 + b2);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(e == cudaErrorMemoryAllocation ? TSNE_ERR_OOM : TSNE_ERR_CUDA,
                         "cudaMalloc of the FFT tables: %s", cudaGetErrorString(e));
    }
    char* c = static_cast<char*>(base);
    f.table = reinterpret_cast<FftEntry*>(c);
    f.tw = reinterpret_cast<float2*>(c + b0);
    f.of_n = reinterpret_cast<int32_t*>(c + b0 + b1);
    f.bytes = b0 + b1 + b2;
    e = cudaMemcpyAsync(f.table, tab.data(), sizeof(FftEntry) * tab.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f.tw, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f.of_n, of_n.data(), sizeof(int32_t) * of_n.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host vectors go out of scope
    if (e != cudaSuccess) {
        cudaFree(base);
        return set_error(TSNE_ERR_CUDA, "FFT table upload: %s", cudaGetErrorString(e));
    }
    *out = f;
    return TSNE_OK;
}

void fft_set_destroy(FftSet* f) {
    if (f->table) cudaFree(f->table);
    *f = FftSet{};
}

JobLayout job_layout(int64_t N, int s, int p, int n_int_max, int L_max) {
    JobLayout l{};
    l.N = N;
    l.s = s;
    l.p = p;
    l.n_int_max = n_int_max;
    l.n_max = p * n_int_max;
    l.L_max = L_max;
    l.n_boxes_max = (s == 2) ? (int64_t)n_int_max * n_int_max : n_int_max;
    l.chunk_cap = N / kMinChunk + std::min<int64_t>(N, l.n_boxes_max) + 1;
    l.G = (s == 2) ? (int64_t)l.n_max * l.n_max : l.n_max;
    l.scan_items = (int)((l.n_boxes_max + kScanBlock - 1) / kScanBlock);
    return l;
}

// Walks the layout; with base == NULL only the size is computed.
static size_t carve(const JobLayout& l, char* base, bool with_state, Job* J) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + off : nullptr;
        off += align256(bytes);
        return p;
    };
    const int64_t ns = l.N * l.s;
    Job tmp{};
    Job* j = J ? J : &tmp;
    j->params = reinterpret_cast<Params*>(take(sizeof(Params)));
    j->box_partial = reinterpret_cast<float*>(take(sizeof(float) * 2 * kBoxBlocks));
    j->tickets = reinterpret_cast<unsigned*>(take(sizeof(unsigned) * 4));
    j->counts = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * l.n_boxes_max));
    j->box_start = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * (l.n_boxes_max + 1)));
    j->cursor = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * l.n_boxes_max));
    j->chunk_start = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * (l.n_boxes_max + 1)));
    j->chunk_box = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * l.chunk_cap));
    j->block_pts = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * l.scan_items));
    j->block_chunks = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * l.scan_items));
    j->sorted_y = reinterpret_cast<float*>(take(sizeof(float) * ns));
    j->w = reinterpret_cast<long long*>(take(sizeof(long long) * (l.s + 1) * l.G));
    j->spec = reinterpret_cast<float2*>(
        take(l.s == 2 ? sizeof(float2) * 4 * (size_t)l.n_max * l.L_max : 0));
    j->hgrid = reinterpret_cast<float4*>(take(sizeof(float4) * l.G));
    j->z_partial = reinterpret_cast<double*>(take(sizeof(double) * (l.L_max / 2 + 1)));
    if (with_state) {
        j->ybuf[1] = reinterpret_cast<float*>(take(sizeof(float) * ns));
        j->uY = reinterpret_cast<float*>(take(sizeof(float) * ns));
        j->gains = reinterpret_cast<float*>(take(sizeof(float) * ns));
    }
    return off;
}

size_t job_scratch_bytes(const JobLayout& lay, bool with_state) {
    return carve(lay, nullptr, with_state, nullptr);
}

void job_carve(const JobLayout& lay, void* base, bool with_state, Job* J) {
    carve(lay, static_cast<char*>(base), with_state, J);
}

cudaError_t job_zero(const JobLayout& lay, const Job& J, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(J.params, 0, sizeof(Params), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(J.tickets, 0, sizeof(unsigned) * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(J.counts, 0, sizeof(int32_t) * lay.n_boxes_max, st);
    return e;
}

void job_set_schedule(Job* J, const tsne_step_params* sp) {
    J->n_iter = sp->n_iter;
    J->early_iters = sp->early_iters;
    J->late_iters = sp->late_iters;
    J->mom_switch_iter = sp->mom_switch_iter;
    J->early_alpha = sp->early_alpha;
    J->late_alpha = sp->late_alpha;
    J->lr = sp->lr;
    J->momentum_early = sp->momentum_early;
    J->momentum_late = sp->momentum_late;
    J->min_gain = sp->min_gain;
    J->gain_inc = sp->gain_inc;
    J->gain_dec = sp->gain_dec;
}

}  // namespace fitsne

namespace {

using fitsne::set_error;

int cuda_fail(cudaError_t e, const char* what) {
    return set_error(TSNE_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CU(call, what)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);  \
    } while (0)

template <typename T>
int dalloc(T** p, size_t count, const char* what) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return set_error(e == cudaErrorMemoryAllocation ? TSNE_ERR_OOM : TSNE_ERR_CUDA,
                         "cudaMalloc of %s (%zu bytes): %s", what, count * sizeof(T),
                         cudaGetErrorString(e));
    }
    return TSNE_OK;
}

// Phase event record of the tracing hooks: five events per timed evaluation
// (start, after box, after sort+spread, after FFT, after forces).
struct Prof {
    std::vector<cudaEvent_t> free_ev;
    std::vector<std::array<cudaEvent_t, 5>> recs;
};

Prof* prof_of(tsne_plan* pl) {
    if (!pl->prof) pl->prof = new Prof();
    return static_cast<Prof*>(pl->prof);
}

cudaEvent_t take_event(Prof* pr) {
    cudaEvent_t e = nullptr;
    if (!pr->free_ev.empty()) {
        e = pr->free_ev.back();
        pr->free_ev.pop_back();
    } else {
        cudaEventCreate(&e);
    }
    return e;
}

void prof_begin(tsne_plan* pl) {
    if (!pl->profiling) return;
    Prof* pr = prof_of(pl);
    std::array<cudaEvent_t, 5> a;
    for (auto& e : a) e = take_event(pr);
    pr->recs.push_back(a);
    cudaEventRecord(a[0], pl->stream);
}

void prof_mark(tsne_plan* pl, int k) {
    if (!pl->profiling || !pl->prof) return;
    Prof* pr = static_cast<Prof*>(pl->prof);
    if (!pr->recs.empty()) cudaEventRecord(pr->recs.back()[k], pl->stream);
}

void free_prof(tsne_plan* pl) {
    if (!pl->prof) return;
    Prof* pr = static_cast<Prof*>(pl->prof);
    for (auto& a : pr->recs)
        for (auto e : a) cudaEventDestroy(e);
    for (auto e : pr->free_ev) cudaEventDestroy(e);
    delete pr;
    pl->prof = nullptr;
}

void free_plan(tsne_plan* pl) {
    free_prof(pl);
    if (pl->step_exec) cudaGraphExecDestroy(pl->step_exec);
    if (pl->g_in) cudaEventDestroy(pl->g_in);
    if (pl->g_out) cudaEventDestroy(pl->g_out);
    if (pl->gstream) cudaStreamDestroy(pl->gstream);
    fitsne::fft_set_destroy(&pl->fft);
    void* ptrs[] = {pl->job_mem,   pl->d_job,      pl->d_dyn,     pl->kl_partial, pl->kl_ticket,
                    pl->kl_out_dev, pl->valid_flag, pl->y_next,    pl->uY_run,     pl->gains_run,
                    pl->h_row_ptr, pl->h_col,      pl->h_val,     pl->h_Y,        pl->perm,
                    pl->inv,       pl->perm_next,  pl->inv_next,  pl->row_len,    pl->cur_of,
                    pl->rp2,       pl->col2,       pl->val2,      pl->sort_keys,  pl->scan_bsum,
                    pl->relabel_ticket, pl->tmp_state, pl->y_cur, pl->region_next,
                    pl->gperm,     pl->ginv,       pl->order_z,   pl->order_stats};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete pl;
}

int check_plan(const tsne_plan* pl) {
    if (!pl) return set_error(TSNE_ERR_INVALID_ARG, "plan is NULL");
    return TSNE_OK;
}

int check_csr(const tsne_plan* pl, const tsne_csr& P) {
    if (!P.row_ptr || (P.nnz > 0 && (!P.col || !P.val)))
        return set_error(TSNE_ERR_INVALID_ARG, "CSR pointer is NULL");
    if (P.nnz < 0 || P.nnz > INT32_MAX)
        return set_error(TSNE_ERR_INVALID_ARG, "nnz %lld out of range [0, 2^31)", (long long)P.nnz);
    (void)pl;
    return TSNE_OK;
}

int check_vec(const tsne_plan* pl, const void* p, const char* name) {
    if (!p) return set_error(TSNE_ERR_INVALID_ARG, "%s is NULL", name);
    if ((reinterpret_cast<uintptr_t>(p) & (pl->s == 2 ? 7 : 3)) != 0)
        return set_error(TSNE_ERR_INVALID_ARG, "%s is not %d-byte aligned", name, pl->s == 2 ? 8 : 4);
    return TSNE_OK;
}

float alpha_at(const tsne_step_params* sp, int it) {
    if (it < sp->early_iters) return sp->early_alpha;
    if (sp->late_iters > 0 && it >= sp->n_iter - sp->late_iters) return sp->late_alpha;
    return 1.0f;
}

// Writes the plan's table row to the device if it changed (and the JobDyn if
// dyn is given).
int upload_job(tsne_plan* pl, const JobDyn* dyn) {
    Job& J = pl->host_job;
    J.force_box = pl->force_box;
    J.force_y_min = pl->force_y_min;
    J.force_width = pl->force_width;
    J.force_n_int = pl->force_n_int;
    const bool same = pl->uploaded_valid && memcmp(&pl->uploaded, &J, sizeof(Job)) == 0;
    if (same && !dyn) return TSNE_OK;
    CU(fitsne::launch_job_write(pl->d_job, J, pl->d_dyn, dyn, pl->stream), "job table write");
    pl->launches += 1;
    pl->uploaded = J;
    pl->uploaded_valid = 1;
    return TSNE_OK;
}

void set_csr(tsne_plan* pl, const tsne_csr& P) {
    pl->host_job.row_ptr = P.row_ptr;
    pl->host_job.col = P.col;
    pl->host_job.val = P.val;
}

// The repulsive half of an iteration: box, sort, spread, convolution, Z.
// With timed set and tracing on, phase events 0..3 are recorded around it;
// the caller records event 4 after the force kernel.
int enqueue_field(tsne_plan* pl, bool timed, bool advance_first = false) {
    if (timed) prof_begin(pl);
    CU(fitsne::launch_box(pl->d_job, pl->caps, pl->tables, 0, pl->stream, advance_first ? 1 : 0),
       "box kernel launch");
    pl->launches += 1;
    if (timed) prof_mark(pl, 1);
    CU(fitsne::launch_sort_and_spread(pl->d_job, pl->caps, pl->stream), "sort/spread launch");
    pl->launches += 5;
    if (timed) prof_mark(pl, 2);
    CU(fitsne::launch_convolution(pl->d_job, pl->caps, pl->tables, pl->stream), "FFT launch");
    pl->launches += pl->s == 2 ? 3 : 1;
    if (timed) prof_mark(pl, 3);
    return TSNE_OK;
}

int enqueue_forces(tsne_plan* pl, int step) {
    if (pl->force_mode == TSNE_FORCE_GRID) {
        CU(fitsne::launch_forces(pl->d_job, pl->caps, step, pl->stream), "force kernel launch");
    } else {
        CU(fitsne::launch_forces_region(pl->d_job, pl->caps, step, pl->region_next,
                                        pl->n_regions, pl->stream),
           "force kernel launch");
    }
    pl->launches += 1;
    prof_mark(pl, 4);
    return TSNE_OK;
}

}  // namespace

extern "C" {

const char* tsne_version(void) { return "fitsne-gb300 0.2 (sm_103a)"; }

const char* tsne_last_error_string(void) { return fitsne::last_error(); }

void tsne_step_params_default(tsne_step_params* out) {
    if (!out) return;
    out->n_iter = 1000;
    out->early_iters = 250;
    out->late_iters = 0;
    out->mom_switch_iter = 250;
    out->early_alpha = 12.0f;
    out->late_alpha = 1.0f;
    out->lr = 200.0f;
    out->momentum_early = 0.5f;
    out->momentum_late = 0.8f;
    out->min_gain = 0.01f;
    out->gain_inc = 0.2f;
    out->gain_dec = 0.8f;
}

float tsne_alpha_at(const tsne_step_params* sp, int32_t iter) { return sp ? alpha_at(sp, iter) : 1.0f; }

int tsne_plan_create(int64_t N, int32_t s, int32_t n_intervals, int32_t p,
                     const tsne_plan_opts* opts, tsne_plan** out) {
    fitsne::clear_error();
    if (!out) return set_error(TSNE_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (s != 1 && s != 2) return set_error(TSNE_ERR_INVALID_ARG, "s must be 1 or 2 (got %d)", s);
    if (p < 2 || p > 5) return set_error(TSNE_ERR_INVALID_ARG, "p must be in [2, 5] (got %d)", p);
    if (N < 2 || N > INT32_MAX / 2) return set_error(TSNE_ERR_INVALID_ARG, "N must be in [2, 2^30) (got %lld)", (long long)N);
    tsne_plan_opts o{};
    if (opts) o = *opts;
    int n_min = o.n_min > 0 ? o.n_min : 50;
    // grid limits: 2-D column FFTs keep ten length-L columns in shared memory
    const int n_cap = (s == 2) ? 1200 : 3000;
    int n_int_max = o.n_int_max > 0 ? o.n_int_max : std::min(s == 2 ? 400 : 1000, n_cap / p);
    if ((int64_t)p * n_int_max > n_cap)
        return set_error(TSNE_ERR_INVALID_ARG, "p * n_int_max = %d exceeds %d nodes per dimension",
                         p * n_int_max, n_cap);
    if (n_intervals < 0 || n_intervals > n_int_max)
        return set_error(TSNE_ERR_INVALID_ARG, "n_intervals %d outside [0, %d]", n_intervals, n_int_max);
    if (n_min > n_int_max) n_min = n_int_max;

    tsne_plan* pl = new tsne_plan();
    memset(pl, 0, sizeof(*pl));
    pl->N = N;
    pl->s = s;
    pl->p = p;
    pl->n_int_fixed = n_intervals;
    pl->n_min = n_min;
    pl->n_int_max = n_int_max;
    pl->stream = (cudaStream_t)o.stream;
    pl->n_max = p * n_int_max;
    pl->fx_shift = fitsne::fixed_point_shift(N, s, p);
    pl->relabel_first = o.relabel_first == 0 ? 100 : o.relabel_first;
    pl->relabel_every = o.relabel_every > 0 ? o.relabel_every : 300;
    pl->force_mode = o.force_mode;
    pl->order_rounds = o.order_rounds == 0 ? 8 : (o.order_rounds < 0 ? 0 : o.order_rounds);
    if (pl->order_rounds > 64) {
        free_plan(pl);
        return set_error(TSNE_ERR_INVALID_ARG, "order_rounds %d exceeds 64", o.order_rounds);
    }
    if (pl->force_mode < TSNE_FORCE_AUTO || pl->force_mode > TSNE_FORCE_REGION) {
        free_plan(pl);
        return set_error(TSNE_ERR_INVALID_ARG, "unknown force_mode %d", o.force_mode);
    }
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&pl->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (ce != cudaSuccess) { free_plan(pl); return cuda_fail(ce, "device query"); }
    if (int rc = fitsne::fft_set_create(pl->n_max, pl->stream, &pl->fft)) { free_plan(pl); return rc; }
    pl->tables = fitsne::Tables{pl->fft.table, pl->fft.tw, pl->fft.of_n};
    pl->lay = fitsne::job_layout(N, s, p, n_int_max, pl->fft.L_max);

    const int kl_blocks = 4 * pl->sm_count;
    int rc = TSNE_OK;
#define ALLOC(ptr, count) \
    if (rc == TSNE_OK) rc = dalloc(&pl->ptr, (size_t)(count), #ptr)
    {
        char* jm = nullptr;
        rc = dalloc(&jm, fitsne::job_scratch_bytes(pl->lay, false), "job scratch");
        pl->job_mem = jm;
    }
    ALLOC(d_job, 1);
    ALLOC(d_dyn, 1);
    ALLOC(kl_partial, 2 * kl_blocks);
    ALLOC(kl_ticket, 1);
    ALLOC(kl_out_dev, 1);
    ALLOC(valid_flag, 1);
    ALLOC(y_next, N * s);
    ALLOC(uY_run, N * s);
    ALLOC(gains_run, N * s);
    int64_t Mpow = 1;
    while (Mpow < N) Mpow <<= 1;
    ALLOC(perm, N);
    ALLOC(inv, N);
    ALLOC(perm_next, N);
    ALLOC(inv_next, N);
    ALLOC(row_len, N);
    ALLOC(cur_of, N);
    ALLOC(rp2, N + 1);
    ALLOC(sort_keys, Mpow);
    ALLOC(scan_bsum, N / 2048 + 1);
    ALLOC(relabel_ticket, 1);
    ALLOC(tmp_state, N * s);
    ALLOC(y_cur, N * s);
    ALLOC(region_next, 1024);
#undef ALLOC
    if (rc != TSNE_OK) { free_plan(pl); return rc; }

    Job& J = pl->host_job;
    memset(&J, 0, sizeof(Job));
    fitsne::job_carve(pl->lay, pl->job_mem, false, &J);
    J.dyn = pl->d_dyn;
    J.N = N;
    J.n_int_fixed = n_intervals;
    J.n_min = n_min;
    J.n_int_max = n_int_max;
    J.fx_shift = pl->fx_shift;
    J.chunk = fitsne::kDefaultChunk;
    J.iter_end = INT32_MAX;
    J.n_int_table = nullptr;

    fitsne::TableCaps& c = pl->caps;
    c.s = s;
    c.p = p;
    c.njobs = 1;
    c.sum_N = N;
    c.sum_box_items = std::min<int64_t>(fitsne::kBoxBlocks, std::max<int64_t>(1, (N * s + 1023) / 1024));
    c.sum_chunk_cap = N / J.chunk + std::min<int64_t>(N, pl->lay.n_boxes_max) + 1;
    c.max_n = pl->n_max;
    c.max_L = pl->fft.L_max;
    c.max_scan_items = pl->lay.scan_items;
    c.sm_count = pl->sm_count;

    cudaStream_t st = pl->stream;
    ce = fitsne::job_zero(pl->lay, J, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(pl->kl_ticket, 0, sizeof(unsigned), st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(pl->relabel_ticket, 0, sizeof(unsigned), st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(pl->d_dyn, 0, sizeof(JobDyn), st);
    if (ce == cudaSuccess) {
        // the SM id range sizes the region schedule of the force kernel
        int* d = reinterpret_cast<int*>(pl->region_next);
        ce = fitsne::query_sm_id_count(d, st);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(&pl->n_regions, d, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce == cudaSuccess && (pl->n_regions < 1 || pl->n_regions > 1023)) pl->n_regions = pl->sm_count;
    }
    if (ce == cudaSuccess) ce = fitsne::fft_configure(s, pl->fft.L_max);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) { free_plan(pl); return cuda_fail(ce, "plan initialisation"); }
    *out = pl;
    return TSNE_OK;
}

int tsne_plan_destroy(tsne_plan* plan) {
    if (!plan) return TSNE_OK;
    cudaStreamSynchronize(plan->stream);
    free_plan(plan);
    return TSNE_OK;
}

int tsne_plan_set_box(tsne_plan* plan, float y_min, float width, int32_t n_int) {
    if (int rc = check_plan(plan)) return rc;
    if (!(width > 0.0f)) {
        plan->force_box = 0;
        return TSNE_OK;
    }
    if (!isfinite(y_min) || !isfinite(width) || n_int < 1 || n_int > plan->n_int_max)
        return set_error(TSNE_ERR_INVALID_ARG, "invalid box (y_min %g, width %g, n_int %d)", y_min,
                         width, n_int);
    plan->force_box = 1;
    plan->force_y_min = y_min;
    plan->force_width = width;
    plan->force_n_int = n_int;
    return TSNE_OK;
}

int tsne_gradient(tsne_plan* plan, tsne_csr P, const float* Y, float alpha, float* dY,
                  double* Z_out) {
    if (int rc = check_plan(plan)) return rc;
    if (int rc = check_csr(plan, P)) return rc;
    if (int rc = check_vec(plan, Y, "Y")) return rc;
    if (int rc = check_vec(plan, dY, "dY")) return rc;
    if (Y == dY) return set_error(TSNE_ERR_INVALID_ARG, "Y and dY must not alias");
    Job& J = plan->host_job;
    set_csr(plan, P);
    J.mode = fitsne::kModeGradient;
    J.alpha = alpha;
    J.ybuf[0] = J.ybuf[1] = const_cast<float*>(Y);
    J.dY = dY;
    J.uY = J.gains = nullptr;
    J.Z_out = Z_out;
    if (int rc = upload_job(plan, nullptr)) return rc;
    if (int rc = enqueue_field(plan, true)) return rc;
    return enqueue_forces(plan, 0);
}

int tsne_step(tsne_plan* plan, tsne_csr P, float* Y, float* uY, float* gains, int32_t iter,
              const tsne_step_params* sp) {
    if (int rc = check_plan(plan)) return rc;
    if (int rc = check_csr(plan, P)) return rc;
    if (int rc = check_vec(plan, Y, "Y")) return rc;
    if (int rc = check_vec(plan, uY, "uY")) return rc;
    if (int rc = check_vec(plan, gains, "gains")) return rc;
    if (!sp) return set_error(TSNE_ERR_INVALID_ARG, "step params are NULL");
    if (iter < 0) return set_error(TSNE_ERR_INVALID_ARG, "iter must be >= 0");
    Job& J = plan->host_job;
    set_csr(plan, P);
    J.mode = fitsne::kModeStep;
    fitsne::job_set_schedule(&J, sp);
    J.ybuf[0] = Y;
    J.ybuf[1] = plan->y_next;
    J.dY = nullptr;
    J.uY = uY;
    J.gains = gains;
    J.Z_out = nullptr;
    const JobDyn d{iter, 0, 0, 0};
    if (int rc = upload_job(plan, &d)) return rc;
    if (int rc = enqueue_field(plan, true)) return rc;
    if (int rc = enqueue_forces(plan, 1)) return rc;
    CU(cudaMemcpyAsync(Y, plan->y_next, sizeof(float) * plan->N * plan->s,
                       cudaMemcpyDeviceToDevice, plan->stream),
       "copy of the new Y");
    return TSNE_OK;
}

static int reset_run_state(tsne_plan* plan) {
    const int64_t M = plan->N * plan->s;
    CU(cudaMemsetAsync(plan->uY_run, 0, sizeof(float) * M, plan->stream), "uY reset");
    CU(fitsne::launch_fill(plan->gains_run, 1.0f, M, plan->sm_count, plan->stream), "gains reset");
    plan->launches += 1;
    plan->reordered = 0;
    return TSNE_OK;
}

static bool relabel_at(const tsne_plan* plan, int it) {
    if (plan->relabel_first < 0 || it < plan->relabel_first) return false;
    return (it - plan->relabel_first) % plan->relabel_every == 0;
}

// Relabels the run at the current state (Y in cur, in the current labels);
// the new-label Y is gathered through nxt and copied back into cur.
static int ensure_p2(tsne_plan* plan, int64_t nnz) {
    if (nnz <= plan->nnz2_cap && plan->col2) return TSNE_OK;
    if (plan->col2) cudaFree(plan->col2);
    if (plan->val2) cudaFree(plan->val2);
    plan->col2 = nullptr;
    plan->val2 = nullptr;
    plan->nnz2_cap = 0;
    plan->p2_holds_gorder = 0;
    plan->p2_is_run = 0;
    if (int rc = dalloc(&plan->col2, nnz, "relabelled col")) return rc;
    if (int rc = dalloc(&plan->val2, nnz, "relabelled val")) return rc;
    plan->nnz2_cap = nnz;
    return TSNE_OK;
}

static bool same_csr(const tsne_csr& a, const tsne_csr& b) {
    return a.row_ptr == b.row_ptr && a.col == b.col && a.val == b.val && a.nnz == b.nnz;
}

// Forgets the graph order and the prepared copy (P's contents may have changed).
static void forget_order(tsne_plan* plan) {
    plan->gorder_valid = 0;
    plan->gorder_prepared = 0;
    plan->p2_holds_gorder = 0;
}

// Graph order of P in gperm/ginv: computed unless it is already there for the
// same P (same pointers and nnz; a stale order after an in-place change of P
// still gives the same results, only the cache locality suffers).
static int graph_order_of(tsne_plan* plan, const tsne_csr& P, bool recompute) {
    if (!recompute && plan->gorder_valid && same_csr(plan->gorder_key, P)) return TSNE_OK;
    const int64_t N = plan->N;
    if (!plan->gperm)
        if (int rc = dalloc(&plan->gperm, N, "graph order")) return rc;
    if (!plan->ginv)
        if (int rc = dalloc(&plan->ginv, N, "graph order inverse")) return rc;
    if (!plan->order_z)
        if (int rc = dalloc(&plan->order_z, 4 * N, "graph order coordinates")) return rc;
    if (!plan->order_stats)
        if (int rc = dalloc(&plan->order_stats, 4 * 256 + 2, "graph order statistics")) return rc;
    forget_order(plan);
    CU(fitsne::launch_graph_order(plan, P, plan->order_rounds, plan->gperm, plan->ginv),
       "graph order launch");
    plan->gorder_valid = 1;
    plan->gorder_key = P;
    return TSNE_OK;
}

// Start of a run (iteration 0, caller's labels): moves the run to the graph
// order of P; the relabelled copy of P is rebuilt unless tsne_plan_order
// prepared it for this P and nothing has overwritten it since.
static int graph_relabel(tsne_plan* plan, const tsne_csr& P, float* cur, float* nxt) {
    if (int rc = ensure_p2(plan, P.nnz)) return rc;
    if (int rc = graph_order_of(plan, P, false)) return rc;
    const bool reuse = plan->gorder_prepared && plan->p2_holds_gorder;
    CU(fitsne::launch_apply_order(plan, P, plan->gperm, reuse ? 0 : 1, cur, plan->uY_run,
                                  plan->gains_run, nxt),
       "graph order relabel");
    plan->p2_holds_gorder = 1;
    plan->p2_is_run = 1;
    CU(cudaMemcpyAsync(cur, nxt, sizeof(float) * plan->N * plan->s, cudaMemcpyDeviceToDevice,
                       plan->stream),
       "relabelled Y copy");
    return TSNE_OK;
}

static int relabel(tsne_plan* plan, const tsne_csr& P, float* cur, float* nxt) {
    if (int rc = ensure_p2(plan, P.nnz)) return rc;
    plan->p2_holds_gorder = 0;  // the copy below replaces the graph-ordered one
    plan->p2_is_run = 1;
    // the box of the current Y (the curve keys are taken on it)
    CU(fitsne::launch_box(plan->d_job, plan->caps, plan->tables, 0, plan->stream), "box kernel launch");
    plan->launches += 1;
    CU(fitsne::launch_relabel(plan, P, cur, plan->uY_run, plan->gains_run, nxt), "relabel launch");
    CU(cudaMemcpyAsync(cur, nxt, sizeof(float) * plan->N * plan->s, cudaMemcpyDeviceToDevice,
                       plan->stream),
       "relabelled Y copy");
    return TSNE_OK;
}

// Captures the steady-state step (a step whose predecessor's advance is
// still pending) on the plan's private stream. The kernels read the job
// table in device memory, so one graph serves every such step of every run
// of the plan (relabellings rewrite the table, not the launches).
static int build_step_graph(tsne_plan* plan) {
    if (!plan->gstream) {
        CU(cudaStreamCreateWithFlags(&plan->gstream, cudaStreamNonBlocking), "graph stream");
        CU(cudaEventCreateWithFlags(&plan->g_in, cudaEventDisableTiming), "graph event");
        CU(cudaEventCreateWithFlags(&plan->g_out, cudaEventDisableTiming), "graph event");
    }
    cudaStream_t user = plan->stream;
    const int prof = plan->profiling;
    const int64_t l0 = plan->launches;
    plan->stream = plan->gstream;
    plan->profiling = 0;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(plan->gstream, cudaStreamCaptureModeThreadLocal);
    int rc = TSNE_OK;
    if (e == cudaSuccess) {
        rc = enqueue_field(plan, false, true);
        if (rc == TSNE_OK) rc = enqueue_forces(plan, 1);
        e = cudaStreamEndCapture(plan->gstream, &g);
    }
    plan->stream = user;
    plan->profiling = prof;
    plan->step_kernels = (int)(plan->launches - l0);
    plan->launches = l0;
    if (rc != TSNE_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "step capture");
    e = cudaGraphInstantiate(&plan->step_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        plan->step_exec = nullptr;
        return cuda_fail(e, "step graph instantiation");
    }
    return TSNE_OK;
}

// Iterations it0 .. it0+count-1. The table row holds ybuf = {y_cur, y_next};
// the device flips the current buffer after every step (advance kernel), the
// host follows the parity. Y (in the caller's labels) holds the input and
// receives the result.
static int run_iters(tsne_plan* plan, const tsne_csr& P, float* Y, const tsne_step_params* sp,
                     int it0, int count) {
    const int64_t ns = plan->N * plan->s;
    float* buf[2] = {plan->y_cur, plan->y_next};
    if (plan->reordered) CU(fitsne::launch_to_labels(plan, Y, 0, buf[0]), "Y to run labels");
    else CU(cudaMemcpyAsync(buf[0], Y, sizeof(float) * ns, cudaMemcpyDeviceToDevice, plan->stream), "Y copy");
    Job& J = plan->host_job;
    J.mode = fitsne::kModeStep;
    fitsne::job_set_schedule(&J, sp);
    J.ybuf[0] = buf[0];
    J.ybuf[1] = buf[1];
    J.dY = nullptr;
    J.uY = plan->uY_run;
    J.gains = plan->gains_run;
    J.Z_out = nullptr;
    if (plan->reordered && !plan->p2_is_run) {
        // a relabelled run continues after tsne_plan_order replaced its copy of P
        if (int rc = ensure_p2(plan, P.nnz)) return rc;
        CU(fitsne::launch_order_copy(plan, P, plan->perm, plan->inv), "relabelled copy of P");
        plan->p2_is_run = 1;
    }
    auto set_p = [&]() {
        if (plan->reordered) set_csr(plan, tsne_csr{plan->rp2, plan->col2, plan->val2, P.nnz});
        else set_csr(plan, P);
    };
    set_p();
    const JobDyn d{it0, 0, 0, 0};
    if (int rc = upload_job(plan, &d)) return rc;
    int par = 0;
    // the move of the job to its next iteration after a step is left to the
    // next step's bounding-box kernel (or to an advance launch before a
    // relabelling and at the end of the call)
    bool pending = false;
    // steady-state steps replay the step graph on gstream (one host call per
    // step) unless the phases are being traced
    const bool use_graph = !plan->profiling;
    bool in_graph = false;  // gstream holds the latest work
    auto join = [&]() -> int {
        if (!in_graph) return TSNE_OK;
        CU(cudaEventRecord(plan->g_out, plan->gstream), "graph fence");
        CU(cudaStreamWaitEvent(plan->stream, plan->g_out, 0), "graph fence");
        in_graph = false;
        return TSNE_OK;
    };
    auto advance = [&]() -> int {
        if (int rc = join()) return rc;
        CU(fitsne::launch_advance(plan->d_job, 1, plan->stream), "advance launch");
        plan->launches += 1;
        pending = false;
        return TSNE_OK;
    };
    for (int it = it0; it < it0 + count; ++it) {
        if (it == 0 && !plan->reordered && plan->order_rounds > 0) {
            if (pending)
                if (int rc = advance()) return rc;
            if (int rc = graph_relabel(plan, P, buf[par], buf[par ^ 1])) return rc;
            set_p();
            if (int rc = upload_job(plan, nullptr)) return rc;
        } else if (relabel_at(plan, it)) {
            if (pending)
                if (int rc = advance()) return rc;
            if (int rc = relabel(plan, P, buf[par], buf[par ^ 1])) return rc;
            set_p();
            if (int rc = upload_job(plan, nullptr)) return rc;
        }
        if (use_graph && pending) {
            if (!plan->step_exec)
                if (int rc = build_step_graph(plan)) return rc;
            if (!in_graph) {
                CU(cudaEventRecord(plan->g_in, plan->stream), "graph fence");
                CU(cudaStreamWaitEvent(plan->gstream, plan->g_in, 0), "graph fence");
                in_graph = true;
            }
            CU(cudaGraphLaunch(plan->step_exec, plan->gstream), "step graph launch");
            plan->launches += plan->step_kernels;
        } else {
            if (int rc = join()) return rc;
            if (int rc = enqueue_field(plan, true, pending)) return rc;
            if (int rc = enqueue_forces(plan, 1)) return rc;
        }
        pending = true;
        par ^= 1;
    }
    if (int rc = join()) return rc;
    if (pending)
        if (int rc = advance()) return rc;
    if (plan->reordered) CU(fitsne::launch_to_labels(plan, buf[par], 1, Y), "Y to caller labels");
    else CU(cudaMemcpyAsync(Y, buf[par], sizeof(float) * ns, cudaMemcpyDeviceToDevice, plan->stream), "Y copy");
    return TSNE_OK;
}

static int run_device(tsne_plan* plan, const tsne_csr& P, float* Y, const tsne_step_params* sp,
                      double* kl_out) {
    if (int rc = reset_run_state(plan)) return rc;
    if (int rc = run_iters(plan, P, Y, sp, 0, sp->n_iter)) return rc;
    if (kl_out) return tsne_kl(plan, P, Y, kl_out);
    return TSNE_OK;
}

int tsne_run_reset(tsne_plan* plan) {
    if (int rc = check_plan(plan)) return rc;
    return reset_run_state(plan);
}

// The run state in the caller's labels: a relabelled run's uY and gains are
// scattered back through the plan's free y_next buffer before the copy.
int tsne_run_state_save(tsne_plan* plan, float* uY_host, float* gains_host) {
    if (int rc = check_plan(plan)) return rc;
    if (!uY_host || !gains_host) return set_error(TSNE_ERR_INVALID_ARG, "NULL host buffer");
    const size_t bytes = sizeof(float) * (size_t)(plan->N * plan->s);
    const float* src[2] = {plan->uY_run, plan->gains_run};
    float* dst[2] = {uY_host, gains_host};
    for (int k = 0; k < 2; ++k) {
        const float* from = src[k];
        if (plan->reordered) {
            CU(fitsne::launch_to_labels(plan, src[k], 1, plan->y_next), "run state to caller labels");
            from = plan->y_next;
        }
        CU(cudaMemcpyAsync(dst[k], from, bytes, cudaMemcpyDeviceToHost, plan->stream), "run state read-back");
        CU(cudaStreamSynchronize(plan->stream), "run state synchronise");
    }
    return TSNE_OK;
}

int tsne_run_state_load(tsne_plan* plan, const float* uY_host, const float* gains_host) {
    if (int rc = check_plan(plan)) return rc;
    if (!uY_host || !gains_host) return set_error(TSNE_ERR_INVALID_ARG, "NULL host buffer");
    const size_t bytes = sizeof(float) * (size_t)(plan->N * plan->s);
    CU(cudaMemcpyAsync(plan->uY_run, uY_host, bytes, cudaMemcpyHostToDevice, plan->stream), "run state upload");
    CU(cudaMemcpyAsync(plan->gains_run, gains_host, bytes, cudaMemcpyHostToDevice, plan->stream),
       "run state upload");
    CU(cudaStreamSynchronize(plan->stream), "run state synchronise");
    plan->reordered = 0;  // the loaded state is in the caller's labels
    return TSNE_OK;
}

int tsne_run_iters(tsne_plan* plan, tsne_csr P, float* Y, const tsne_step_params* sp,
                   int32_t it_begin, int32_t count) {
    if (int rc = check_plan(plan)) return rc;
    if (int rc = check_csr(plan, P)) return rc;
    if (int rc = check_vec(plan, Y, "Y")) return rc;
    if (!sp || it_begin < 0 || count < 0) return set_error(TSNE_ERR_INVALID_ARG, "invalid iteration range");
    return run_iters(plan, P, Y, sp, it_begin, count);
}

int tsne_run(tsne_plan* plan, tsne_csr P, float* Y, const tsne_step_params* sp, double* kl_out) {
    if (int rc = check_plan(plan)) return rc;
    if (int rc = check_csr(plan, P)) return rc;
    if (int rc = check_vec(plan, Y, "Y")) return rc;
    if (!sp || sp->n_iter < 0) return set_error(TSNE_ERR_INVALID_ARG, "invalid step params");
    return run_device(plan, P, Y, sp, kl_out);
}

int tsne_plan_order(tsne_plan* plan, tsne_csr P) {
    if (int rc = check_plan(plan)) return rc;
    if (int rc = check_csr(plan, P)) return rc;
    if (plan->order_rounds <= 0)
        return set_error(TSNE_ERR_INVALID_ARG, "the plan was created without a graph order");
    if (int rc = ensure_p2(plan, P.nnz)) return rc;
    if (int rc = graph_order_of(plan, P, true)) return rc;
    CU(fitsne::launch_order_copy(plan, P, plan->gperm, plan->ginv), "graph order copy of P");
    plan->p2_holds_gorder = 1;
    plan->gorder_prepared = 1;
    plan->p2_is_run = 0;  // a relabelled run in progress rebuilds its copy when it continues
    return TSNE_OK;
}

int tsne_kl(tsne_plan* plan, tsne_csr P, const float* Y, double* kl_out) {
    if (int rc = check_plan(plan)) return rc;
    if (int rc = check_csr(plan, P)) return rc;
    if (int rc = check_vec(plan, Y, "Y")) return rc;
    if (!kl_out) return set_error(TSNE_ERR_INVALID_ARG, "kl_out is NULL");
    Job& J = plan->host_job;
    set_csr(plan, P);
    J.mode = fitsne::kModeGradient;
    J.ybuf[0] = J.ybuf[1] = const_cast<float*>(Y);
    J.dY = nullptr;
    J.Z_out = nullptr;
    if (int rc = upload_job(plan, nullptr)) return rc;
    if (int rc = enqueue_field(plan, false)) return rc;
    CU(fitsne::launch_kl_raw(P, Y, plan->N, plan->s, &J.params->Z, 0.0, plan->kl_partial,
                             plan->kl_ticket, plan->kl_out_dev, 4 * plan->sm_count, plan->stream),
       "KL kernel launch");
    plan->launches += 1;
    CU(cudaMemcpyAsync(kl_out, plan->kl_out_dev, sizeof(double), cudaMemcpyDeviceToHost,
                       plan->stream),
       "KL read-back");
    CU(cudaStreamSynchronize(plan->stream), "KL synchronise");
    return TSNE_OK;
}

int tsne_validate_csr(tsne_plan* plan, tsne_csr P) {
    if (int rc = check_plan(plan)) return rc;
    if (int rc = check_csr(plan, P)) return rc;
    CU(cudaMemsetAsync(plan->valid_flag, 0, sizeof(int32_t), plan->stream), "flag reset");
    CU(fitsne::launch_validate(P, plan->N, plan->valid_flag, plan->sm_count, plan->stream), "validate launch");
    plan->launches += 1;
    int32_t flag = 0;
    CU(cudaMemcpyAsync(&flag, plan->valid_flag, sizeof(int32_t), cudaMemcpyDeviceToHost,
                       plan->stream),
       "flag read-back");
    CU(cudaStreamSynchronize(plan->stream), "validate synchronise");
    if (flag) return set_error(TSNE_ERR_INVALID_ARG, "malformed CSR (row_ptr, col or val out of range)");
    return TSNE_OK;
}

int tsne_run_host(tsne_plan* plan, const int32_t* row_ptr, const int32_t* col, const float* val,
                  int64_t nnz, float* Y, const tsne_step_params* sp, double* kl_out) {
    if (int rc = check_plan(plan)) return rc;
    if (!row_ptr || !Y || (nnz > 0 && (!col || !val)) || !sp)
        return set_error(TSNE_ERR_INVALID_ARG, "NULL host pointer");
    if (nnz < 0 || nnz > INT32_MAX) return set_error(TSNE_ERR_INVALID_ARG, "nnz out of range");
    const int64_t N = plan->N;
    if (row_ptr[0] != 0 || row_ptr[N] != nnz)
        return set_error(TSNE_ERR_INVALID_ARG, "row_ptr[0] must be 0 and row_ptr[N] = nnz");
    if (nnz > plan->host_nnz_cap) {
        if (plan->h_col) cudaFree(plan->h_col);
        if (plan->h_val) cudaFree(plan->h_val);
        plan->h_col = nullptr;
        plan->h_val = nullptr;
        plan->host_nnz_cap = 0;
        if (int rc = dalloc(&plan->h_col, nnz, "host-path col")) return rc;
        if (int rc = dalloc(&plan->h_val, nnz, "host-path val")) return rc;
        plan->host_nnz_cap = nnz;
    }
    if (!plan->h_row_ptr)
        if (int rc = dalloc(&plan->h_row_ptr, N + 1, "host-path row_ptr")) return rc;
    if (!plan->h_Y)
        if (int rc = dalloc(&plan->h_Y, N * plan->s, "host-path Y")) return rc;
    cudaStream_t st = plan->stream;
    CU(cudaMemcpyAsync(plan->h_row_ptr, row_ptr, sizeof(int32_t) * (N + 1), cudaMemcpyHostToDevice, st), "row_ptr upload");
    if (nnz > 0) {
        CU(cudaMemcpyAsync(plan->h_col, col, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st), "col upload");
        CU(cudaMemcpyAsync(plan->h_val, val, sizeof(float) * nnz, cudaMemcpyHostToDevice, st), "val upload");
    }
    CU(cudaMemcpyAsync(plan->h_Y, Y, sizeof(float) * N * plan->s, cudaMemcpyHostToDevice, st), "Y upload");
    tsne_csr P{plan->h_row_ptr, plan->h_col, plan->h_val, nnz};
    forget_order(plan);  // new contents at the same device addresses
    if (int rc = tsne_validate_csr(plan, P)) return rc;
    if (int rc = run_device(plan, P, plan->h_Y, sp, kl_out)) return rc;
    CU(cudaMemcpyAsync(Y, plan->h_Y, sizeof(float) * N * plan->s, cudaMemcpyDeviceToHost, st), "Y download");
    CU(cudaStreamSynchronize(st), "run synchronise");
    return TSNE_OK;
}

int tsne_plan_status(tsne_plan* plan) {
    if (int rc = check_plan(plan)) return rc;
    int32_t err = 0;
    Params* pr = plan->host_job.params;
    CU(cudaMemcpyAsync(&err, &pr->error, sizeof(int32_t), cudaMemcpyDeviceToHost, plan->stream),
       "status read-back");
    CU(cudaStreamSynchronize(plan->stream), "status synchronise");
    if (err) {
        CU(cudaMemsetAsync(&pr->error, 0, sizeof(int32_t), plan->stream), "status clear");
        CU(cudaStreamSynchronize(plan->stream), "status synchronise");
        return set_error(err, "non-finite coordinate in Y");
    }
    return TSNE_OK;
}

int tsne_plan_info(tsne_plan* plan, tsne_plan_info_t* out) {
    if (int rc = check_plan(plan)) return rc;
    if (!out) return set_error(TSNE_ERR_INVALID_ARG, "out is NULL");
    Params P;
    CU(cudaMemcpyAsync(&P, plan->host_job.params, sizeof(Params), cudaMemcpyDeviceToHost, plan->stream),
       "params read-back");
    CU(cudaStreamSynchronize(plan->stream), "info synchronise");
    out->y_min = P.y_min;
    out->width = P.width;
    out->b = P.b;
    out->delta = P.delta;
    out->n_int = P.n_int;
    out->n = P.n;
    out->fft_len = P.L;
    out->n_chunks = P.n_chunks;
    out->Z = P.Z;
    out->status = P.error;
    out->pad = 0;
    return TSNE_OK;
}

int tsne_debug_copy(tsne_plan* plan, int32_t which, void* host_dst, size_t bytes,
                    size_t* bytes_needed) {
    if (int rc = check_plan(plan)) return rc;
    const Job& J = plan->host_job;
    Params P;
    CU(cudaMemcpyAsync(&P, J.params, sizeof(Params), cudaMemcpyDeviceToHost, plan->stream),
       "params read-back");
    CU(cudaStreamSynchronize(plan->stream), "debug synchronise");
    const int64_t G = (plan->s == 2) ? (int64_t)P.n * P.n : P.n;
    size_t need = 0;
    switch (which) {
        case 0: need = sizeof(double) * (plan->s + 1) * G; break;
        case 1: need = sizeof(float4) * G; break;
        case 2: need = sizeof(int32_t) * (P.n_boxes + 1); break;
        default: return set_error(TSNE_ERR_INVALID_ARG, "unknown buffer %d", which);
    }
    if (bytes_needed) *bytes_needed = need;
    if (!host_dst) return TSNE_OK;
    if (bytes < need) return set_error(TSNE_ERR_INVALID_ARG, "buffer too small (%zu < %zu)", bytes, need);
    if (which == 0) {
        std::vector<long long> raw((size_t)((plan->s + 1) * G));
        CU(cudaMemcpyAsync(raw.data(), J.w, sizeof(long long) * raw.size(),
                           cudaMemcpyDeviceToHost, plan->stream),
           "debug copy");
        CU(cudaStreamSynchronize(plan->stream), "debug synchronise");
        double* out = static_cast<double*>(host_dst);
        const double inv = ldexp(1.0, -P.fx_shift);
        for (size_t k = 0; k < raw.size(); ++k) out[k] = (double)raw[k] * inv;
        return TSNE_OK;
    }
    const void* src = which == 1 ? (const void*)J.hgrid : (const void*)J.box_start;
    CU(cudaMemcpyAsync(host_dst, src, need, cudaMemcpyDeviceToHost, plan->stream), "debug copy");
    CU(cudaStreamSynchronize(plan->stream), "debug synchronise");
    return TSNE_OK;
}

int tsne_plan_profile(tsne_plan* plan, int32_t enable) {
    if (int rc = check_plan(plan)) return rc;
    plan->profiling = enable != 0;
    return TSNE_OK;
}

int tsne_plan_profile_read(tsne_plan* plan, double* ms_out, int64_t* count_out) {
    if (int rc = check_plan(plan)) return rc;
    double ms[4] = {0, 0, 0, 0};
    int64_t cnt = 0;
    CU(cudaStreamSynchronize(plan->stream), "profile synchronise");
    if (plan->prof) {
        Prof* pr = static_cast<Prof*>(plan->prof);
        for (auto& a : pr->recs) {
            for (int k = 0; k < 4; ++k) {
                float t = 0.0f;
                CU(cudaEventElapsedTime(&t, a[k], a[k + 1]), "event elapsed time");
                ms[k] += t;
            }
            ++cnt;
            for (auto e : a) pr->free_ev.push_back(e);
        }
        pr->recs.clear();
    }
    for (int k = 0; k < 4; ++k) {
        if (ms_out) ms_out[k] = ms[k];
        if (count_out) count_out[k] = cnt;
    }
    return TSNE_OK;
}

int64_t tsne_plan_launch_count(const tsne_plan* plan) { return plan ? plan->launches : 0; }

}  // extern "C"
