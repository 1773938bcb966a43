// Batched form of the gradient iteration: many independent embedding jobs
// (each its own P, Y, optimizer state, box, grid and FFT length) advance
// together, one launch per phase serving every job of a device job table,
// with the whole iteration captured once in a CUDA graph and replayed. Jobs
// join and leave between iterations (their scratch comes from the
// stream-ordered allocator, so this never synchronises the device); an
// autotuner picks the spread work-item size, the threads per CTA of the FFT
// passes and the interval-count policy by timing the jobs themselves.
//
// Nothing here changes the arithmetic of a job: a job's iterations in a
// batch are bitwise equal to the same job run alone (in a batch or a plan
// without relabelling, at the same tuning), because no kernel combines
// values of different jobs and every reduction has a fixed order.
#include <string.h>

#include <algorithm>
#include <vector>

#include "fitsne_internal.cuh"

using fitsne::Job;
using fitsne::JobDyn;
using fitsne::JobLayout;
using fitsne::set_error;

namespace {

struct Slot {
    bool used = false;
    int64_t N = 0;
    int64_t nnz = 0;
    JobLayout lay{};
    char* mem = nullptr;
    size_t bytes = 0;
    Job job{};
};

}  // namespace

struct tsne_batch {
    int s, p, n_min, n_int_max, max_jobs;
    cudaStream_t stream;
    bool own_stream;
    int sm_count;
    fitsne::FftSet fft;
    fitsne::Tables tables;
    Job* d_table;          // [max_jobs] rows of the used slots, in slot order
    Job* h_table;          // pinned staging of the table upload
    cudaEvent_t table_ev;  // the last upload from h_table has been read
    JobDyn* d_dyn;         // [max_jobs] by slot
    JobDyn* h_dyn;         // pinned [max_jobs]
    int32_t* d_fill_table; // [n_int_max + 1] interval policy "fill the FFT length"
    std::vector<Slot> slots;
    std::vector<int> order;  // slot of each table row
    fitsne::TableCaps caps;
    bool dirty;
    tsne_batch_tuning tuning;
    bool use_graph;
    cudaGraphExec_t exec;
    double* kl_partial;
    unsigned* kl_ticket;
    double* kl_out;
    unsigned* region_next;  // [n_regions + 1] counters of the SM-local force schedule
    int n_regions;
    int64_t launches;
    int64_t bytes_in_use;
};

namespace {

int cuda_fail(cudaError_t e, const char* what) {
    return set_error(TSNE_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CU(call, what)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);  \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t slot_bytes(const JobLayout& lay) {
    return fitsne::job_scratch_bytes(lay, true) + align256(sizeof(float) * lay.N * lay.s);
}

int check_batch(const tsne_batch* b) {
    if (!b) return set_error(TSNE_ERR_INVALID_ARG, "batch is NULL");
    return TSNE_OK;
}

int check_id(const tsne_batch* b, int32_t id) {
    if (id < 0 || id >= b->max_jobs || !b->slots[id].used)
        return set_error(TSNE_ERR_INVALID_ARG, "no job %d in the batch", id);
    return TSNE_OK;
}

void drop_graph(tsne_batch* b) {
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
}

// Interval policy "fill": for rule value r, the largest N_int whose node
// count still fits the FFT length the rule's own N_int gets (more intervals
// at the same transform size), capped at n_int_max.
std::vector<int32_t> fill_table(int n_int_max, int p, const std::vector<int>& lengths) {
    std::vector<int32_t> t(n_int_max + 1);
    for (int r = 0; r <= n_int_max; ++r) {
        int L = 0;
        for (int x : lengths)
            if (x >= 2 * p * r) { L = x; break; }
        int m = L / (2 * p);
        if (m < r) m = r;
        if (m > n_int_max) m = n_int_max;
        t[r] = m;
    }
    return t;
}

void apply_tuning(tsne_batch* b, Job* J) {
    J->chunk = b->tuning.chunk;
    J->n_int_table = b->tuning.n_int_policy == TSNE_NINT_FILL ? b->d_fill_table : nullptr;
}

void recompute_caps(tsne_batch* b) {
    fitsne::TableCaps& c = b->caps;
    c.s = b->s;
    c.p = b->p;
    c.njobs = (int)b->order.size();
    c.sum_N = 0;
    c.sum_box_items = 0;
    c.sum_chunk_cap = 0;
    c.max_n = b->p * b->n_int_max;
    c.max_L = b->fft.L_max;
    c.max_scan_items = 1;
    c.sm_count = b->sm_count;
    c.fft_threads = b->tuning.fft_threads;
    for (int sl : b->order) {
        const Slot& S = b->slots[sl];
        c.sum_N += S.N;
        c.sum_box_items += std::min<int64_t>(fitsne::kBoxBlocks, std::max<int64_t>(1, (S.N * b->s + 1023) / 1024));
        c.sum_chunk_cap += S.N / b->tuning.chunk + std::min<int64_t>(S.N, S.lay.n_boxes_max) + 1;
        c.max_scan_items = std::max(c.max_scan_items, S.lay.scan_items);
    }
}

int upload_table(tsne_batch* b) {
    b->order.clear();
    for (int i = 0; i < b->max_jobs; ++i)
        if (b->slots[i].used) b->order.push_back(i);
    CU(cudaEventSynchronize(b->table_ev), "table staging wait");
    for (size_t k = 0; k < b->order.size(); ++k) {
        Job& J = b->slots[b->order[k]].job;
        apply_tuning(b, &J);
        b->h_table[k] = J;
    }
    if (!b->order.empty())
        CU(cudaMemcpyAsync(b->d_table, b->h_table, sizeof(Job) * b->order.size(),
                           cudaMemcpyHostToDevice, b->stream),
           "table upload");
    CU(cudaEventRecord(b->table_ev, b->stream), "table event");
    recompute_caps(b);
    drop_graph(b);
    b->dirty = false;
    return TSNE_OK;
}

int enqueue_iteration(tsne_batch* b) {
    const fitsne::TableCaps& c = b->caps;
    CU(fitsne::launch_box(b->d_table, c, b->tables, 0, b->stream), "box launch");
    CU(fitsne::launch_sort_and_spread(b->d_table, c, b->stream), "sort/spread launch");
    CU(fitsne::launch_convolution(b->d_table, c, b->tables, b->stream), "FFT launch");
    CU(fitsne::launch_forces_region(b->d_table, c, 1, b->region_next, b->n_regions, b->stream),
       "force launch");
    CU(fitsne::launch_advance(b->d_table, c.njobs, b->stream), "advance launch");
    return TSNE_OK;
}

int capture(tsne_batch* b) {
    drop_graph(b);
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    int rc = enqueue_iteration(b);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (rc != TSNE_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        return cuda_fail(e, "graph instantiation");
    }
    return TSNE_OK;
}

int iterate(tsne_batch* b, int count) {
    if (b->dirty)
        if (int rc = upload_table(b)) return rc;
    if (b->order.empty() || count <= 0) return TSNE_OK;
    if (b->use_graph && !b->exec)
        if (int rc = capture(b)) return rc;
    for (int k = 0; k < count; ++k) {
        if (b->use_graph) CU(cudaGraphLaunch(b->exec, b->stream), "graph launch");
        else if (int rc = enqueue_iteration(b)) return rc;
    }
    b->launches += (int64_t)count * fitsne::phase_launches(b->s);
    return TSNE_OK;
}

int table_row(const tsne_batch* b, int32_t id) {
    for (size_t k = 0; k < b->order.size(); ++k)
        if (b->order[k] == id) return (int)k;
    return -1;
}

// Saved optimizer state of every job (for the autotuner's trials).
struct Snapshot {
    char* mem = nullptr;
    std::vector<size_t> off;
};

int snapshot(tsne_batch* b, Snapshot* sn, bool restore) {
    size_t total = 0;
    if (!restore) {
        sn->off.assign(b->max_jobs, 0);
        for (int sl : b->order) {
            sn->off[sl] = total;
            total += 4 * align256(sizeof(float) * b->slots[sl].N * b->s);
        }
        total += align256(sizeof(JobDyn) * b->max_jobs);
        CU(cudaMallocAsync((void**)&sn->mem, total, b->stream), "snapshot allocation");
    }
    for (int sl : b->order) {
        const Slot& S = b->slots[sl];
        const size_t one = sizeof(float) * S.N * b->s;
        float* bufs[4] = {S.job.ybuf[0], S.job.ybuf[1], S.job.uY, S.job.gains};
        for (int q = 0; q < 4; ++q) {
            char* keep = sn->mem + sn->off[sl] + q * align256(one);
            if (restore) CU(cudaMemcpyAsync(bufs[q], keep, one, cudaMemcpyDeviceToDevice, b->stream), "restore");
            else CU(cudaMemcpyAsync(keep, bufs[q], one, cudaMemcpyDeviceToDevice, b->stream), "save");
        }
    }
    size_t dyn_off = 0;
    for (int sl : b->order) dyn_off = std::max(dyn_off, sn->off[sl] + 4 * align256(sizeof(float) * b->slots[sl].N * b->s));
    char* keep = sn->mem + dyn_off;
    if (restore) CU(cudaMemcpyAsync(b->d_dyn, keep, sizeof(JobDyn) * b->max_jobs, cudaMemcpyDeviceToDevice, b->stream), "restore");
    else CU(cudaMemcpyAsync(keep, b->d_dyn, sizeof(JobDyn) * b->max_jobs, cudaMemcpyDeviceToDevice, b->stream), "save");
    return TSNE_OK;
}

}  // namespace

extern "C" {

void tsne_batch_opts_default(tsne_batch_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->max_jobs = 64;
    o->use_graph = 1;
}

int tsne_batch_create(int32_t s, int32_t p, const tsne_batch_opts* opts, tsne_batch** out) {
    fitsne::clear_error();
    if (!out) return set_error(TSNE_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (s != 1 && s != 2) return set_error(TSNE_ERR_INVALID_ARG, "s must be 1 or 2 (got %d)", s);
    if (p < 2 || p > 5) return set_error(TSNE_ERR_INVALID_ARG, "p must be in [2, 5] (got %d)", p);
    tsne_batch_opts o;
    tsne_batch_opts_default(&o);
    if (opts) o = *opts;
    const int max_jobs = o.max_jobs > 0 ? o.max_jobs : 64;
    if (max_jobs > fitsne::kMaxJobs)
        return set_error(TSNE_ERR_INVALID_ARG, "max_jobs %d exceeds %d", max_jobs, fitsne::kMaxJobs);
    int n_min = o.n_min > 0 ? o.n_min : 50;
    const int n_cap = (s == 2) ? 1200 : 3000;
    const int n_int_max = o.n_int_max > 0 ? o.n_int_max : std::min(s == 2 ? 400 : 1000, n_cap / p);
    if ((int64_t)p * n_int_max > n_cap)
        return set_error(TSNE_ERR_INVALID_ARG, "p * n_int_max = %d exceeds %d nodes per dimension",
                         p * n_int_max, n_cap);
    if (n_min > n_int_max) n_min = n_int_max;
    tsne_batch* b = new tsne_batch();
    b->s = s;
    b->p = p;
    b->n_min = n_min;
    b->n_int_max = n_int_max;
    b->max_jobs = max_jobs;
    b->slots.resize(max_jobs);
    b->dirty = true;
    b->use_graph = o.use_graph != 0;
    b->tuning = tsne_batch_tuning{fitsne::kDefaultChunk, 0, TSNE_NINT_RULE, 0.0f};
    auto fail_free = [&](int rc) {
        tsne_batch_destroy(b);
        return rc;
    };
    cudaError_t e = cudaSuccess;
    if (o.stream) {
        b->stream = (cudaStream_t)o.stream;
    } else {
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete b; return cuda_fail(e, "stream creation"); }
        b->own_stream = true;
    }
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->table_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return fail_free(cuda_fail(e, "batch initialisation"));
    if (int rc = fitsne::fft_set_create(p * n_int_max, b->stream, &b->fft)) return fail_free(rc);
    b->tables = fitsne::Tables{b->fft.table, b->fft.tw, b->fft.of_n};
    e = cudaMalloc((void**)&b->d_table, sizeof(Job) * max_jobs);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_dyn, sizeof(JobDyn) * max_jobs);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_fill_table, sizeof(int32_t) * (n_int_max + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->kl_partial, sizeof(double) * 2 * 4 * b->sm_count);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->kl_ticket, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->kl_out, sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->region_next, sizeof(unsigned) * 1024);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_table, sizeof(Job) * max_jobs);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_dyn, sizeof(JobDyn) * max_jobs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail_free(set_error(e == cudaErrorMemoryAllocation ? TSNE_ERR_OOM : TSNE_ERR_CUDA,
                                   "batch allocation: %s", cudaGetErrorString(e)));
    }
    // the FFT lengths of the table, for the "fill" interval policy
    std::vector<fitsne::FftEntry> tab(b->fft.n_fft);
    e = cudaMemcpy(tab.data(), b->fft.table, sizeof(fitsne::FftEntry) * tab.size(), cudaMemcpyDeviceToHost);
    std::vector<int> lengths;
    for (auto& t : tab) lengths.push_back(t.L);
    const std::vector<int32_t> fill = fill_table(n_int_max, p, lengths);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_fill_table, fill.data(), sizeof(int32_t) * fill.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_dyn, 0, sizeof(JobDyn) * max_jobs, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->kl_ticket, 0, sizeof(unsigned), b->stream);
    if (e == cudaSuccess) e = fitsne::fft_configure(s, b->fft.L_max);
    if (e == cudaSuccess) {
        // the SM id range sizes the SM-local force schedule
        int* d = reinterpret_cast<int*>(b->region_next);
        e = fitsne::query_sm_id_count(d, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&b->n_regions, d, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e == cudaSuccess && (b->n_regions < 1 || b->n_regions > 1023)) b->n_regions = b->sm_count;
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->table_ev, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return fail_free(cuda_fail(e, "batch initialisation"));
    *out = b;
    return TSNE_OK;
}

int tsne_batch_destroy(tsne_batch* b) {
    if (!b) return TSNE_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (Slot& S : b->slots)
        if (S.mem) cudaFree(S.mem);
    fitsne::fft_set_destroy(&b->fft);
    void* dev[] = {b->d_table, b->d_dyn, b->d_fill_table, b->kl_partial, b->kl_ticket, b->kl_out,
                   b->region_next};
    for (void* p : dev)
        if (p) cudaFree(p);
    if (b->h_table) cudaFreeHost(b->h_table);
    if (b->h_dyn) cudaFreeHost(b->h_dyn);
    if (b->table_ev) cudaEventDestroy(b->table_ev);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return TSNE_OK;
}

int64_t tsne_batch_job_bytes(const tsne_batch* b, int64_t N) {
    if (!b || N < 2) return -1;
    return (int64_t)slot_bytes(fitsne::job_layout(N, b->s, b->p, b->n_int_max, b->fft.L_max));
}

int tsne_batch_add_job(tsne_batch* b, int64_t N, tsne_csr P, const float* Y0, int32_t n_intervals,
                       const tsne_step_params* sp, int32_t* job_id) {
    if (int rc = check_batch(b)) return rc;
    if (!job_id || !sp || !Y0) return set_error(TSNE_ERR_INVALID_ARG, "NULL argument");
    if (N < 2 || N > INT32_MAX / 2) return set_error(TSNE_ERR_INVALID_ARG, "N must be in [2, 2^30)");
    if (!P.row_ptr || (P.nnz > 0 && (!P.col || !P.val)) || P.nnz < 0 || P.nnz > INT32_MAX)
        return set_error(TSNE_ERR_INVALID_ARG, "invalid CSR");
    if (n_intervals < 0 || n_intervals > b->n_int_max)
        return set_error(TSNE_ERR_INVALID_ARG, "n_intervals %d outside [0, %d]", n_intervals, b->n_int_max);
    if (sp->n_iter < 0) return set_error(TSNE_ERR_INVALID_ARG, "n_iter < 0");
    if ((reinterpret_cast<uintptr_t>(Y0) & (b->s == 2 ? 7 : 3)) != 0)
        return set_error(TSNE_ERR_INVALID_ARG, "Y0 is not aligned");
    int id = -1;
    for (int i = 0; i < b->max_jobs; ++i)
        if (!b->slots[i].used) { id = i; break; }
    if (id < 0) return set_error(TSNE_ERR_CAPACITY, "all %d job slots are in use", b->max_jobs);
    Slot& S = b->slots[id];
    S.lay = fitsne::job_layout(N, b->s, b->p, b->n_int_max, b->fft.L_max);
    S.bytes = slot_bytes(S.lay);
    cudaError_t e = cudaMallocAsync((void**)&S.mem, S.bytes, b->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        S.mem = nullptr;
        return set_error(e == cudaErrorMemoryAllocation ? TSNE_ERR_OOM : TSNE_ERR_CUDA,
                         "job allocation (%zu bytes): %s", S.bytes, cudaGetErrorString(e));
    }
    Job& J = S.job;
    memset(&J, 0, sizeof(Job));
    fitsne::job_carve(S.lay, S.mem, true, &J);
    J.ybuf[0] = reinterpret_cast<float*>(S.mem + fitsne::job_scratch_bytes(S.lay, true));
    J.row_ptr = P.row_ptr;
    J.col = P.col;
    J.val = P.val;
    J.dyn = b->d_dyn + id;
    J.N = N;
    J.mode = fitsne::kModeStep;
    J.alpha = 1.0f;
    fitsne::job_set_schedule(&J, sp);
    J.iter_end = sp->n_iter;
    J.n_int_fixed = n_intervals;
    J.n_min = b->n_min;
    J.n_int_max = b->n_int_max;
    J.fx_shift = fitsne::fixed_point_shift(N, b->s, b->p);
    J.chunk = b->tuning.chunk;
    const int64_t ns = N * b->s;
    e = fitsne::job_zero(S.lay, J, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(J.ybuf[0], Y0, sizeof(float) * ns, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(J.uY, 0, sizeof(float) * ns, b->stream);
    if (e == cudaSuccess) e = fitsne::launch_fill(J.gains, 1.0f, ns, b->sm_count, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(J.dyn, 0, sizeof(JobDyn), b->stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(S.mem, b->stream);
        S.mem = nullptr;
        return cuda_fail(e, "job initialisation");
    }
    b->launches += 1;
    S.used = true;
    S.N = N;
    S.nnz = P.nnz;
    b->bytes_in_use += (int64_t)S.bytes;
    b->dirty = true;
    *job_id = id;
    return TSNE_OK;
}

int tsne_batch_remove_job(tsne_batch* b, int32_t id) {
    if (int rc = check_batch(b)) return rc;
    if (int rc = check_id(b, id)) return rc;
    Slot& S = b->slots[id];
    CU(cudaFreeAsync(S.mem, b->stream), "job free");
    b->bytes_in_use -= (int64_t)S.bytes;
    S = Slot{};
    b->dirty = true;
    return TSNE_OK;
}

int tsne_batch_iterate(tsne_batch* b, int32_t count) {
    if (int rc = check_batch(b)) return rc;
    if (count < 0) return set_error(TSNE_ERR_INVALID_ARG, "count < 0");
    return iterate(b, count);
}

int tsne_batch_poll(tsne_batch* b, int32_t* iter_out, int32_t* status_out) {
    if (int rc = check_batch(b)) return rc;
    CU(cudaMemcpyAsync(b->h_dyn, b->d_dyn, sizeof(JobDyn) * b->max_jobs, cudaMemcpyDeviceToHost,
                       b->stream),
       "poll read-back");
    CU(cudaStreamSynchronize(b->stream), "poll synchronise");
    for (int i = 0; i < b->max_jobs; ++i) {
        const bool u = b->slots[i].used;
        if (iter_out) iter_out[i] = u ? b->h_dyn[i].iter : -1;
        if (status_out) status_out[i] = u ? b->h_dyn[i].error : 0;
    }
    return TSNE_OK;
}

int tsne_batch_get_y(tsne_batch* b, int32_t id, float* Y_out) {
    if (int rc = check_batch(b)) return rc;
    if (int rc = check_id(b, id)) return rc;
    if (!Y_out) return set_error(TSNE_ERR_INVALID_ARG, "Y_out is NULL");
    if (b->dirty)
        if (int rc = upload_table(b)) return rc;
    const int row = table_row(b, id);
    CU(fitsne::launch_copy_current(b->d_table + row, b->slots[id].N * b->s, Y_out, b->stream),
       "copy of the current Y");
    b->launches += 1;
    return TSNE_OK;
}

int tsne_batch_kl(tsne_batch* b, int32_t id, double* kl_out) {
    if (int rc = check_batch(b)) return rc;
    if (int rc = check_id(b, id)) return rc;
    if (!kl_out) return set_error(TSNE_ERR_INVALID_ARG, "kl_out is NULL");
    if (b->dirty)
        if (int rc = upload_table(b)) return rc;
    const int row = table_row(b, id);
    const Slot& S = b->slots[id];
    // the current buffer, then Z at the current Y (the job alone, schedule ignored)
    CU(cudaMemcpyAsync(b->h_dyn + id, b->d_dyn + id, sizeof(JobDyn), cudaMemcpyDeviceToHost, b->stream),
       "state read-back");
    CU(cudaStreamSynchronize(b->stream), "state synchronise");
    const float* Y = S.job.ybuf[b->h_dyn[id].cur];
    fitsne::TableCaps c = b->caps;
    c.njobs = 1;
    c.sum_N = S.N;
    c.sum_box_items = std::min<int64_t>(fitsne::kBoxBlocks, std::max<int64_t>(1, (S.N * b->s + 1023) / 1024));
    c.sum_chunk_cap = S.N / b->tuning.chunk + std::min<int64_t>(S.N, S.lay.n_boxes_max) + 1;
    c.max_scan_items = S.lay.scan_items;
    const Job* rowp = b->d_table + row;
    CU(fitsne::launch_box(rowp, c, b->tables, 1, b->stream), "box launch");
    CU(fitsne::launch_sort_and_spread(rowp, c, b->stream), "sort/spread launch");
    CU(fitsne::launch_convolution(rowp, c, b->tables, b->stream), "FFT launch");
    const tsne_csr P{S.job.row_ptr, S.job.col, S.job.val, S.nnz};
    CU(fitsne::launch_kl_raw(P, Y, S.N, b->s, &S.job.params->Z, 0.0, b->kl_partial, b->kl_ticket,
                             b->kl_out, 4 * b->sm_count, b->stream),
       "KL launch");
    b->launches += fitsne::phase_launches(b->s) - 1;
    CU(cudaMemcpyAsync(kl_out, b->kl_out, sizeof(double), cudaMemcpyDeviceToHost, b->stream), "KL read-back");
    CU(cudaStreamSynchronize(b->stream), "KL synchronise");
    return TSNE_OK;
}

int tsne_batch_set_tuning(tsne_batch* b, const tsne_batch_tuning* t) {
    if (int rc = check_batch(b)) return rc;
    if (!t) return set_error(TSNE_ERR_INVALID_ARG, "tuning is NULL");
    const int ch = t->chunk;
    if (ch != 32 && ch != 64 && ch != 128 && ch != 256)
        return set_error(TSNE_ERR_INVALID_ARG, "chunk must be 32, 64, 128 or 256 (got %d)", ch);
    if (t->fft_threads != 0 && t->fft_threads != 256 && t->fft_threads != 512 && t->fft_threads != 1024)
        return set_error(TSNE_ERR_INVALID_ARG, "fft_threads must be 0, 256, 512 or 1024");
    if (t->n_int_policy != TSNE_NINT_RULE && t->n_int_policy != TSNE_NINT_FILL)
        return set_error(TSNE_ERR_INVALID_ARG, "unknown interval policy %d", t->n_int_policy);
    b->tuning.chunk = ch;
    b->tuning.fft_threads = t->fft_threads;
    b->tuning.n_int_policy = t->n_int_policy;
    b->dirty = true;
    return TSNE_OK;
}

int tsne_batch_get_tuning(const tsne_batch* b, tsne_batch_tuning* out) {
    if (int rc = check_batch(b)) return rc;
    if (!out) return set_error(TSNE_ERR_INVALID_ARG, "out is NULL");
    *out = b->tuning;
    return TSNE_OK;
}

int tsne_batch_autotune(tsne_batch* b, int32_t iters, tsne_batch_tuning* out) {
    if (int rc = check_batch(b)) return rc;
    if (iters < 1) return set_error(TSNE_ERR_INVALID_ARG, "iters must be >= 1");
    if (b->dirty)
        if (int rc = upload_table(b)) return rc;
    if (b->order.empty()) return set_error(TSNE_ERR_INVALID_ARG, "the batch has no jobs");
    Snapshot sn;
    if (int rc = snapshot(b, &sn, false)) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CU(cudaEventCreate(&e0), "event");
    CU(cudaEventCreate(&e1), "event");
    const tsne_batch_tuning start = b->tuning;
    int rc = TSNE_OK;
    // time of `iters` iterations from the saved state under tuning t
    auto trial = [&](const tsne_batch_tuning& t, float* ms) -> int {
        if (int r = tsne_batch_set_tuning(b, &t)) return r;
        if (int r = snapshot(b, &sn, true)) return r;
        if (int r = iterate(b, 1)) return r;  // capture and warm-up
        if (int r = snapshot(b, &sn, true)) return r;
        CU(cudaEventRecord(e0, b->stream), "event record");
        if (int r = iterate(b, iters)) return r;
        CU(cudaEventRecord(e1, b->stream), "event record");
        CU(cudaEventSynchronize(e1), "event synchronise");
        CU(cudaEventElapsedTime(ms, e0, e1), "elapsed time");
        *ms /= (float)iters;
        return TSNE_OK;
    };
    // coordinate search: spread chunk, then FFT threads. Both change only the
    // launch shapes, not a result bit; the interval policy changes the
    // arithmetic (and a run's final KL by about 1 %), so it stays the caller's.
    tsne_batch_tuning best = start;
    float best_ms = 0.0f;
    rc = trial(best, &best_ms);
    const int chunks[] = {32, 64, 128, 256};
    for (int k = 0; rc == TSNE_OK && k < 4; ++k) {
        if (chunks[k] == best.chunk) continue;
        tsne_batch_tuning t = best;
        t.chunk = chunks[k];
        float ms = 0.0f;
        rc = trial(t, &ms);
        if (rc == TSNE_OK && ms < best_ms) { best = t; best_ms = ms; }
    }
    if (b->s == 2) {
        const int thr[] = {256, 512, 1024};
        for (int k = 0; rc == TSNE_OK && k < 3; ++k) {
            tsne_batch_tuning t = best;
            t.fft_threads = thr[k];
            if (t.fft_threads == best.fft_threads) continue;
            float ms = 0.0f;
            rc = trial(t, &ms);
            if (rc == TSNE_OK && ms < best_ms) { best = t; best_ms = ms; }
        }
    }
    int rc2 = tsne_batch_set_tuning(b, rc == TSNE_OK ? &best : &start);
    if (rc == TSNE_OK) rc = rc2;
    int rc3 = snapshot(b, &sn, true);
    if (rc == TSNE_OK) rc = rc3;
    cudaFreeAsync(sn.mem, b->stream);
    cudaStreamSynchronize(b->stream);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != TSNE_OK) return rc;
    best.ms_per_iter = best_ms;
    b->tuning = best;
    if (out) *out = best;
    return TSNE_OK;
}

int64_t tsne_batch_bytes_in_use(const tsne_batch* b) { return b ? b->bytes_in_use : -1; }

int64_t tsne_batch_launch_count(const tsne_batch* b) { return b ? b->launches : 0; }

void* tsne_batch_stream(const tsne_batch* b) { return b ? (void*)b->stream : nullptr; }

}  // extern "C"
