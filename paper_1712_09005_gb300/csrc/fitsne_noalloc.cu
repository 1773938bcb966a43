// tsne_kl_noalloc: the KL reduction without any device allocation.
//
// Callers that cannot call cudaMalloc - a process whose own allocator owns
// all device memory and forbids new allocations while it serves requests, or
// code that must not let cudaMalloc/cudaFree synchronise the device in the
// middle of its work - cannot create a plan, because a plan allocates its
// scratch. This entry point computes the same quantity as tsne_kl from the
// caller's P, Y and Z, and keeps its only scratch (the per-block partial sums
// of the reduction and its completion counter) in a file-scope device array
// that the module holds from load until process exit, on every GPU that
// loads the library.
#include <stdio.h>

#include <mutex>

#include "fitsne_internal.cuh"

namespace {

constexpr int kNoAllocMaxBlocks = 1024;
constexpr size_t kNoAllocBytes = 256 + sizeof(double) * 2 * kNoAllocMaxBlocks;  // 16,640 B

// [0, 256): completion counter; [256, ...): 2 doubles per reduction block.
static __device__ __align__(256) unsigned char g_kl_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};

thread_local char g_err[256] = "";

int fail(int code, const char* msg, cudaError_t e = cudaSuccess) {
    snprintf(g_err, sizeof(g_err), "%s%s%s", msg, e != cudaSuccess ? ": " : "",
             e != cudaSuccess ? cudaGetErrorString(e) : "");
    return code;
}

// Once per device, with that device current: the device address of the
// scratch array (in host code its name is only a host-side stand-in). The
// address is kept for the life of the process: after cudaDeviceReset the
// module may be loaded again at another address, so this entry point must not
// be called on a device that the process has reset.
int setup(int dev, void** ptr, int* sms) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_kl_scratch);
        if (e != cudaSuccess) return fail(TSNE_ERR_CUDA, "cudaGetSymbolAddress of the KL scratch", e);
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return fail(TSNE_ERR_CUDA, "device query", e);
        g_sm_count[dev] = n;
        g_scratch_ptr[dev] = p;
    }
    *ptr = g_scratch_ptr[dev];
    *sms = g_sm_count[dev];
    return TSNE_OK;
}

}  // namespace

extern "C" const char* tsne_noalloc_last_error_string(void) { return g_err; }

extern "C" int tsne_kl_noalloc(tsne_csr P, const float* Y, int64_t N, int32_t s, double Z,
                               double* kl_out, void* stream) {
    g_err[0] = 0;
    if (s != 1 && s != 2) return fail(TSNE_ERR_INVALID_ARG, "s must be 1 or 2");
    if (N < 1 || N > INT32_MAX - 1) return fail(TSNE_ERR_INVALID_ARG, "N outside [1, 2^31 - 2]");
    if (P.nnz < 0 || P.nnz > INT32_MAX) return fail(TSNE_ERR_INVALID_ARG, "nnz outside [0, 2^31 - 1]");
    if (!P.row_ptr || (P.nnz > 0 && (!P.col || !P.val)) || !Y || !kl_out)
        return fail(TSNE_ERR_INVALID_ARG, "NULL pointer");
    if (!(Z > 0.0)) return fail(TSNE_ERR_INVALID_ARG, "Z must be positive");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(TSNE_ERR_CUDA, "cudaGetDevice", e);
    if (dev < 0 || dev >= kMaxDevices) return fail(TSNE_ERR_INVALID_ARG, "device index too large");
    void* base = nullptr;
    int sms = 0;
    if (int rc = setup(dev, &base, &sms)) return rc;
    int blocks = 4 * sms;
    if ((N + 7) / 8 < blocks) blocks = (int)((N + 7) / 8);
    if (blocks > kNoAllocMaxBlocks) blocks = kNoAllocMaxBlocks;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned* ticket = static_cast<unsigned*>(base);
    double* partial = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + 256);
    // the counter must start at zero whatever an earlier (possibly failed) call left
    e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return fail(TSNE_ERR_CUDA, "counter reset", e);
    e = fitsne::launch_kl_raw(P, Y, N, s, nullptr, Z, partial, ticket, kl_out, blocks, st);
    if (e != cudaSuccess) return fail(TSNE_ERR_CUDA, "KL kernel launch", e);
    return TSNE_OK;
}
