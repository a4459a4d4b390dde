// An entry point for callers that cannot allocate device memory.
//
// Every other entry point takes a caller-provided workspace.  Some callers have
// no way to provide one: a plain C host that links this library but owns no
// device allocator, or code whose device memory is owned by another runtime, or a
// thread that must not make the blocking, device-wide synchronising cudaMalloc
// call.  hawkes_loglik_grad_static serves them from a fixed scratch array that is
// part of the library image itself, so neither the caller nor the library
// allocates anything at call time.
//
// The scratch array is a file-scope __device__ array of kStaticScratchBytes;
// every GPU that loads the library holds it until the process exits.  The first
// call on a device looks up the array's device address with cudaGetSymbolAddress
// (once per device, with that device current) and caches it; make that first call
// before any stream capture.  All calls share the array: they are correct one at a
// time, but calls that overlap on the GPU (other streams, other host threads)
// race on it.  Every region the kernels read is written or zeroed by the same
// call first, so contents left by the previous call do not matter.
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kStaticScratchBytes = 16u << 20;   // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_lock;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device (nullptr on error).
void* scratch_for_current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess) return nullptr;
        g_scratch_ptr[dev] = p;
    }
    return g_scratch_ptr[dev];
}

}  // namespace

extern "C" {

size_t hawkes_static_scratch_bytes(void) { return kStaticScratchBytes; }

hawkes_status hawkes_loglik_grad_static(const double* t, const int32_t* c, int64_t N, double T,
                                        int32_t M, const float* mu, const float* alpha,
                                        const float* beta, const hawkes_opts* opts,
                                        double* out_ll, float* d_mu, float* d_alpha,
                                        float* d_beta, void* stream) {
    // the same checks, in the same order, as hawkes_loglik_grad: a call that one rejects,
    // the other rejects with the same status; only then the size of the scratch array
    const int rc = hk::check_single_args(t, c, N, T, M, mu, alpha, beta, opts, out_ll, d_mu,
                                         d_alpha, d_beta, 1);
    if (rc) return (hawkes_status)rc;
    const size_t need = hawkes_workspace_size(N, M, 1, 1, opts);
    if (need == 0) return HAWKES_ERR_UNSUPPORTED;
    if (need > kStaticScratchBytes) return HAWKES_ERR_WORKSPACE;   // problem too large
    void* ws = scratch_for_current_device();
    if (!ws) return HAWKES_ERR_CUDA;
    return hawkes_loglik_grad(t, c, N, T, M, mu, alpha, beta, opts, ws, kStaticScratchBytes,
                              out_ll, d_mu, d_alpha, d_beta, stream);
}

}  // extern "C"
