// es_gather_noalloc: es_gather without any device allocation.
//
// es_gather stages the requested cell indices and the gathered values in a
// device buffer that it allocates on its first use (cudaMalloc, or the
// context's allocator hook).  Some callers must not allocate device memory
// when they read values back: a real-time loop that cannot wait on an
// allocator, or an embedding application that hands out all device memory up
// front and fails any later request.  This variant stages through a fixed
// array that lives in the library's own device memory instead.
//
// The array holds ES_GATHER_NOALLOC_MAX cells: 4,096 int64 indices followed
// by 19 x 4,096 doubles, 640 KiB.  Every GPU that loads the library keeps it
// until the process exits.  All calls share it and it keeps the contents of
// the last call; nothing in it has to start at zero, because every call
// writes the indices it uses and every value it returns.  Calls whose GPU
// work overlaps (two streams, or two host threads) race on it.  The call
// copies the indices from pageable host memory and waits for the context's
// stream, like es_gather.
#include <mutex>

#include "es_internal.cuh"

namespace {

constexpr int kMaxCells = ES_GATHER_NOALLOC_MAX;
constexpr size_t kIndexBytes = (size_t)kMaxCells * 8;
constexpr size_t kScratchBytes = kIndexBytes + (size_t)19 * kMaxCells * 8;
constexpr int kMaxDevices = 64;

// The scratch array.  In host code this name is only a stand-in for the
// symbol, not a device address: its address on a device comes from
// cudaGetSymbolAddress, taken once per device with that device current.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices];

// Device address of g_scratch on device `dev`, which must be current
// (looked up on the first call on that device).
cudaError_t scratch_address(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int es_gather_noalloc(es_ctx* c, int which, const int64_t* idx, int n, double* out) {
    const int rc = es::check_gather_args(c, which, idx, n, kMaxCells, out);
    if (rc != ES_OK) return rc;
    // (the array's address is that of the context's device, which must be
    // current: the context's stream and kernels belong to it)
    int cur = 0;
    cudaError_t e = cudaGetDevice(&cur);
    if (e == cudaSuccess && cur != c->device) {
        c->err = "the current CUDA device is not the context's device";
        return ES_EINVAL;
    }
    void* base = nullptr;
    if (e == cudaSuccess) e = scratch_address(c->device, &base);
    if (e == cudaSuccess) {
        long long* didx = (long long*)base;
        double* dval = (double*)((unsigned char*)base + kIndexBytes);
        e = cudaMemcpyAsync(didx, idx, (size_t)n * 8, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = es::launch_gather(c, which, didx, n, dval);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out, dval, (size_t)es::field_components(which) * n * 8, cudaMemcpyDeviceToHost,
                                c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (e != cudaSuccess) {
        c->err = cudaGetErrorString(e);
        return ES_ECUDA;
    }
    return ES_OK;
}
