// es_noalloc.cu -- es_gather_noalloc: es_gather without any device allocation.
//
// es_gather stages the requested cell indices and the gathered values in a
// device buffer that it allocates on its first use (cudaMalloc, or the
// context's allocator hook).  Some callers cannot allocate at that moment: a
// thread that is capturing CUDA work into a graph (cudaMalloc is not allowed
// during stream capture), a real-time loop that must not stall on the
// allocator, or an embedding application that hands out all device memory up
// front.  This variant stages through a fixed array that lives in the
// library's own device memory instead.
//
// The array holds ES_GATHER_NOALLOC_MAX cells: 4,096 int64 indices followed
// by 19 x 4,096 doubles, 640 KiB.  Every GPU that loads the library keeps it
// until the process exits.  All calls share it and it keeps the contents of
// the last call; nothing in it has to start at zero, because every call
// writes the indices it uses and every value it returns.  Calls whose GPU
// work overlaps (two streams, or two host threads) race on it.
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

// Device address of g_scratch on the current device (set up on first use).
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

int components(int which) {
    if (which == ES_FIELD_PDF || which == ES_FIELD_PDF_LAST) return 19;
    if (which == ES_FIELD_U || which == ES_FIELD_FB) return 3;
    return 1;
}

}  // namespace

extern "C" int es_gather_noalloc(es_ctx* c, int which, const int64_t* idx, int n, double* out) {
    if (!c || !idx || !out) return ES_EINVAL;
    if (n < 1 || n > kMaxCells) {
        c->err = "n must be in 1..4096 (ES_GATHER_NOALLOC_MAX)";
        return ES_EINVAL;
    }
    if (which < ES_FIELD_PSI || which > ES_FIELD_PDF_LAST) {
        c->err = "unknown field";
        return ES_EINVAL;
    }
    if (which == ES_FIELD_PDF_LAST && c->last_src < 0) {
        c->err = "no LBM step yet";
        return ES_EINVAL;
    }
    for (int i = 0; i < n; i++)
        if (idx[i] < 0 || idx[i] >= c->g.N) {
            c->err = "cell index out of range";
            return ES_EINVAL;
        }
    void* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e == cudaSuccess) {
        long long* didx = (long long*)base;
        double* dval = (double*)((unsigned char*)base + kIndexBytes);
        e = cudaMemcpyAsync(didx, idx, (size_t)n * 8, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = es::launch_gather(c, which, didx, n, dval);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out, dval, (size_t)components(which) * n * 8, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (e != cudaSuccess) {
        c->err = cudaGetErrorString(e);
        return ES_ECUDA;
    }
    return ES_OK;
}
