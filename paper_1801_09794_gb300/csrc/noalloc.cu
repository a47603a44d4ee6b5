// Allocation-free Gram product G = Q^H Q (feast_nl_gram_noalloc).
//
// The split-K GEMM that forms Gram and projection matrices elsewhere in the
// library takes its partial sums from handle-owned device memory.  This entry
// point runs the same kernels with the partial sums in a fixed, file-scope
// device array instead, so a caller that must not touch the CUDA allocator
// (its device memory is owned by another framework's pool, or it runs in a
// latency-critical loop where cudaMalloc/cudaFree would stall or synchronise
// the device) can still form Gram matrices of device-resident blocks.
#include "../../include/feast_nl.h"
#include "internal.h"

#include <mutex>

using namespace fnl;

namespace {

// Split-K partial sums: 262144 complex128 = 4 MiB, held by every GPU that loads
// the library until the process exits.
constexpr int64_t kScratchElems = 262144;
__device__ __align__(256) double2 g_gram_scratch[kScratchElems];

// Column stride cap: (m - 1) * ldq stays far inside int64 for every m <= 512.
constexpr int64_t kMaxLd = (int64_t)1 << 40;

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Device address of the scratch array for the current device, looked up once
// per device (with that device current) and cached.
cudaError_t scratch_for_current_device(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_gram_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// True when p is device memory of device dev, or managed memory (reachable from
// every device).  Device memory of another GPU is rejected: the kernel runs on
// the current device and would otherwise touch a peer's memory.
bool on_device(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

int bad(int code, const char* msg) {
    set_last_error(msg);
    return code;
}

}  // namespace

extern "C" int feast_nl_gram_noalloc(int64_t n, int32_t m, const void* Q, int64_t ldq, void* G,
                                     void* stream) {
    if (n < 1 || m < 1) return bad(FEAST_NL_EINVAL, "n and m must be positive");
    if ((int64_t)m * m > kScratchElems)
        return bad(FEAST_NL_EINVAL, "m*m exceeds the 262144-element static scratch (m <= 512)");
    if (n > (int64_t)1 << 30 || ldq < n) return bad(FEAST_NL_EINVAL, "need n <= 2^30 and ldq >= n");
    if (ldq > kMaxLd) return bad(FEAST_NL_EINVAL, "ldq exceeds 2^40 elements");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return bad(FEAST_NL_EDEVICE, "no current CUDA device");
    }
    if (!Q || !G || !on_device(Q, dev) || !on_device(G, dev))
        return bad(FEAST_NL_EINVAL, "Q and G must be device (or managed) memory of the current device");
    void* scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) return bad(FEAST_NL_EDEVICE, "cudaGetSymbolAddress of the scratch failed");
    // as many k-splits as the scratch holds (and the GPU can use)
    int64_t fit = kScratchElems / ((int64_t)m * m);
    int64_t tiles = ((m + 63) / 64) * ((m + 63) / 64);
    int64_t want = 304 / tiles;
    int64_t splits = fit < want ? fit : want;
    if (splits > n / 16) splits = n / 16;
    if (splits < 1) splits = 1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    e = gemm_splitk_d(st, 1, m, m, (int)n, make_double2(1.0, 0.0),
                      static_cast<const double2*>(Q), ldq, static_cast<const double2*>(Q), ldq,
                      make_double2(0.0, 0.0), static_cast<double2*>(G), m,
                      static_cast<double2*>(scratch), (int)splits);
    if (e != cudaSuccess) return bad(FEAST_NL_EDEVICE, cudaGetErrorString(e));
    return FEAST_NL_OK;
}
