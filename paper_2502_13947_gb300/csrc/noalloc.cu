// noalloc.cu -- icd2s_apply_flips_static: the flip write-back on buffers the
// caller owns, with no device allocation by the library.
//
// Who needs it: callers that cannot call cudaMalloc -- code whose device
// memory is handed out by someone else (a host framework that owns the whole
// budget and forbids foreign allocations, a plugin living inside another
// process's allocator), or a service that must not allocate once it is
// running.  Everything else in the library allocates scratch inside its
// handles; this entry point instead keeps its scratch (flip lists, per-replica
// counters, the diagonal of Q) in one file-scope static device array of
// kStaticScratchBytes, which every GPU that loads the library holds until the
// process exits.
//
// Set-up: a call that is not being captured into a CUDA graph looks up the
// device address of the array (cudaGetSymbolAddress) in the current context
// of the current device and caches it per device; a captured call uses the
// cached address, so the first call on a device, and the first after a device
// reset or a change of context, must be made outside stream capture.  Every call on a
// device shares the same array, and the array keeps the last call's contents,
// so each call clears the counters it needs at zero; calls whose work
// overlaps on the GPU (different streams, no ordering between them) race on
// the array and must be serialised by the caller.
#include <cstdio>
#include <mutex>

#include "../../include/icd2s.h"
#include "common.cuh"

namespace icd2s {

namespace {

constexpr int kStaticMaxListEntries = 1 << 20;  // replicas * ld flip-list entries (4 MiB)
constexpr int kStaticMaxReplicas = kMaxReplicas;
constexpr int kStaticMaxLd = kMaxN + kLdAlign;
constexpr size_t kOffFL = 0;
constexpr size_t kOffFCNT = kOffFL + sizeof(int32_t) * (size_t)kStaticMaxListEntries;
constexpr size_t kOffDEACC = kOffFCNT + sizeof(int32_t) * (size_t)kStaticMaxReplicas;
constexpr size_t kOffDONE = kOffDEACC + sizeof(unsigned long long) * (size_t)kStaticMaxReplicas;
constexpr size_t kOffDIAG = kOffDONE + sizeof(unsigned int) * (size_t)kStaticMaxReplicas;
constexpr size_t kStaticScratchBytes = kOffDIAG + sizeof(int32_t) * (size_t)kStaticMaxLd;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {};

__global__ void k_diag_static(const int8_t* __restrict__ Q, int n, int ld, int32_t* __restrict__ diag)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) diag[j] = Q[(size_t)j * ld + j];
}

thread_local char g_err_static[256] = "";

}  // namespace
}  // namespace icd2s

using namespace icd2s;

extern "C" int icd2s_apply_flips_static(const int8_t* Q_dev, int32_t n, int32_t ld, int32_t replicas,
                                        const uint8_t* flips_dev, uint8_t* x_dev, int32_t* g_dev, int64_t* E_dev,
                                        void* stream)
{
    // argument checks (the same thread-local message mechanism as the rest of the ABI)
    auto bad = [](int code, const char* msg) {
        set_error_message(msg);
        return code;
    };
    if (!Q_dev || !flips_dev || !x_dev || !g_dev || !E_dev) return bad(ICD2S_ERR_ARG, "apply_flips_static: NULL pointer");
    if (n < 1 || n > kMaxN) return bad(ICD2S_ERR_RANGE, "apply_flips_static: n outside 1..16384");
    if (ld < n || ld % 4 != 0 || ld > kStaticMaxLd)
        return bad(ICD2S_ERR_ARG, "apply_flips_static: ld must be a multiple of 4 with n <= ld <= 16512");
    if (replicas < 1 || replicas > kStaticMaxReplicas)
        return bad(ICD2S_ERR_RANGE, "apply_flips_static: replicas outside 1..4096");
    if ((long long)replicas * ld > kStaticMaxListEntries)
        return bad(ICD2S_ERR_RANGE, "apply_flips_static: replicas * ld exceeds the static scratch (1048576 entries)");
    if (((uintptr_t)Q_dev & 3) || ((uintptr_t)x_dev & 3) || ((uintptr_t)g_dev & 15) || ((uintptr_t)E_dev & 7))
        return bad(ICD2S_ERR_ARG, "apply_flips_static: Q and x must be 4-byte, g 16-byte, E 8-byte aligned");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return bad(ICD2S_ERR_CUDA, "apply_flips_static: cudaGetDevice failed");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // The array's device address belongs to the device's current context: a
    // device reset or another context on the same device can move it.  Outside
    // stream capture every call therefore looks it up again (a host-side table
    // lookup) and refreshes the cache; inside a capture, where the lookup may
    // not be allowed, the address cached by an earlier uncaptured call is used.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();  // clear the query's error so the launches below report their own
        cap = cudaStreamCaptureStatusActive;
    }
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (cap == cudaStreamCaptureStatusNone) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess || !p) {
                snprintf(g_err_static, sizeof g_err_static, "apply_flips_static: cudaGetSymbolAddress failed: %s",
                         cudaGetErrorString(e));
                return bad(ICD2S_ERR_CUDA, g_err_static);
            }
            g_scratch_addr[dev] = static_cast<unsigned char*>(p);
        } else if (!g_scratch_addr[dev]) {
            return bad(ICD2S_ERR_CUDA, "apply_flips_static: first call on this device made during stream capture");
        }
        base = g_scratch_addr[dev];
    }
    Dev d{};
    d.Q = Q_dev; d.n = n; d.ld = ld; d.R = replicas;
    d.diag = reinterpret_cast<int32_t*>(base + kOffDIAG);
    d.X = x_dev; d.G = g_dev; d.E = E_dev;
    d.FL = reinterpret_cast<int32_t*>(base + kOffFL);
    d.FCNT = reinterpret_cast<int32_t*>(base + kOffFCNT);
    d.DEACC = reinterpret_cast<unsigned long long*>(base + kOffDEACC);
    d.DONE = reinterpret_cast<unsigned int*>(base + kOffDONE);
    // the array keeps the previous call's contents: clear the counters that must start at zero
    if ((e = cudaMemsetAsync(d.FCNT, 0, sizeof(int32_t) * replicas, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(d.DEACC, 0, sizeof(unsigned long long) * replicas, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(d.DONE, 0, sizeof(unsigned int) * replicas, s)) != cudaSuccess)
        return bad(ICD2S_ERR_CUDA, "apply_flips_static: cudaMemsetAsync failed");
    k_diag_static<<<(n + 255) / 256, 256, 0, s>>>(Q_dev, n, ld, const_cast<int32_t*>(d.diag));
    if ((e = cudaGetLastError()) != cudaSuccess) return bad(ICD2S_ERR_CUDA, "apply_flips_static: launch failed");
    note_launch(1);
    if ((e = launch_compact_mask(d, flips_dev, n, s)) != cudaSuccess ||
        (e = launch_apply(d, s)) != cudaSuccess)
        return bad(ICD2S_ERR_CUDA, "apply_flips_static: launch failed");
    return ICD2S_OK;
}
