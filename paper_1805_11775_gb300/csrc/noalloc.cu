// noalloc.cu -- hos_bispectrum_noalloc: the bispectrum for callers that cannot
// allocate device memory.
//
// Some callers have no way to obtain device memory for the workspace the other
// entry points need: code that runs where cudaMalloc is forbidden or unsafe
// (inside a host callback or a real-time loop that must not block on the
// allocator), plug-ins that live inside a host application which owns every
// allocation, or programs that have no PyTorch (or other allocator) at hand.
// For them this entry point runs the same bispectrum computation with its
// scratch in a fixed array that is part of the library itself.
//
// The array is a file-scope __device__ variable, so each GPU that loads the
// library reserves HOS_NOALLOC_SCRATCH_BYTES of device memory for it until the
// process exits.  No call here allocates or frees anything.
#include <mutex>

#include "launch.cuh"

namespace {

static __device__ __align__(256) uint8_t g_noalloc_scratch[HOS_NOALLOC_SCRATCH_BYTES];

// Host code cannot use g_noalloc_scratch as an address (on the host it names a
// stand-in object, not device memory), so its device address is looked up with
// cudaGetSymbolAddress while the device is current: once per device, and again
// whenever the device's context has changed (after a device reset the module is
// loaded anew and the array may sit elsewhere).
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_addr[MAX_DEVICES] = {nullptr};
uint64_t g_ctx[MAX_DEVICES] = {0};  // context the address was looked up in (~0: unknown)

hos_status scratch_for_current_device(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return HOS_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    // 0: no context current yet (the lookup below makes the device's primary
    // context current) or the driver cannot say
    const uint64_t ctx = hos::current_context_id();
    if (g_addr[dev] == nullptr || (ctx != 0 && g_ctx[dev] != ctx)) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return HOS_ERR_CUDA;
        const uint64_t now = hos::current_context_id();
        g_addr[dev] = p;
        g_ctx[dev] = now ? now : ~0ull;
    }
    *out = g_addr[dev];
    return HOS_OK;
}

}  // namespace

extern "C" hos_status hos_bispectrum_noalloc(const void* d_x, int32_t dtype, int64_t n, const hos_params* params,
                                             void* d_B, hos_stream_t stream) {
    if (!d_x || !d_B || n < 1 || !params || (dtype != HOS_F32 && dtype != HOS_F64)) return HOS_ERR_INVALID_ARG;
    size_t need = 0;
    hos_status s = hos_workspace_size(HOS_OP_BISPECTRUM, n, 1, n, params, &need);
    if (s != HOS_OK) return s;
    if (need > (size_t)HOS_NOALLOC_SCRATCH_BYTES) return HOS_ERR_WORKSPACE;  // problem too large for the fixed array
    void* ws = nullptr;
    s = scratch_for_current_device(&ws);
    if (s != HOS_OK) return s;
    // The array keeps whatever the previous call left.  Every region the
    // computation reads is written earlier in the same call, except the device
    // status word, which is sticky: clear it so that this call reports only
    // its own device-side failures.
    if (cudaMemsetAsync(ws, 0, 256, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) return HOS_ERR_CUDA;
    return hos_bispectrum(d_x, dtype, n, params, d_B, ws, (size_t)HOS_NOALLOC_SCRATCH_BYTES, stream);
}

extern "C" hos_status hos_bispectrum_noalloc_status(int32_t* status) {
    if (!status) return HOS_ERR_INVALID_ARG;
    void* ws = nullptr;
    hos_status s = scratch_for_current_device(&ws);
    if (s != HOS_OK) return s;
    return hos_get_device_status(ws, status);
}
