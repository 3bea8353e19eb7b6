// nedner_ned_stage_static: the NED stage (spread + x-FFT, then y-FFT) with its
// intermediate array in a fixed device buffer that is part of the library
// image, instead of the plan's workspace.  The paper has no counterpart; this
// exists for callers that must not call cudaMalloc when they run the stage.
//
// The buffer is a file-scope __device__ array of NEDNER_STATIC_SCRATCH_BYTES.
// In host code its name only stands for the symbol; the device address is
// obtained with cudaGetSymbolAddress (with that device current) on the first
// call per device and cached.  Later calls on a stream that is not being
// captured look it up again (so a device reset, after which the module is
// loaded anew, does not leave a stale address); calls on a capturing stream
// use the cached address.  The intermediate [nx/2+1][2 ny][Nt] complex64 array is
// written in full by the first kernel before the second reads it, so nothing
// in the buffer has to start at zero.  All calls share the buffer: calls that
// overlap on the GPU (other streams, other threads) race.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace {

static __device__ __align__(256) unsigned char g_ned_static_scratch[NEDNER_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 256;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the static buffer on the current device.  Looked up on
// the first call per device and whenever the stream is not being captured;
// during a capture the cached address is used (and a capture without one is
// refused).
cudaError_t scratch_address(cudaStream_t s, void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_ned_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    } else if (!g_scratch_addr[dev]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" nedner_status nedner_ned_stage_static(nedner_plan_t p, const float* g, void* Ghat, void* stream) {
    if (!p || !Ghat || (p->M > 0 && !g)) return NEDNER_EINVAL;
    if (((uintptr_t)g & 15) != 0 || ((uintptr_t)Ghat & 15) != 0) return NEDNER_EINVAL;
    if (p->tp.enabled) return NEDNER_EINVAL;          // tensor-product plans: see nedner.h
    const nedner::Geo& G = p->geo;
    const size_t need = (size_t)G.nxh * G.Ly * G.Nt * sizeof(float2);
    if (need > (size_t)NEDNER_STATIC_SCRATCH_BYTES) return NEDNER_ENOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    void* scratch = nullptr;
    if (scratch_address(s, &scratch) != cudaSuccess) return NEDNER_ECUDA;
    float2* R = (float2*)scratch;
    if (nedner::launch_ned_spread_xfft(*p, g, R, s) != cudaSuccess) return NEDNER_ECUDA;
    if (nedner::launch_ned_yfft(*p, R, (float2*)Ghat, s) != cudaSuccess) return NEDNER_ECUDA;
    return NEDNER_OK;
}
