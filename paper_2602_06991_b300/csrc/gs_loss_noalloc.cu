// gs_loss_noalloc.cu -- gs_loss_cos_l1_noalloc: the training loss without any
// caller-provided scratch.
//
// Who needs this: callers that cannot allocate device memory themselves.  Examples are
// code in a real-time loop, where cudaMalloc/cudaFree may synchronise the device and
// take milliseconds; a plug-in running inside a host framework that owns all device
// memory through its own pool and forbids raw allocations; and a component that is
// handed only its input and output buffers.  The regular gs_loss_cos_l1 needs a
// scratch buffer of gs_loss_scratch_size(n_pix) bytes for the per-pixel partial sums
// of the loss.  This variant keeps those partial sums in a fixed array that the library
// itself holds: a file-scope __device__ array of GS_LOSS_NOALLOC_MAX_PIX + 360 floats
// (about 16.8 MB) on every GPU that loads the library, kept until the process exits.
//
// Rules for callers:
//   - n_pix above GS_LOSS_NOALLOC_MAX_PIX is rejected with GS_ERR_WORKSPACE before
//     anything is launched;
//   - the first call on a device looks up the array's device address (the set-up for
//     that device, done with that device current); make that first call before any
//     stream capture.  Every later call made outside a capture looks the address up
//     again (it is only valid for the device's current context, so after a
//     cudaDeviceReset the next such call finds the array's new address); a call made
//     while its stream is being captured reuses the address found last;
//   - every call shares the one array, so calls whose kernels overlap on the GPU (on
//     different streams, or from different host threads without ordering) race on it;
//   - nothing has to start at zero: each call writes every element it later reads.
// Nothing here calls cudaMalloc, cudaFree or any allocating routine.
#include "gs_internal.cuh"

#include <mutex>

namespace gs {

constexpr long long kNoallocScratchFloats = (long long)GS_LOSS_NOALLOC_MAX_PIX + kSortBlocks + 64;

// The array's name is only a host-side stand-in in host code; kernels get the address
// returned by cudaGetSymbolAddress for the current device.
static __device__ __align__(256) float g_loss_scratch[kNoallocScratchFloats];

constexpr int kMaxDevices = 64;
static std::mutex g_scratch_mu;
static float *g_scratch_ptr[kMaxDevices];

// Device address of g_loss_scratch on the current device: looked up on every call made
// outside a stream capture (the address belongs to the device's current context), and
// the last one found is reused while `s` is being captured.  A failed lookup leaves no
// CUDA error pending for the next call.
static int noalloc_scratch(cudaStream_t s, float **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GS_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return GS_ERR_UNSUPPORTED;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return GS_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (cs == cudaStreamCaptureStatusNone || !g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_loss_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return GS_ERR_CUDA;
        }
        g_scratch_ptr[dev] = (float *)p;
    }
    *out = g_scratch_ptr[dev];
    return GS_OK;
}

}  // namespace gs

using namespace gs;

extern "C" int gs_loss_cos_l1_noalloc(const gs_config *cfg, int64_t n_pix, const void *F, const void *F_gt,
                                      const float *rgb, const float *rgb_gt, const float *depth,
                                      const float *depth_gt, float w_feat, float w_rgb, float w_depth, void *dL_dF,
                                      float *dL_dC, float *dL_dD, float *loss, void *stream)
{
    // the same argument rules as gs_loss_cos_l1
    if (!cfg_ok(cfg) || n_pix < 1) return GS_ERR_ARG;
    if (!F || !F_gt || !rgb || !rgb_gt || !depth || !depth_gt || !dL_dF || !dL_dC || !dL_dD || !loss)
        return GS_ERR_ARG;
    if (((uintptr_t)F & 15) || ((uintptr_t)F_gt & 15) || ((uintptr_t)dL_dF & 15)) return GS_ERR_ARG;
    if (n_pix > (int64_t)GS_LOSS_NOALLOC_MAX_PIX) return GS_ERR_WORKSPACE;
    float *part = nullptr;
    int st = noalloc_scratch((cudaStream_t)stream, &part);
    if (st != GS_OK) return st;
    launch_loss(cfg->feat_dtype, cfg->D, n_pix, F, F_gt, rgb, rgb_gt, depth, depth_gt, w_feat, w_rgb, w_depth, dL_dF,
                dL_dC, dL_dD, loss, part, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}
