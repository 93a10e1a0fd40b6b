// bf_filter_noalloc: bf_filter for callers that must not allocate device
// memory while filtering.
//
// Some hosts reserve all the device memory they will use at start-up: for
// example a framework whose caching allocator owns the GPU's memory, or a
// real-time loop where an allocation may block on device synchronisation or
// fail under memory pressure in the middle of a frame.  bf_filter allocates
// (stream-ordered) scratch for the partial numerator / denominator planes of
// plans whose cosine terms are split into groups; this entry point instead
// uses a fixed array that is part of the library's device image.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds its kScratchBytes until the process exits.  Host code cannot
// use the array's name as a device address, so the address is looked up once
// per device with cudaGetSymbolAddress (with that device current) and passed
// to the kernels as a plain pointer.  The first call on a device does this
// look-up; make that first call before any stream capture.
//
// Every call shares the one array and it keeps the previous call's contents.
// Nothing needs clearing: each partial plane element the finalize pass reads
// is written earlier in the same call.  Calls whose work overlaps on the GPU
// (different streams, or different host threads) race on the array; order
// them on one stream or with events.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "bf_internal.h"

namespace {

constexpr size_t kScratchBytes = 64u << 20;  // 64 MiB = 16,777,216 floats
constexpr int kMaxDevices = 64;

__device__ __align__(256) float g_scratch[kScratchBytes / sizeof(float)];

std::mutex g_mu;
float *g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device).
bf_status scratch_address(int device, float **out) {
    if (device < 0 || device >= kMaxDevices) return bfi::fail(BF_ERR_NO_DEVICE, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return bfi::fail(BF_ERR_CUDA, std::string("scratch symbol address: ") + cudaGetErrorString(e));
        }
        g_scratch_addr[device] = static_cast<float *>(p);
    }
    *out = g_scratch_addr[device];
    return BF_OK;
}

}  // namespace

extern "C" bf_status bf_filter_noalloc(const bf_plan *plan, const float *d_in, size_t in_pitch, float *d_out,
                                       size_t out_pitch, int height, int width, void *stream) {
    if (!plan) return bfi::fail(BF_ERR_INVALID_ARG, "NULL plan");
    bf_status st = bfi::check_image(d_in, in_pitch, d_out, out_pitch, height, width);
    if (st != BF_OK || height == 0 || width == 0) return st;
    if (plan->desc.device < 0) return bfi::fail(BF_ERR_NO_DEVICE, "host-only plan (device = -1)");
    const int device = plan->desc.device;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || (prev != device && cudaSetDevice(device) != cudaSuccess)) {
        cudaGetLastError();
        return bfi::fail(BF_ERR_NO_DEVICE, "cannot select the plan's device");
    }
    // the geometry bf_filter would use, else the best-ranked one whose planes fit the array
    bfi::TileConfig tc = bfi::choose_tile(plan->kp, height, width, plan->desc.precision);
    if (bfi::scratch_bytes(tc, height, width, plan->kp.zbins) > kScratchBytes) {
        tc.ncols = 0;
        for (const auto &c : bfi::tile_candidates(plan->kp, height, width, plan->desc.precision, 64))
            if (bfi::scratch_bytes(c, height, width, plan->kp.zbins) <= kScratchBytes) {
                tc = c;
                break;
            }
    }
    if (tc.ncols == 0) {
        st = bfi::fail(BF_ERR_RANGE, "image needs more than the fixed 64 MiB scratch (2 x term groups x height x "
                                     "width floats); use bf_filter");
    } else {
        float *scratch = nullptr;
        st = bfi::scratch_bytes(tc, height, width, plan->kp.zbins) ? scratch_address(device, &scratch) : BF_OK;
        if (st == BF_OK)
            st = bfi::launch_filter(plan->kp, plan->desc.precision, plan->desc.kahan, tc, d_in, in_pitch / sizeof(float),
                                    d_out, out_pitch / sizeof(float), scratch, height, width, stream);
    }
    if (prev != device) cudaSetDevice(prev);
    return st;
}
