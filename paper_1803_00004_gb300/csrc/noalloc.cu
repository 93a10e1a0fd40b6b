// bf_filter_noalloc: bf_filter for callers that must not allocate device
// memory while filtering.
//
// Some hosts reserve all the device memory they will use at start-up: for
// example a framework whose caching allocator owns the GPU's memory, or a
// real-time loop where an allocation may block on device synchronisation or
// fail under memory pressure in the middle of a frame.  bf_filter allocates
// (stream-ordered) scratch for the partial numerator / denominator planes of
// plans whose cosine terms are split into groups, and for the 3-D form's
// slice work list; this entry point instead uses a fixed array that is part
// of the library's device image.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds its kScratchBytes until the process exits.  Host code cannot
// use the array's name as a device address, so the address is looked up with
// cudaGetSymbolAddress, with the device current, and passed to the kernels as
// a plain pointer.  The look-up is done once per CUDA context (keyed by the
// context's unique id, so a context torn down by cudaDeviceReset and created
// again gets a fresh look-up): the first call in a context does it, and that
// first call should come before any stream capture.
//
// Every call shares the one array and it keeps the previous call's contents.
// Nothing needs clearing beyond the 3-D form's two work-list counters, which
// each call zeroes on its stream: every partial-plane element the finalize
// pass reads is written earlier in the same call.  Calls whose work overlaps
// on the GPU (different streams, or different host threads) race on the
// array; order them on one stream or with events, and consume a call's
// output before a later call's work can start.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "bf_internal.h"

namespace bfi {
bool debug_range_checks();
bf_status count_out_of_range(const float *d_in, size_t in_pitch_elems, int h, int w, float lo, float hi, void *stream,
                             unsigned long long *count);
}  // namespace bfi

namespace {

constexpr size_t kScratchBytes = 64u << 20;  // 64 MiB = 16,777,216 floats

__device__ __align__(256) float g_scratch[kScratchBytes / sizeof(float)];

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

std::mutex g_mu;
struct Cached {
    unsigned long long ctx_id;
    float *addr;
};
std::vector<Cached> g_cache;  // one entry per context seen

// Unique id of the current context (0 when the driver cannot tell).
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of g_scratch in the current context (the plan's device is current).
bf_status scratch_address(float **out) {
    // (the caller's device buffers imply a current context; without one the id is 0 and the address is
    // looked up on every call)
    const unsigned long long id = current_context_id();
    std::lock_guard<std::mutex> lk(g_mu);
    if (id != 0)
        for (const Cached &c : g_cache)
            if (c.ctx_id == id) {
                *out = c.addr;
                return BF_OK;
            }
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return bfi::fail(BF_ERR_CUDA, std::string("scratch symbol address: ") + cudaGetErrorString(e));
    }
    if (id != 0) g_cache.push_back(Cached{id, static_cast<float *>(p)});  // id 0: look it up on every call
    *out = static_cast<float *>(p);
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
    // the debug input-range check of bf_filter (its counter is a __device__ variable: no allocation)
    if (bfi::debug_range_checks()) {
        unsigned long long n = 0;
        st = bfi::count_out_of_range(d_in, in_pitch / sizeof(float), height, width, plan->desc.i_lo, plan->desc.i_hi,
                                     stream, &n);
        if (st == BF_OK && n > 0)
            st = bfi::fail(BF_ERR_RANGE, std::to_string(n) + " input pixels outside [i_lo, i_hi] (range check on)");
        if (st != BF_OK) {
            if (prev != device) cudaSetDevice(prev);
            return st;
        }
    }
    // the geometry bf_filter would use, else the best-ranked of all geometries whose scratch fits the array
    bfi::TileConfig tc = bfi::choose_tile(plan->kp, height, width, plan->desc.precision);
    if (bfi::scratch_bytes(tc, height, width, plan->kp.zbins) > kScratchBytes) {
        tc.ncols = 0;
        for (const auto &c : bfi::tile_candidates(plan->kp, height, width, plan->desc.precision, 1 << 20))
            if (bfi::scratch_bytes(c, height, width, plan->kp.zbins) <= kScratchBytes) {
                tc = c;
                break;
            }
    }
    if (tc.ncols == 0) {
        st = bfi::fail(BF_ERR_SCRATCH, "no launch geometry's scratch (partial planes: 2 x term groups x height x "
                                       "width floats; 3-D form: also its slice list) fits the fixed 64 MiB array; "
                                       "use bf_filter");
    } else {
        float *scratch = nullptr;
        st = bfi::scratch_bytes(tc, height, width, plan->kp.zbins) ? scratch_address(&scratch) : BF_OK;
        if (st == BF_OK)
            st = bfi::launch_filter(plan->kp, plan->desc.precision, plan->desc.kahan, tc, d_in, in_pitch / sizeof(float),
                                    d_out, out_pitch / sizeof(float), scratch, height, width, stream);
    }
    if (prev != device) cudaSetDevice(prev);
    return st;
}
