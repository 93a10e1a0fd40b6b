// bf_filter_host: the filter for images in host memory.  One call uploads the
// image, filters it with each of n plans (the paper's use of one image under
// several parameter settings, Sec. V-C) on internal compute streams, and
// downloads each result as soon as its filter ends.  Device buffers (the
// input, n outputs and each plan's scratch) come from one block per device,
// allocated on first use and grown when a call needs more, so steady-state
// calls allocate nothing.  Calls on a device are chained on the device by an
// event (each call's upload waits for the previous call's last download), so
// the shared block is never used by two calls at once.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "bf_internal.h"

namespace bfi {
bf_status filter_image(const bf_plan *plan, const TileConfig &tc, const float *d_in, size_t in_pitch, float *d_out,
                       size_t out_pitch, int h, int w, float *d_scratch, void *stream);
}  // namespace bfi

namespace {

constexpr int kMaxStreams = 8;
constexpr int kMaxDevices = 64;

struct DeviceState {
    std::mutex mu;
    char *block = nullptr;
    size_t bytes = 0;
    cudaStream_t streams[kMaxStreams] = {};
    cudaEvent_t fork = nullptr, joins[kMaxStreams] = {}, done = nullptr;
    bool ready = false;
};

DeviceState g_dev[kMaxDevices];

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

bf_status cuda_fail(cudaError_t e, const char *what) {
    cudaGetLastError();
    return bfi::fail(BF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bf_status setup(DeviceState &d) {
    if (d.ready) return BF_OK;
    cudaError_t e = cudaEventCreateWithFlags(&d.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d.done, cudaEventDisableTiming);
    for (int i = 0; i < kMaxStreams && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&d.streams[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d.joins[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return cuda_fail(e, "host-filter streams");
    e = cudaEventRecord(d.done, d.streams[0]);  // nothing to wait for yet
    if (e != cudaSuccess) return cuda_fail(e, "host-filter events");
    d.ready = true;
    return BF_OK;
}

}  // namespace

extern "C" bf_status bf_filter_host(const bf_plan *const *plans, int n, const float *h_in, size_t in_pitch,
                                    float *const *h_outs, size_t out_pitch, int height, int width, int n_streams,
                                    void *stream) {
    if (!plans || !h_outs || n < 1 || n > 256 || n_streams < 1 || n_streams > kMaxStreams)
        return bfi::fail(BF_ERR_INVALID_ARG, "bad plan list or stream count");
    const int device = plans[0] ? plans[0]->desc.device : -1;
    for (int i = 0; i < n; ++i) {
        if (!plans[i] || !h_outs[i]) return bfi::fail(BF_ERR_INVALID_ARG, "NULL plan or output");
        if (plans[i]->desc.device != device) return bfi::fail(BF_ERR_INVALID_ARG, "plans on several devices");
        bf_status st = bfi::check_image(h_in, in_pitch, h_outs[i], out_pitch, height, width);
        if (st != BF_OK) return st;
    }
    if (height == 0 || width == 0) return BF_OK;
    if (device < 0 || device >= kMaxDevices) return bfi::fail(BF_ERR_NO_DEVICE, "host-only plan (device = -1)");
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || (prev != device && cudaSetDevice(device) != cudaSuccess)) {
        cudaGetLastError();
        return bfi::fail(BF_ERR_NO_DEVICE, "cannot select the plans' device");
    }
    DeviceState &d = g_dev[device];
    std::lock_guard<std::mutex> lk(d.mu);
    bf_status st = setup(d);
    // the block: input, n outputs, then each plan's scratch
    const size_t row = (size_t)width * sizeof(float), img = align_up(row * height);
    std::vector<bfi::TileConfig> tcs(n);
    std::vector<size_t> scr(n);
    size_t need = img * (1 + (size_t)n);
    for (int i = 0; i < n && st == BF_OK; ++i) {
        tcs[i] = bfi::choose_tile(plans[i]->kp, height, width, plans[i]->desc.precision);
        scr[i] = align_up(bfi::scratch_bytes(tcs[i], height, width, plans[i]->kp.zbins));
        need += scr[i];
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (st == BF_OK && need > d.bytes) {
        // the previous call's work must finish before its block goes
        cudaError_t e = cudaEventSynchronize(d.done);
        if (e == cudaSuccess && d.block) e = cudaFree(d.block);
        d.block = nullptr;
        d.bytes = 0;
        if (e == cudaSuccess) e = cudaMalloc((void **)&d.block, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            st = bfi::fail(BF_ERR_OOM, "host-filter device block of " + std::to_string(need) + " bytes");
        } else {
            d.bytes = need;
        }
    }
    cudaError_t e = cudaSuccess;
    float *d_in = reinterpret_cast<float *>(d.block);
    if (st == BF_OK) {
        // upload after the previous call's last download, then fork to the compute streams
        e = cudaStreamWaitEvent(s, d.done, 0);
        if (e == cudaSuccess) e = cudaMemcpy2DAsync(d_in, row, h_in, in_pitch, row, height, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaEventRecord(d.fork, s);
        for (int k = 0; k < n_streams && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(d.streams[k], d.fork, 0);
        if (e != cudaSuccess) st = cuda_fail(e, "host-filter upload");
    }
    char *scratch = d.block + img * (1 + (size_t)n);
    for (int i = 0; i < n && st == BF_OK; ++i) {
        cudaStream_t cs = d.streams[i % n_streams];
        float *d_out = reinterpret_cast<float *>(d.block + img * (1 + (size_t)i));
        st = bfi::filter_image(plans[i], tcs[i], d_in, row, d_out, row, height, width,
                               scr[i] ? reinterpret_cast<float *>(scratch) : nullptr, cs);
        scratch += scr[i];
        if (st == BF_OK) {
            e = cudaMemcpy2DAsync(h_outs[i], out_pitch, d_out, row, row, height, cudaMemcpyDeviceToHost, cs);
            if (e != cudaSuccess) st = cuda_fail(e, "host-filter download");
        }
    }
    // join (also after a failure, so that the chain stays ordered)
    if (d.ready && d.block) {
        for (int k = 0; k < n_streams; ++k)
            if (cudaEventRecord(d.joins[k], d.streams[k]) != cudaSuccess ||
                cudaStreamWaitEvent(s, d.joins[k], 0) != cudaSuccess) {
                cudaGetLastError();
                if (st == BF_OK) st = bfi::fail(BF_ERR_CUDA, "host-filter join");
            }
        if (cudaEventRecord(d.done, s) != cudaSuccess) {
            cudaGetLastError();
            if (st == BF_OK) st = bfi::fail(BF_ERR_CUDA, "host-filter join");
        }
    }
    if (prev != device) cudaSetDevice(prev);
    return st;
}
