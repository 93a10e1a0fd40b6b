// bf_filter_host: the filter for images in host memory.  One call uploads the
// image, filters it with each of n plans (the paper's use of one image under
// several parameter settings, Sec. V-C) on internal compute streams, and
// downloads each result on an internal copy stream as soon as its filter ends.
// Device buffers (the input, n outputs and each plan's scratch) come from two
// blocks per device, used by alternate calls, allocated on first use and grown
// when a call needs more, so steady-state calls allocate nothing.  A call's
// upload waits for the last download of the call two before it (the previous
// user of its block), so a call issued on another stream than the one before it
// uploads while that one still computes; calls on one stream run one after
// another, as that stream orders them.
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

constexpr int kMaxStreams = 16;
constexpr int kCopyStreams = 2;
constexpr int kBlocks = 2;
constexpr int kMaxDevices = 64;

struct Block {
    char *mem = nullptr;
    size_t bytes = 0;
    cudaEvent_t done = nullptr;  // the last download of the call that used this block last
};

struct DeviceState {
    std::mutex mu;
    Block blocks[kBlocks];
    unsigned next = 0;  // block of the next call
    cudaStream_t streams[kMaxStreams] = {}, copies[kCopyStreams] = {};
    cudaEvent_t fork = nullptr, filtered[kMaxStreams] = {}, copied[kCopyStreams] = {};
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
    const unsigned flags = cudaEventDisableTiming;
    cudaError_t e = cudaEventCreateWithFlags(&d.fork, flags);
    for (int i = 0; i < kMaxStreams && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&d.streams[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d.filtered[i], flags);
    }
    for (int i = 0; i < kCopyStreams && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&d.copies[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d.copied[i], flags);
    }
    for (int b = 0; b < kBlocks && e == cudaSuccess; ++b) {
        e = cudaEventCreateWithFlags(&d.blocks[b].done, flags);
        if (e == cudaSuccess) e = cudaEventRecord(d.blocks[b].done, d.streams[0]);  // nothing to wait for yet
    }
    if (e != cudaSuccess) return cuda_fail(e, "host-filter streams and events");
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
    Block &blk = d.blocks[d.next % kBlocks];
    cudaStream_t s = (cudaStream_t)stream;
    if (st == BF_OK && need > blk.bytes) {
        // the block's previous call must finish before the block goes
        cudaError_t e = cudaEventSynchronize(blk.done);
        if (e == cudaSuccess && blk.mem) e = cudaFree(blk.mem);
        blk.mem = nullptr;
        blk.bytes = 0;
        if (e == cudaSuccess) e = cudaMalloc((void **)&blk.mem, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            st = bfi::fail(BF_ERR_OOM, "host-filter device block of " + std::to_string(need) + " bytes");
        } else {
            blk.bytes = need;
        }
    }
    if (st != BF_OK) {
        if (prev != device) cudaSetDevice(prev);
        return st;
    }
    ++d.next;
    cudaError_t e = cudaSuccess;
    float *d_in = reinterpret_cast<float *>(blk.mem);
    // upload once the block's previous call has downloaded its last result, then fork to the compute streams
    e = cudaStreamWaitEvent(s, blk.done, 0);
    if (e == cudaSuccess) e = cudaMemcpy2DAsync(d_in, row, h_in, in_pitch, row, height, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(d.fork, s);
    for (int k = 0; k < n_streams && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(d.streams[k], d.fork, 0);
    // the copy streams start after the fork too, so that a join below never waits on older work only
    for (int k = 0; k < kCopyStreams && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(d.copies[k], d.fork, 0);
    if (e != cudaSuccess) st = cuda_fail(e, "host-filter upload");
    char *scratch = blk.mem + img * (1 + (size_t)n);
    for (int i = 0; i < n && st == BF_OK; ++i) {
        const int k = i % n_streams;
        cudaStream_t cs = d.streams[k], ds = d.copies[i % kCopyStreams];
        float *d_out = reinterpret_cast<float *>(blk.mem + img * (1 + (size_t)i));
        st = bfi::filter_image(plans[i], tcs[i], d_in, row, d_out, row, height, width,
                               scr[i] ? reinterpret_cast<float *>(scratch) : nullptr, cs);
        scratch += scr[i];
        if (st == BF_OK) {
            // the download waits for this filter only (the event's record at this point of the compute stream)
            e = cudaEventRecord(d.filtered[k], cs);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(ds, d.filtered[k], 0);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(h_outs[i], out_pitch, d_out, row, row, height, cudaMemcpyDeviceToHost, ds);
            if (e != cudaSuccess) st = cuda_fail(e, "host-filter download");
        }
    }
    // join the compute and copy streams back to `stream` (also after a failure, so that the block's next call
    // waits for everything this one enqueued)
    for (int k = 0; k < n_streams; ++k)
        if (cudaEventRecord(d.filtered[k], d.streams[k]) != cudaSuccess ||
            cudaStreamWaitEvent(s, d.filtered[k], 0) != cudaSuccess) {
            cudaGetLastError();
            if (st == BF_OK) st = bfi::fail(BF_ERR_CUDA, "host-filter join");
        }
    for (int k = 0; k < kCopyStreams; ++k)
        if (cudaEventRecord(d.copied[k], d.copies[k]) != cudaSuccess ||
            cudaStreamWaitEvent(s, d.copied[k], 0) != cudaSuccess) {
            cudaGetLastError();
            if (st == BF_OK) st = bfi::fail(BF_ERR_CUDA, "host-filter join");
        }
    if (cudaEventRecord(blk.done, s) != cudaSuccess) {
        cudaGetLastError();
        if (st == BF_OK) st = bfi::fail(BF_ERR_CUDA, "host-filter join");
    }
    if (prev != device) cudaSetDevice(prev);
    return st;
}
