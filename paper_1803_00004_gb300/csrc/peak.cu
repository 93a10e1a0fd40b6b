// bf_fp32_peak: measured fp32 throughput of the device, the denominator of the
// fused filter's roofline.  The filter's algorithmic count is in fp32 lane
// operations (an add, a multiply or a fused multiply-add is one operation on
// one lane), and its hot loops issue both the scalar FFMA and Blackwell's
// two-wide FFMA2, so the rate of each is measured: kChains independent FMA
// chains per thread (enough to cover the pipeline latency), every SM filled
// with 2048 threads, CUDA events around each launch, best of three.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "bf_internal.h"

namespace {

constexpr int kChains = 8, kUnroll = 16, kThreads = 256, kBlocksPerSm = 8;

__global__ void __launch_bounds__(kThreads) peak_ffma_kernel(float *out, float a, float b, int iters) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3f + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.2345f) out[threadIdx.x] = s;  // never true; keeps the chains
}

__global__ void __launch_bounds__(kThreads) peak_ffma2_kernel(float *out, float a, float b, int iters) {
    float2 x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = make_float2(threadIdx.x * 1e-3f + c, threadIdx.x * 2e-3f - c);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
    if (s == -1.2345f) out[threadIdx.x] = s;
}

}  // namespace

extern "C" bf_status bf_fp32_peak(int device, int iters, double *ffma_ops, double *ffma2_ops) {
    if (!ffma_ops || !ffma2_ops || iters < 1 || iters > (1 << 24)) return bfi::fail(BF_ERR_INVALID_ARG, "bad arguments");
    int prev = 0, sms = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        return bfi::fail(BF_ERR_NO_DEVICE, "cannot select the device");
    }
    bf_status st = BF_OK;
    float *d_out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t s = nullptr;
    cudaError_t e = cudaMalloc((void **)&d_out, kThreads * sizeof(float));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    const int blocks = sms * kBlocksPerSm;
    const double lane_ops = (double)blocks * kThreads * iters * kUnroll * kChains;  // per launch, scalar kernel
    for (int kind = 0; kind < 2 && e == cudaSuccess; ++kind) {
        float best = 0.f;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms up
            e = cudaEventRecord(e0, s);
            if (kind == 0) peak_ffma_kernel<<<blocks, kThreads, 0, s>>>(d_out, 0.9999999f, 1e-7f, iters);
            else peak_ffma2_kernel<<<blocks, kThreads, 0, s>>>(d_out, 0.9999999f, 1e-7f, iters);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && rep > 0) best = best > 0.f ? std::min(best, ms) : ms;
        }
        if (e == cudaSuccess) {
            // an FFMA2 instruction does two lane operations
            const double ops = kind == 0 ? lane_ops : 2.0 * lane_ops;
            (kind == 0 ? *ffma_ops : *ffma2_ops) = ops / (best * 1e-3);
        }
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        st = bfi::fail(BF_ERR_CUDA, std::string("fp32 peak: ") + cudaGetErrorString(e));
    }
    if (s) cudaStreamDestroy(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (d_out) cudaFree(d_out);
    cudaSetDevice(prev);
    return st;
}
