// pic_probe.cu -- throughput probe of the FP64 pipe, the denominator of the
// particle kernel's FP64 roofline (GB300 issues FP64 instructions at about 2
// lanes per SM per clock, far below its FP32 rate, so the particle push is
// bound by this pipe and not by HBM).  Every SM runs 64 warps of 8 independent
// fused multiply-add chains; the chains stay bounded (|a| < 1) and their sum is
// written only under a condition that never holds, so no chain can be removed.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/pic_api.h"

int pic_sm_count();
pic_status pic_record_error(pic_status st, const char* msg);

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

__global__ void __launch_bounds__(kThreads) dfma_probe_kernel(double a, double b, int iters, double* sink) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * (double)threadIdx.x + (double)c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.0) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" pic_status pic_probe_fp64_fma(int64_t iters, double* tflops_out) {
    if (iters < 1 || iters > 10000000 || !tflops_out)
        return pic_record_error(PIC_EINVAL, "pic_probe_fp64_fma: iters must be in [1, 1e7] and tflops_out non-null");
    const int blocks = pic_sm_count() * kBlocksPerSm;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double* sink = nullptr;
    pic_status rc = PIC_OK;
    float best = 1e30f;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMalloc(&sink, blocks * sizeof(double));
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // one warm-up, three timed
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) {
            dfma_probe_kernel<<<blocks, kThreads, 0, st>>>(0.999999, 1e-7, (int)iters, sink);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0) best = std::min(best, ms);
    }
    if (e != cudaSuccess) {
        rc = pic_record_error(PIC_ECUDA, cudaGetErrorString(e));
    } else {
        const double flop = 2.0 * kChains * (double)iters * (double)blocks * kThreads;
        *tflops_out = flop / (best * 1e-3) / 1e12;
    }
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    return rc;
}
