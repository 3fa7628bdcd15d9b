// peaks.cu -- the L2 read bandwidth the update's gathers run against. The trace and
// hit-preparation stages gather far more bytes than reach DRAM (the SDF's neighbourhood of a
// probe's rays, the material and probe maps), so besides the measured HBM copy their
// rooflines are quoted against what this kernel reads from an L2-resident buffer: vector
// loads that bypass L1 (ld.global.cg), every SM's threads sweeping the buffer in turn.
#include "internal.h"

namespace sdfddgi {

namespace {

__global__ void __launch_bounds__(256) l2_read_kernel(const uint4* __restrict__ buf, size_t n, int reps,
                                                      uint32_t* sink) {
    uint32_t acc = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r)
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            const uint4 v = __ldcg(buf + i);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    if (acc == 0x9e3779b9u) *sink = acc;  // a data-dependent store keeps every load
}

}  // namespace

}  // namespace sdfddgi

extern "C" {

SDFDDGI_API int sdfddgi_l2_read_bandwidth(const void* buf, size_t bytes, int32_t reps, float* gbs, void* stream) {
    using namespace sdfddgi;
    if (gbs) *gbs = 0.f;
    if (!buf || !gbs || bytes < 16 || bytes % 16 != 0 || reinterpret_cast<uintptr_t>(buf) % 16 != 0 || reps < 1 ||
        reps > 1000)
        return report_error(SDFDDGI_ERR_INVALID_ARG,
                            "l2_read_bandwidth: buf (16-byte aligned), bytes (a multiple of 16), gbs, reps 1..1000");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaEvent_t a = nullptr, b = nullptr;
    uint32_t* sink = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&sink), sizeof(uint32_t), st);
    const size_t n = bytes / 16;
    const unsigned grid = (unsigned)(sms > 0 ? 8 * sms : 1184);
    const uint4* p = static_cast<const uint4*>(buf);
    if (e == cudaSuccess) {
        l2_read_kernel<<<grid, 256, 0, st>>>(p, n, 1, sink);  // brings the buffer into L2
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(a, st);
    if (e == cudaSuccess) {
        l2_read_kernel<<<grid, 256, 0, st>>>(p, n, reps, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (sink) cudaFreeAsync(sink, st);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e != cudaSuccess) return report_error(SDFDDGI_ERR_CUDA, cudaGetErrorString(e));
    if (!(ms > 0.f)) return report_error(SDFDDGI_ERR_CUDA, "l2_read_bandwidth: no time elapsed");
    *gbs = (float)((double)bytes * reps / (ms * 1e-3) / 1e9);
    return SDFDDGI_OK;
}

}  // extern "C"
