// sample.cu -- probe interpolation at arbitrary points (the probe-interpolation rule
// of Sec. 3.4 of Hu et al., arXiv 2007.14394, without the per-pixel visibility trace).
#include "device.cuh"

namespace sdfddgi {

__global__ void __launch_bounds__(256) sample_irradiance_kernel(const __grid_constant__ SampleParams P) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const float3 x = f3(P.points[3 * i], P.points[3 * i + 1], P.points[3 * i + 2]);
    const float3 n = f3(P.normals[3 * i], P.normals[3 * i + 1], P.normals[3 * i + 2]);
    const float3 e = interpolate_irradiance(P.gdims, P.gorigin, P.gspacing, P.irr, P.valid, x, n);
    P.out[3 * i] = e.x;
    P.out[3 * i + 1] = e.y;
    P.out[3 * i + 2] = e.z;
}

cudaError_t launch_sample(const SampleParams& p, cudaStream_t stream) {
    if (p.n == 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = (p.n + threads - 1) / threads;
    sample_irradiance_kernel<<<(unsigned)blocks, threads, 0, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace sdfddgi
