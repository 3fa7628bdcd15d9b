// sample.cu -- probe interpolation at arbitrary points (the probe-interpolation rule of
// Sec. 3.4 of Hu et al., arXiv 2007.14394), without or with the paper's per-pixel probe
// visibility test by SDF trace. One thread per point.
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

// The interpolation with each probe's weight times its visibility from the point.
template <typename T>
__global__ void __launch_bounds__(256) sample_visible_kernel(const __grid_constant__ SampleParams P,
                                                             const __grid_constant__ VisParams V) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const float3 x = f3(P.points[3 * i], P.points[3 * i + 1], P.points[3 * i + 2]);
    const float3 nrm = f3(P.normals[3 * i], P.normals[3 * i + 1], P.normals[3 * i + 2]);
    const float3 e = interpolate_irradiance_visible<T>(P.gdims, P.gorigin, P.gspacing, P.irr, P.valid, V, x, nrm);
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

cudaError_t launch_sample_visible(const SampleParams& p, const VisParams& v, cudaStream_t stream) {
    if (p.n == 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = (p.n + threads - 1) / threads;
    if (v.vol.dtype == kAnalytic)
        sample_visible_kernel<Analytic><<<(unsigned)blocks, threads, 0, stream>>>(p, v);
    else if (v.vol.dtype == SDFDDGI_F16)
        sample_visible_kernel<__half><<<(unsigned)blocks, threads, 0, stream>>>(p, v);
    else
        sample_visible_kernel<float><<<(unsigned)blocks, threads, 0, stream>>>(p, v);
    return cudaGetLastError();
}

}  // namespace sdfddgi
