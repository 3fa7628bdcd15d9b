// validate.cu -- FP64 reductions that check a volume's irradiance maps against a known value.
//
// Eq. 3 is used in its self-normalised form (the weighted sum of the rays' radiance divided
// by the sum of the weights), so two situations have an exact answer that holds for every
// texel, whatever the ray set and its rotation:
//  - the white furnace: every ray brings the same radiance L (a sky of L with no geometry, or
//    surfaces of emission L and albedo 0), and every interior texel is L;
//  - a closed room whose surfaces all have emission Le and albedo rho, lit only by itself
//    through the multi-bounce term (Sec. 3.3, previous frame's probes, coefficient 1): with
//    hysteresis h the maps follow s_0 = Le, s_n = h s_(n-1) + (1-h)(Le + rho s_(n-1)), that is
//    s_n = S + (Le - S) r^n with S = Le / (1 - rho) and r = h + (1 - h) rho.
// These reductions measure the maps' deviation from such a value on the device, in double
// precision. They are the only FP64 arithmetic of the library on the GPU; no step of an
// update uses it.
#include "handles.h"
#include "internal.h"

#include <math.h>

namespace sdfddgi {

namespace {

constexpr int kDevThreads = 256;
constexpr int kDevWarps = kDevThreads / 32;
constexpr int kStatWords = 11;  // count, sum[3], max|dev|[3], sum dev^2[3], non-finite texels

struct DevStat {
    double v[kStatWords];
};

__device__ __forceinline__ void stat_zero(DevStat& s) {
#pragma unroll
    for (int k = 0; k < kStatWords; ++k) s.v[k] = 0.0;
}

// a + b in a fixed order; the maxima propagate NaN (which no finite texel produces)
__device__ __forceinline__ void stat_merge(DevStat& a, const DevStat& b) {
    a.v[0] += b.v[0];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        a.v[1 + c] += b.v[1 + c];
        const double m = b.v[4 + c];
        if (m > a.v[4 + c] || m != m) a.v[4 + c] = m;
        a.v[7 + c] += b.v[7 + c];
    }
    a.v[10] += b.v[10];
}

__device__ __forceinline__ void stat_warp_reduce(DevStat& s) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        DevStat o;
#pragma unroll
        for (int k = 0; k < kStatWords; ++k) o.v[k] = __shfl_xor_sync(0xffffffffu, s.v[k], off);
        stat_merge(s, o);
    }
}

// Block-wide reduction of one DevStat per thread; thread 0 returns the total (deterministic:
// the same tree for every launch of the same size).
__device__ DevStat stat_block_reduce(DevStat s) {
    __shared__ double part[kDevWarps][kStatWords];
    stat_warp_reduce(s);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < kStatWords; ++k) part[warp][k] = s.v[k];
    __syncthreads();
    DevStat t;
    stat_zero(t);
    if (threadIdx.x == 0)
        for (int w = 0; w < kDevWarps; ++w) {
            DevStat o;
#pragma unroll
            for (int k = 0; k < kStatWords; ++k) o.v[k] = part[w][k];
            stat_merge(t, o);
        }
    return t;
}

// One pass over the interior irradiance texels of the active probes: each block writes its
// partial statistics (relative deviations (E - ref) / ref per channel) to partial[blockIdx.x].
__global__ void __launch_bounds__(kDevThreads) irradiance_deviation_kernel(
    const float4* __restrict__ irr, int64_t P, const sdfddgi_probe_state* __restrict__ states, double3 ref,
    double* __restrict__ partial) {
    DevStat s;
    stat_zero(s);
    const double inv[3] = {1.0 / ref.x, 1.0 / ref.y, 1.0 / ref.z};
    const double r[3] = {ref.x, ref.y, ref.z};
    const int64_t n = P * kIrrTexels;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t p = i / kIrrTexels;
        if (states && !(states[p].flags & SDFDDGI_PROBE_ACTIVE)) continue;
        const int t = (int)(i - p * kIrrTexels);
        const int row = 1 + t / kIrrN, col = 1 + t % kIrrN;
        const float4 e = irr[p * (kIrrT * kIrrT) + row * kIrrT + col];
        const float ec[3] = {e.x, e.y, e.z};
        if (!isfinite(ec[0]) || !isfinite(ec[1]) || !isfinite(ec[2])) {
            s.v[10] += 1.0;
            continue;
        }
        s.v[0] += 1.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double v = (double)ec[c];
            const double d = (v - r[c]) * inv[c];
            s.v[1 + c] += v;
            s.v[4 + c] = fmax(s.v[4 + c], fabs(d));
            s.v[7 + c] += d * d;
        }
    }
    const DevStat t = stat_block_reduce(s);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < kStatWords; ++k) partial[(size_t)blockIdx.x * kStatWords + k] = t.v[k];
}

// Sums the blocks' partials in a fixed order and writes the 11 results (means and RMS formed).
__global__ void __launch_bounds__(kDevThreads) deviation_finish_kernel(const double* __restrict__ partial,
                                                                        int n_parts, double* __restrict__ out) {
    DevStat s;
    stat_zero(s);
    for (int j = threadIdx.x; j < n_parts; j += blockDim.x) {
        DevStat o;
#pragma unroll
        for (int k = 0; k < kStatWords; ++k) o.v[k] = partial[(size_t)j * kStatWords + k];
        stat_merge(s, o);
    }
    const DevStat t = stat_block_reduce(s);
    if (threadIdx.x == 0) {
        const double cnt = t.v[0];
        out[0] = cnt;
        for (int c = 0; c < 3; ++c) {
            out[1 + c] = cnt > 0.0 ? t.v[1 + c] / cnt : 0.0;
            out[4 + c] = t.v[4 + c];
            out[7 + c] = cnt > 0.0 ? sqrt(t.v[7 + c] / cnt) : 0.0;
        }
        out[10] = t.v[10];
    }
}

}  // namespace

}  // namespace sdfddgi

extern "C" {

SDFDDGI_API int sdfddgi_irradiance_deviation(const sdfddgi_volume* v, const sdfddgi_probe_state* states,
                                             const float ref_rgb[3], double out[11], void* stream) {
    using namespace sdfddgi;
    if (!v || !ref_rgb || !out)
        return report_error(SDFDDGI_ERR_INVALID_ARG, "irradiance_deviation: volume, ref_rgb and out must be given");
    for (int c = 0; c < 3; ++c)
        if (!(ref_rgb[c] > 0.f) || !isfinite(ref_rgb[c]))
            return report_error(SDFDDGI_ERR_INVALID_ARG,
                                "irradiance_deviation: ref_rgb must be finite and > 0 in every channel");
    for (int k = 0; k < kStatWords; ++k) out[k] = 0.0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t n = v->P * kIrrTexels;
    const int64_t want = (n + kDevThreads - 1) / kDevThreads, cap = 4LL * (sms > 0 ? sms : 148);
    const int grid = (int)(want < 1 ? 1 : (want < cap ? want : cap));
    if (e == cudaSuccess && states) {  // the kernel reads the states: they must be device memory
        cudaPointerAttributes a{};
        e = cudaPointerGetAttributes(&a, states);
        if (e == cudaSuccess && a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
            return report_error(SDFDDGI_ERR_INVALID_ARG, "irradiance_deviation: states must be device memory");
    }
    double* buf = nullptr;  // grid partials, then the 11 results
    if (e == cudaSuccess)
        e = cudaMallocAsync(reinterpret_cast<void**>(&buf), sizeof(double) * kStatWords * (grid + 1), st);
    if (e == cudaSuccess) {
        const double3 ref = make_double3(ref_rgb[0], ref_rgb[1], ref_rgb[2]);
        irradiance_deviation_kernel<<<grid, kDevThreads, 0, st>>>(v->irr[v->cur], v->P, states, ref, buf);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        deviation_finish_kernel<<<1, kDevThreads, 0, st>>>(buf, grid, buf + (size_t)kStatWords * grid);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, buf + (size_t)kStatWords * grid, sizeof(double) * kStatWords,
                            cudaMemcpyDeviceToHost, st);
    if (buf) {
        const cudaError_t f = cudaFreeAsync(buf, st);
        if (e == cudaSuccess) e = f;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return report_error(SDFDDGI_ERR_CUDA, cudaGetErrorString(e));
    return SDFDDGI_OK;
}

}  // extern "C"
