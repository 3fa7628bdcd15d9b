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

// Visibility of probe position q from x (normal n), the paper's per-pixel visibility test
// (Sec. 3.4) as a soft SDF shadow trace: from x + bias * n toward q, vis = min over the
// march (t > 0) of softness * sdf / t, 0 on a hit (sdf < eps), clamped to [0, 1]; the march
// ends when t reaches |q - x_s| or after max_steps.
template <typename T>
__device__ float probe_visibility(const VisParams& V, float3 x, float3 n, float3 q) {
    const float3 xs = fma3(V.bias_w, n, x);
    const float3 v = q - xs;
    const float L = sqrtf(dot(v, v));
    if (!(L > 0.f)) return 1.f;
    const float inv_l = 1.0f / L;
    const float3 d = f3(v.x * inv_l, v.y * inv_l, v.z * inv_l);
    float vis = 1.f, t = 0.f;
    for (int s = 0; s < V.max_steps; ++s) {
        if (t >= L) break;
        const float sd = sample_sdf<T>(V.vol, fma3(t, d, xs));
        if (sd < V.eps_w) return 0.f;
        if (t > 0.f) vis = fminf(vis, V.softness * sd / t);
        t += sd;
    }
    return fminf(fmaxf(vis, 0.f), 1.f);
}

// The interpolation of interpolate_irradiance with each probe's weight times its
// visibility from x; probes at their grid positions or at the states' positions.
template <typename T>
__global__ void __launch_bounds__(256) sample_visible_kernel(const __grid_constant__ SampleParams P,
                                                             const __grid_constant__ VisParams V) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const float3 x = f3(P.points[3 * i], P.points[3 * i + 1], P.points[3 * i + 2]);
    const float3 nrm = f3(P.normals[3 * i], P.normals[3 * i + 1], P.normals[3 * i + 2]);
    const float xs[3] = {x.x, x.y, x.z};
    int base[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float c = fminf(fmaxf((xs[a] - P.gorigin[a]) / P.gspacing[a], 0.f), (float)(P.gdims[a] - 1));
        int b = (int)floorf(c);
        b = max(0, min(b, P.gdims[a] - 2));
        base[a] = b;
        f[a] = P.gdims[a] > 1 ? c - (float)b : 0.f;
    }
    const float2 uv = oct_encode(nrm);
    const float cx = fmaf(uv.x, (float)kIrrN, 0.5f), cy = fmaf(uv.y, (float)kIrrN, 0.5f);
    const int x0 = min((int)floorf(cx), kIrrN), y0 = min((int)floorf(cy), kIrrN);
    const float fx = cx - (float)x0, fy = cy - (float)y0;
    float sw = 0.f, r = 0.f, g = 0.f, bl = 0.f;
    for (int k = 0; k < 8; ++k) {
        const int dx = k & 1, dy = (k >> 1) & 1, dz = (k >> 2) & 1;
        const int ix = min(base[0] + dx, P.gdims[0] - 1), iy = min(base[1] + dy, P.gdims[1] - 1),
                  iz = min(base[2] + dz, P.gdims[2] - 1);
        const size_t p = ((size_t)iz * P.gdims[1] + iy) * P.gdims[0] + ix;
        float w = (dx ? f[0] : 1.f - f[0]) * (dy ? f[1] : 1.f - f[1]) * (dz ? f[2] : 1.f - f[2]);
        if (!__ldg(P.valid + p)) w = 0.f;
        if (!(w > 0.f)) continue;
        float3 q;
        if (V.states) {
            q = f3(V.states[p].pos[0], V.states[p].pos[1], V.states[p].pos[2]);
        } else {
            q = f3(fmaf((float)ix, P.gspacing[0], P.gorigin[0]), fmaf((float)iy, P.gspacing[1], P.gorigin[1]),
                   fmaf((float)iz, P.gspacing[2], P.gorigin[2]));
        }
        w *= probe_visibility<T>(V, x, nrm, q);
        if (!(w > 0.f)) continue;
        const float4* m = P.irr + p * (kIrrT * kIrrT);
        const float4 t00 = __ldg(m + y0 * kIrrT + x0), t01 = __ldg(m + y0 * kIrrT + x0 + 1);
        const float4 t10 = __ldg(m + (y0 + 1) * kIrrT + x0), t11 = __ldg(m + (y0 + 1) * kIrrT + x0 + 1);
        const float w00 = (1.f - fx) * (1.f - fy), w01 = fx * (1.f - fy), w10 = (1.f - fx) * fy, w11 = fx * fy;
        r = fmaf(w, w00 * t00.x + w01 * t01.x + w10 * t10.x + w11 * t11.x, r);
        g = fmaf(w, w00 * t00.y + w01 * t01.y + w10 * t10.y + w11 * t11.y, g);
        bl = fmaf(w, w00 * t00.z + w01 * t01.z + w10 * t10.z + w11 * t11.z, bl);
        sw += w;
    }
    float3 e = f3(0.f, 0.f, 0.f);
    if (sw > 0.f) {
        const float inv = 1.0f / sw;
        e = f3(r * inv, g * inv, bl * inv);
    }
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
