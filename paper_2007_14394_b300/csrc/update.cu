// update.cu -- the fused per-probe update kernel (Sec. 3.3 of Hu et al., arXiv 2007.14394).
//
// One CTA per probe. Phase 1: every thread traces rays i = tid, tid + blockDim, ...
// of the probe's rotated spherical-Fibonacci set through the SDF volume, shades the
// hit (emission, lights behind SDF shadow rays, last frame's probes) and leaves the
// radiance and clamped distance of the ray in shared memory -- the paper keeps its
// samples in group-shared memory for the same reason: every texel reuses all of
// them. Phase 2: each thread owns one octahedral texel (36 irradiance + 196 depth
// texels) and gathers the cosine-weighted mean of Eq. 3 over all samples, then mixes
// it with last frame's texel. Phase 3: the one-texel borders are filled in shared
// memory and each map leaves as contiguous 16-byte stores.
#include "device.cuh"

namespace sdfddgi {

__device__ __forceinline__ float powi(float c, int p) {
    float r = 1.f, b = c;
    while (p) {
        if (p & 1) r *= b;
        b *= b;
        p >>= 1;
    }
    return r;
}

// Radiance leaving hit point x back along -d.
template <typename T>
__device__ float3 shade(const UpdateParams& P, float3 x, float3 d, uint32_t* lit_mask, uint32_t* shadow_steps) {
    const VolumeView& v = P.vol;
    const float hh = 0.5f * v.h;
    const float gx = sample_sdf<T>(v, f3(x.x + hh, x.y, x.z)) - sample_sdf<T>(v, f3(x.x - hh, x.y, x.z));
    const float gy = sample_sdf<T>(v, f3(x.x, x.y + hh, x.z)) - sample_sdf<T>(v, f3(x.x, x.y - hh, x.z));
    const float gz = sample_sdf<T>(v, f3(x.x, x.y, x.z + hh)) - sample_sdf<T>(v, f3(x.x, x.y, x.z - hh));
    const float glen = sqrtf(gx * gx + gy * gy + gz * gz);
    const float3 n = glen > 0.f ? f3(gx / glen, gy / glen, gz / glen) : f3(-d.x, -d.y, -d.z);

    float3 albedo, emission;
    sample_material(v, x, &albedo, &emission);
    const float3 xs = fma3(P.bias_w, n, x);

    float3 direct = f3(0.f, 0.f, 0.f);
    uint32_t lit = 0, steps = 0;
    for (int l = 0; l < P.n_lights; ++l) {
        const LightDev& li = P.lights[l];
        float3 ldir;
        float scale, tlimit;
        if (li.type == SDFDDGI_LIGHT_DIRECTIONAL) {
            ldir = f3(li.v[0], li.v[1], li.v[2]);
            const float c = dot(n, ldir);
            if (!(c > 0.f)) continue;
            scale = c;
            tlimit = P.tmax_w;
        } else {
            const float3 Lv = f3(li.v[0], li.v[1], li.v[2]) - x;
            const float dist = sqrtf(dot(Lv, Lv));
            if (!(dist > 0.f)) continue;
            const float c = dot(n, Lv) / dist;
            const float q = dist / li.range;
            const float q2 = q * q;
            float win = fminf(fmaxf(1.f - q2 * q2, 0.f), 1.f);
            win *= win;
            if (!(c > 0.f) || !(win > 0.f)) continue;
            scale = c * win / (dist * dist);
            const float3 Ls = f3(li.v[0], li.v[1], li.v[2]) - xs;
            const float ds = sqrtf(dot(Ls, Ls));
            ldir = (1.f / ds) * Ls;
            tlimit = ds;
        }
        const Trace tr = sphere_trace<T>(v, xs, ldir, P.eps_w, tlimit, P.max_steps);
        steps += (uint32_t)tr.steps;
        if (!is_miss(tr.event)) continue;  // occluded (a hit, or a budget-exhausted graze)
        lit |= 1u << l;
        direct = fma3(scale, f3(li.rgb[0], li.rgb[1], li.rgb[2]), direct);
    }
    *lit_mask = lit;
    *shadow_steps = steps;

    float3 ind = f3(0.f, 0.f, 0.f);
    if (P.k_bounce != 0.f)
        ind = interpolate_irradiance(P.gdims, P.gorigin, P.gspacing, P.prev_irr, P.prev_valid, x, n);
    const float inv_pi = 0.318309886183790671538f;
    return f3(emission.x + albedo.x * (inv_pi * direct.x + P.k_bounce * ind.x),
              emission.y + albedo.y * (inv_pi * direct.y + P.k_bounce * ind.y),
              emission.z + albedo.z * (inv_pi * direct.z + P.k_bounce * ind.z));
}

template <typename T>
__global__ void __launch_bounds__(256) probe_update_kernel(const __grid_constant__ UpdateParams P) {
    extern __shared__ float4 smem[];
    float4* s_dir = smem;        // [R] ray direction
    float4* s_val = smem + P.R;  // [R] radiance rgb, clamped distance
    __shared__ float4 s_irr[kIrrT * kIrrT];
    __shared__ __align__(16) float2 s_dep[kDepT * kDepT];  // stored out as float4 pairs

    const int p = blockIdx.x;
    const int tid = threadIdx.x, nt = blockDim.x;
    float3 o;
    uint32_t flags;
    if (P.states) {
        const sdfddgi_probe_state st = P.states[p];
        o = f3(st.pos[0], st.pos[1], st.pos[2]);
        flags = st.flags;
    } else {
        const int ix = p % P.gdims[0], iy = (p / P.gdims[0]) % P.gdims[1], iz = p / (P.gdims[0] * P.gdims[1]);
        o = f3(fmaf((float)ix, P.gspacing[0], P.gorigin[0]), fmaf((float)iy, P.gspacing[1], P.gorigin[1]),
               fmaf((float)iz, P.gspacing[2], P.gorigin[2]));
        flags = SDFDDGI_PROBE_ACTIVE;
    }
    const float4* prev_i = P.prev_irr + (size_t)p * (kIrrT * kIrrT);
    const float2* prev_d = P.prev_depth + (size_t)p * (kDepT * kDepT);
    float4* cur_i = P.cur_irr + (size_t)p * (kIrrT * kIrrT);
    float4* cur_d4 = reinterpret_cast<float4*>(P.cur_depth + (size_t)p * (kDepT * kDepT));

    if (!(flags & SDFDDGI_PROBE_ACTIVE)) {  // inactive: keep maps and history, cast nothing
        for (int k = tid; k < kIrrT * kIrrT; k += nt) cur_i[k] = __ldg(prev_i + k);
        const float4* pd4 = reinterpret_cast<const float4*>(prev_d);
        for (int k = tid; k < kDepT * kDepT / 2; k += nt) cur_d4[k] = __ldg(pd4 + k);
        if (tid == 0) P.cur_valid[p] = P.prev_valid[p];
        if (P.records)
            for (int i = tid; i < P.R; i += nt) {
                sdfddgi_ray_record rec = {};
                rec.event = kNoRay;
                P.records[(size_t)p * P.R + i] = rec;
            }
        return;
    }
    const float hyst = (P.prev_valid[p] && !(flags & SDFDDGI_PROBE_REJECT_HISTORY)) ? P.hyst : 0.f;

    // ---- phase 1: trace and shade every ray of the probe
    for (int i = tid; i < P.R; i += nt) {
        const float3 d = ray_direction(i, P.R, P.rot);
        const Trace tr = sphere_trace<T>(P.vol, o, d, P.eps_w, P.tmax_w, P.max_steps);
        float3 L;
        uint32_t lit = 0, ssteps = 0;
        if (is_miss(tr.event)) {
            L = f3(P.sky[0], P.sky[1], P.sky[2]);
        } else {
            L = shade<T>(P, fma3(tr.t, d, o), d, &lit, &ssteps);
        }
        const float td = is_miss(tr.event) ? P.tmax_w : fminf(tr.t, P.tmax_w);
        s_dir[i] = make_float4(d.x, d.y, d.z, 0.f);
        s_val[i] = make_float4(L.x, L.y, L.z, td);
        if (P.records) {
            sdfddgi_ray_record rec;
            rec.t = tr.t;
            rec.L[0] = L.x;
            rec.L[1] = L.y;
            rec.L[2] = L.z;
            rec.lit_mask = lit;
            rec.shadow_steps = ssteps;
            rec.steps = (uint16_t)tr.steps;
            rec.event = (uint8_t)tr.event;
            rec.reserved0 = 0;
            rec.reserved1 = 0;
            P.records[(size_t)p * P.R + i] = rec;
        }
    }
    __syncthreads();

    // ---- phase 2: one texel per thread, cosine-lobe gather over all samples (Eq. 3)
    for (int task = tid; task < kIrrTexels + kDepTexels; task += nt) {
        if (task < kIrrTexels) {
            const int a = task % kIrrN, b = task / kIrrN;
            const float3 u = texel_dir(a, b, kIrrN);
            float sw = 0.f, r = 0.f, g = 0.f, bl = 0.f;
            for (int i = 0; i < P.R; ++i) {
                const float4 di = s_dir[i];
                const float c = fmaf(u.x, di.x, fmaf(u.y, di.y, u.z * di.z));
                if (c > 0.f) {
                    const float4 vi = s_val[i];
                    sw += c;
                    r = fmaf(c, vi.x, r);
                    g = fmaf(c, vi.y, g);
                    bl = fmaf(c, vi.z, bl);
                }
            }
            const int k = (b + 1) * kIrrT + (a + 1);
            float4 out = __ldg(prev_i + k);
            if (sw > 0.f) {
                const float inv = 1.f / sw, keep = 1.f - hyst;
                out.x = fmaf(hyst, out.x, keep * (r * inv));
                out.y = fmaf(hyst, out.y, keep * (g * inv));
                out.z = fmaf(hyst, out.z, keep * (bl * inv));
                out.w = 1.f;
            }
            s_irr[k] = out;
        } else {
            const int j = task - kIrrTexels;
            const int a = j % kDepN, b = j / kDepN;
            const float3 u = texel_dir(a, b, kDepN);
            float sw = 0.f, m1 = 0.f, m2 = 0.f;
            for (int i = 0; i < P.R; ++i) {
                const float4 di = s_dir[i];
                const float c = fmaf(u.x, di.x, fmaf(u.y, di.y, u.z * di.z));
                if (c > 0.f) {
                    const float w = powi(c, P.depth_exp);
                    const float t = s_val[i].w;
                    sw += w;
                    m1 = fmaf(w, t, m1);
                    m2 = fmaf(w, t * t, m2);
                }
            }
            const int k = (b + 1) * kDepT + (a + 1);
            float2 out = __ldg(prev_d + k);
            if (sw > 0.f) {
                const float inv = 1.f / sw, keep = 1.f - hyst;
                out.x = fmaf(hyst, out.x, keep * (m1 * inv));
                out.y = fmaf(hyst, out.y, keep * (m2 * inv));
            }
            s_dep[k] = out;
        }
    }
    __syncthreads();

    // ---- phase 3: borders from the interior, then contiguous vector stores
    for (int k = tid; k < kIrrT * kIrrT; k += nt) {
        const int y = k / kIrrT, x = k % kIrrT;
        const int2 s = border_source(y, x, kIrrN);
        if (s.x != y || s.y != x) s_irr[k] = s_irr[s.x * kIrrT + s.y];
    }
    for (int k = tid; k < kDepT * kDepT; k += nt) {
        const int y = k / kDepT, x = k % kDepT;
        const int2 s = border_source(y, x, kDepN);
        if (s.x != y || s.y != x) s_dep[k] = s_dep[s.x * kDepT + s.y];
    }
    __syncthreads();
    for (int k = tid; k < kIrrT * kIrrT; k += nt) cur_i[k] = s_irr[k];
    const float4* sd4 = reinterpret_cast<const float4*>(s_dep);
    for (int k = tid; k < kDepT * kDepT / 2; k += nt) cur_d4[k] = sd4[k];
    if (tid == 0) P.cur_valid[p] = 1;
}

cudaError_t launch_update(const UpdateParams& p, cudaStream_t stream) {
    if (p.P == 0) return cudaSuccess;
    const int threads = p.R >= 256 ? 256 : ((p.R + 31) / 32) * 32;
    const size_t smem = (size_t)p.R * 2 * sizeof(float4);
    if (p.vol.dtype == SDFDDGI_F16)
        probe_update_kernel<__half><<<p.P, threads, smem, stream>>>(p);
    else
        probe_update_kernel<float><<<p.P, threads, smem, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace sdfddgi
