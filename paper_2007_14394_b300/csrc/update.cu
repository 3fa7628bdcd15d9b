// update.cu -- the fused per-probe update kernel (Sec. 3.3 of Hu et al., arXiv 2007.14394).
//
// One CTA per probe; the probe's rays are processed in chunks of blockDim rays.
//  1. primary traces   -- a lane-persistent pool: every lane takes the next ray from a
//                         shared counter as soon as its current trace ends, so a warp keeps
//                         all its lanes stepping while trace lengths differ wildly;
//  2. hit preparation  -- one lane per ray: normal, material, last-frame irradiance
//                         (multi-bounce term) and the set of lights that can reach the hit;
//                         the (ray, light) pairs are compacted into a shadow-task list;
//  3. shadow traces    -- the same lane-persistent pool over the task list; a visible light
//                         sets its bit in the ray's mask (atomicOr: order-independent);
//  4. finalize         -- one lane per ray sums its visible lights in light order
//                         (deterministic) and leaves radiance + clamped distance in shared
//                         memory, where the paper also keeps its samples;
//  5. gather (Eq. 3)   -- one thread per octahedral texel averages all samples of the probe
//                         with cosine (irradiance) or cosine^p (depth moments) weights and
//                         mixes the result with last frame's texel;
//  6. borders + store  -- the 1-texel borders are filled in shared memory and each map
//                         leaves as contiguous 16-byte stores.
#include "device.cuh"

namespace sdfddgi {

constexpr int kMaxThreads = 256;

// c^p for the depth weights; p = 50 (the usual sharpness) as a fixed product chain.
template <int P>
__device__ __forceinline__ float pow_fixed(float c) {
    static_assert(P == 50, "only the fixed exponent 50 has a chain");
    const float c2 = c * c, c4 = c2 * c2, c8 = c4 * c4, c16 = c8 * c8, c32 = c16 * c16;
    return c32 * c16 * c2;
}

__device__ __forceinline__ float pow_runtime(float c, int p) {
    float r = 1.f, b = c;
    while (p) {
        if (p & 1) r *= b;
        b *= b;
        p >>= 1;
    }
    return r;
}

struct TraceState {
    float3 o, d;
    float t, tlimit;
    int s;
};

// Advances a sphere trace by one step (the test sequence of sphere_trace in device.cuh:
// leave-box, hit, past-limit, budget). Returns the event, or -1 while it continues;
// on an event, *steps and *t_end receive the step count and the recorded distance.
template <typename T>
__device__ __forceinline__ int trace_step(const VolumeView& v, TraceState& st, float eps, int max_steps,
                                          int* steps, float* t_end) {
    const float3 p = fma3(st.t, st.d, st.o);
    if (p.x < v.lo[0] || p.x > v.hi[0] || p.y < v.lo[1] || p.y > v.hi[1] || p.z < v.lo[2] || p.z > v.hi[2]) {
        *steps = st.s;
        *t_end = st.tlimit;
        return kLeftVolume;
    }
    const float sd = sample_sdf<T>(v, p);
    if (sd < eps) {
        *steps = st.s + 1;
        *t_end = st.t;
        return kHit;
    }
    st.t += sd;
    if (st.t > st.tlimit) {
        *steps = st.s + 1;
        *t_end = st.tlimit;
        return kPastLimit;
    }
    if (++st.s == max_steps) {
        *steps = max_steps;
        *t_end = st.t;
        return kExhausted;
    }
    return -1;
}

// Lane-persistent pool of sphere traces: tasks 0..n-1 are handed out through *counter
// (one shared atomic per warp and round, for the lanes that need work); init(k, st)
// sets up trace k, done(k, event, steps, t) consumes its result. Every lane of every
// warp of the CTA must call this (it uses full-warp votes).
template <typename T, typename Init, typename Done>
__device__ __forceinline__ void trace_pool(const VolumeView& v, int n, int* counter, float eps, int max_steps,
                                           Init init, Done done) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int task = -1;
    bool need = true;
    TraceState st;
    for (;;) {
        const unsigned want = __ballot_sync(full, need);
        if (want) {
            const int leader = __ffs(want) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(counter, __popc(want));
            base = __shfl_sync(full, base, leader);
            if (need) {
                const int k = base + __popc(want & ((1u << lane) - 1u));
                need = false;
                task = k < n ? k : -1;  // a lane that finds the pool dry stays idle
                if (task >= 0) {
                    init(task, st);
                    st.t = 0.f;
                    st.s = 0;
                }
            }
        }
        if (!__any_sync(full, task >= 0)) break;
        if (task >= 0) {
            int steps;
            float t_end;
            const int ev = trace_step<T>(v, st, eps, max_steps, &steps, &t_end);
            if (ev >= 0) {
                done(task, ev, steps, t_end);
                task = -1;
                need = true;
            }
        }
    }
}

// Inclusive prefix sum over the CTA (blockDim a multiple of 32, <= 1024).
__device__ __forceinline__ int block_inclusive_scan(int x, int* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) s_warp[lane] = w;
    }
    __syncthreads();
    return x + (warp > 0 ? s_warp[warp - 1] : 0);
}

// Shared-memory layout of one CTA (dynamic part): all R samples, then the per-chunk
// scratch of chunk = blockDim rays.
struct Smem {
    float4* dir;         // [R] ray direction
    float4* val;         // [R] radiance rgb, clamped distance
    float* t;            // [chunk] primary hit distance
    uint32_t* evsteps;   // [chunk] event | steps << 8
    float4* nrm;         // [chunk] normal
    float4* alb;         // [chunk] albedo
    float4* base;        // [chunk] emission + k * albedo * last-frame irradiance
    float4* xs;          // [chunk] shadow-ray origin
    uint32_t* lit;       // [chunk] visible-light mask
    uint32_t* ssteps;    // [chunk] shadow steps
    uint16_t* tasks;     // [chunk * n_lights] (ray << 5 | light)
};

__host__ __device__ inline size_t smem_bytes(int R, int chunk, int n_lights) {
    return (size_t)R * 32 + (size_t)chunk * (4 + 4 + 16 * 4 + 4 + 4) + (size_t)chunk * n_lights * 2 + 16;
}

__device__ __forceinline__ Smem carve(unsigned char* raw, int R, int chunk) {
    Smem s;
    s.dir = reinterpret_cast<float4*>(raw);
    s.val = s.dir + R;
    s.nrm = s.val + R;
    s.alb = s.nrm + chunk;
    s.base = s.alb + chunk;
    s.xs = s.base + chunk;
    s.t = reinterpret_cast<float*>(s.xs + chunk);
    s.evsteps = reinterpret_cast<uint32_t*>(s.t + chunk);
    s.lit = s.evsteps + chunk;
    s.ssteps = s.lit + chunk;
    s.tasks = reinterpret_cast<uint16_t*>(s.ssteps + chunk);
    return s;
}

// Light l's contribution factor at x with normal n: cos for a directional light,
// cos * window / d^2 for a point light (0 where the light cannot reach x).
__device__ __forceinline__ float light_scale(const LightDev& li, float3 x, float3 n, bool* gate) {
    if (li.type == SDFDDGI_LIGHT_DIRECTIONAL) {
        const float c = dot(n, f3(li.v[0], li.v[1], li.v[2]));
        *gate = c > 0.f;
        return c;
    }
    const float3 Lv = f3(li.v[0], li.v[1], li.v[2]) - x;
    const float dist = sqrtf(dot(Lv, Lv));
    if (!(dist > 0.f)) {
        *gate = false;
        return 0.f;
    }
    const float c = dot(n, Lv) / dist;
    const float q = dist / li.range;
    const float q2 = q * q;
    float win = fminf(fmaxf(1.f - q2 * q2, 0.f), 1.f);
    win *= win;
    *gate = c > 0.f && win > 0.f;
    return c * win / (dist * dist);
}

template <typename T, int PEXP>
__global__ void __launch_bounds__(kMaxThreads, 3) probe_update_kernel(const __grid_constant__ UpdateParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float4 s_irr[kIrrT * kIrrT];
    __shared__ __align__(16) float2 s_dep[kDepT * kDepT];  // stored out as float4 pairs
    __shared__ int s_counter[2];
    __shared__ int s_warp[32];
    __shared__ int s_ntasks;

    const int chunk = blockDim.x;
    const Smem S = carve(smem_raw, P.R, chunk);
    const int p = blockIdx.x;
    const int tid = threadIdx.x, nt = blockDim.x;
    const VolumeView& V = P.vol;
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

    for (int c0 = 0; c0 < P.R; c0 += chunk) {
        const int nc = min(chunk, P.R - c0);
        if (tid == 0) {
            s_counter[0] = 0;
            s_counter[1] = 0;
        }
        __syncthreads();

        // ---- 1. primary traces
        trace_pool<T>(
            V, nc, &s_counter[0], P.eps_w, P.max_steps,
            [&](int k, TraceState& st) {
                st.o = o;
                st.d = ray_direction(c0 + k, P.R, P.rot);
                st.tlimit = P.tmax_w;
            },
            [&](int k, int ev, int steps, float t_end) {
                S.t[k] = t_end;
                S.evsteps[k] = (uint32_t)ev | ((uint32_t)steps << 8);
            });
        __syncthreads();

        // ---- 2. hit preparation and shadow-task compaction (one lane per ray)
        uint32_t gate = 0;
        if (tid < nc) {
            const int i = c0 + tid;
            const float3 d = ray_direction(i, P.R, P.rot);
            S.dir[i] = make_float4(d.x, d.y, d.z, 0.f);
            S.lit[tid] = 0;
            S.ssteps[tid] = 0;
            const int ev = (int)(S.evsteps[tid] & 0xffu);
            if (!is_miss(ev)) {
                const float3 x = fma3(S.t[tid], d, o);
                const float hh = 0.5f * V.h;
                const float gx = sample_sdf<T>(V, f3(x.x + hh, x.y, x.z)) - sample_sdf<T>(V, f3(x.x - hh, x.y, x.z));
                const float gy = sample_sdf<T>(V, f3(x.x, x.y + hh, x.z)) - sample_sdf<T>(V, f3(x.x, x.y - hh, x.z));
                const float gz = sample_sdf<T>(V, f3(x.x, x.y, x.z + hh)) - sample_sdf<T>(V, f3(x.x, x.y, x.z - hh));
                const float glen = sqrtf(gx * gx + gy * gy + gz * gz);
                const float3 n = glen > 0.f ? f3(gx / glen, gy / glen, gz / glen) : f3(-d.x, -d.y, -d.z);
                float3 albedo, emission;
                sample_material(V, x, &albedo, &emission);
                float3 ind = f3(0.f, 0.f, 0.f);
                if (P.k_bounce != 0.f)
                    ind = interpolate_irradiance(P.gdims, P.gorigin, P.gspacing, P.prev_irr, P.prev_valid, x, n);
                const float3 xs = fma3(P.bias_w, n, x);
                for (int l = 0; l < P.n_lights; ++l) {
                    bool g;
                    light_scale(P.lights[l], x, n, &g);
                    if (g) gate |= 1u << l;
                }
                S.nrm[tid] = make_float4(n.x, n.y, n.z, 0.f);
                S.alb[tid] = make_float4(albedo.x, albedo.y, albedo.z, 0.f);
                S.base[tid] = make_float4(emission.x + albedo.x * P.k_bounce * ind.x,
                                          emission.y + albedo.y * P.k_bounce * ind.y,
                                          emission.z + albedo.z * P.k_bounce * ind.z, 0.f);
                S.xs[tid] = make_float4(xs.x, xs.y, xs.z, 0.f);
            }
        }
        const int cnt = __popc(gate);
        const int incl = block_inclusive_scan(cnt, s_warp);
        if (tid == nt - 1) s_ntasks = incl;
        {
            int pos = incl - cnt;
            uint32_t g = gate;
            while (g) {
                const int l = __ffs(g) - 1;
                g &= g - 1;
                S.tasks[pos++] = (uint16_t)((tid << 5) | l);
            }
        }
        __syncthreads();

        // ---- 3. shadow traces toward every light that can reach a hit
        trace_pool<T>(
            V, s_ntasks, &s_counter[1], P.eps_w, P.max_steps,
            [&](int k, TraceState& st) {
                const uint32_t tk = S.tasks[k];
                const int r = (int)(tk >> 5), l = (int)(tk & 31u);
                const LightDev& li = P.lights[l];
                const float4 xs = S.xs[r];
                st.o = f3(xs.x, xs.y, xs.z);
                if (li.type == SDFDDGI_LIGHT_DIRECTIONAL) {
                    st.d = f3(li.v[0], li.v[1], li.v[2]);
                    st.tlimit = P.tmax_w;
                } else {
                    const float3 Ls = f3(li.v[0], li.v[1], li.v[2]) - st.o;
                    const float ds = sqrtf(dot(Ls, Ls));
                    st.d = (1.f / ds) * Ls;
                    st.tlimit = ds;
                }
            },
            [&](int k, int ev, int steps, float) {
                const uint32_t tk = S.tasks[k];
                const int r = (int)(tk >> 5), l = (int)(tk & 31u);
                atomicAdd(&S.ssteps[r], (uint32_t)steps);
                if (is_miss(ev)) atomicOr(&S.lit[r], 1u << l);  // occluded by a hit or an exhausted graze
            });
        __syncthreads();

        // ---- 4. finalize radiance (one lane per ray, lights in order)
        if (tid < nc) {
            const int i = c0 + tid;
            const float4 d4 = S.dir[i];
            const uint32_t es = S.evsteps[tid];
            const int ev = (int)(es & 0xffu);
            const float t = S.t[tid];
            float3 L;
            uint32_t lit = 0;
            if (is_miss(ev)) {
                L = f3(P.sky[0], P.sky[1], P.sky[2]);
            } else {
                const float3 d = f3(d4.x, d4.y, d4.z);
                const float3 x = fma3(t, d, o);
                const float4 n4 = S.nrm[tid];
                const float3 n = f3(n4.x, n4.y, n4.z);
                lit = S.lit[tid];
                float3 direct = f3(0.f, 0.f, 0.f);
                for (int l = 0; l < P.n_lights; ++l) {
                    if (!((lit >> l) & 1u)) continue;
                    bool g;
                    const float sc = light_scale(P.lights[l], x, n, &g);
                    direct = fma3(sc, f3(P.lights[l].rgb[0], P.lights[l].rgb[1], P.lights[l].rgb[2]), direct);
                }
                const float inv_pi = 0.318309886183790671538f;
                const float4 a = S.alb[tid], b = S.base[tid];
                L = f3(fmaf(a.x * inv_pi, direct.x, b.x), fmaf(a.y * inv_pi, direct.y, b.y),
                       fmaf(a.z * inv_pi, direct.z, b.z));
            }
            const float td = is_miss(ev) ? P.tmax_w : fminf(t, P.tmax_w);
            S.val[i] = make_float4(L.x, L.y, L.z, td);
            if (P.records) {
                sdfddgi_ray_record rec;
                rec.t = t;
                rec.L[0] = L.x;
                rec.L[1] = L.y;
                rec.L[2] = L.z;
                rec.lit_mask = lit;
                rec.shadow_steps = S.ssteps[tid];
                rec.steps = (uint16_t)(es >> 8);
                rec.event = (uint8_t)ev;
                rec.reserved0 = 0;
                rec.reserved1 = 0;
                P.records[(size_t)p * P.R + i] = rec;
            }
        }
        __syncthreads();
    }

    // ---- 5. one texel per thread, cosine-lobe gather over all samples (Eq. 3)
    for (int task = tid; task < kIrrTexels + kDepTexels; task += nt) {
        if (task < kIrrTexels) {
            const int a = task % kIrrN, b = task / kIrrN;
            const float3 u = texel_dir(a, b, kIrrN);
            float sw = 0.f, r = 0.f, g = 0.f, bl = 0.f;
            for (int i = 0; i < P.R; ++i) {
                const float4 di = S.dir[i];
                const float c = fmaf(u.x, di.x, fmaf(u.y, di.y, u.z * di.z));
                if (c > 0.f) {
                    const float4 vi = S.val[i];
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
                const float4 di = S.dir[i];
                const float c = fmaf(u.x, di.x, fmaf(u.y, di.y, u.z * di.z));
                if (c > 0.f) {
                    const float w = PEXP > 0 ? pow_fixed<(PEXP > 0 ? PEXP : 50)>(c) : pow_runtime(c, P.depth_exp);
                    const float t = S.val[i].w;
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

    // ---- 6. borders from the interior, then contiguous vector stores
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

template <typename T, int PEXP>
static cudaError_t launch_typed(const UpdateParams& p, int threads, size_t smem, cudaStream_t stream) {
    auto* k = probe_update_kernel<T, PEXP>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<p.P, threads, smem, stream>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_update(const UpdateParams& p, cudaStream_t stream) {
    if (p.P == 0) return cudaSuccess;
    const int threads = p.R >= kMaxThreads ? kMaxThreads : ((p.R + 31) / 32) * 32;
    const size_t smem = smem_bytes(p.R, threads, p.n_lights);
    const bool p50 = p.depth_exp == 50;
    if (p.vol.dtype == SDFDDGI_F16)
        return p50 ? launch_typed<__half, 50>(p, threads, smem, stream) : launch_typed<__half, 0>(p, threads, smem, stream);
    return p50 ? launch_typed<float, 50>(p, threads, smem, stream) : launch_typed<float, 0>(p, threads, smem, stream);
}

}  // namespace sdfddgi
