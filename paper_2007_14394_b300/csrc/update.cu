// update.cu -- the per-frame probe update (Sec. 3.3 of Hu et al., arXiv 2007.14394) as
// four stages over device-wide work pools:
//
//  1. primary traces   -- a persistent grid; every lane takes the next ray (of any probe)
//                         as soon as its current sphere trace ends, so all lanes keep
//                         stepping however much trace lengths differ; tasks come from a
//                         global counter in batches of 64 per warp;
//  2. hit preparation  -- one thread per ray: normal, material, last frame's interpolated
//                         irradiance (the multi-bounce term) and the lights that can reach
//                         the hit; the (ray, light) pairs are appended to a shadow-task list;
//  3. shadow traces    -- the same persistent pool over the task list; a visible light sets
//                         its bit in the ray's mask (atomicOr, order-independent);
//  4. gather           -- one CTA per probe: each ray's radiance (visible lights summed in
//                         light order, deterministic) and clamped distance go to shared
//                         memory, where the paper also keeps its samples; one thread per
//                         octahedral texel averages them with cosine (irradiance) or
//                         cosine^p (depth moments) weights (Eq. 3), mixes with last frame's
//                         texel, fills the 1-texel borders, and each map leaves as
//                         contiguous 16-byte stores.
// Device-wide pools pay the latency of the longest ray once per launch instead of once
// per probe.
#include <cstring>
#include <mutex>
#include <type_traits>

#include "device.cuh"
#include "dfloat.cuh"

namespace sdfddgi {

constexpr int kThreads = 256;
// Tasks a warp takes from a global pool at once. 64 measured 7 % faster than 32 on open256
// (half the atomics on the one counter); counters split over several segments of the task
// range were slower, because warps then trace rays from distant parts of the volume at once
// and the SDF working set no longer stays in L2. The shadow pool takes 128: its traces
// measured 3 % faster, while 128 slowed the primary traces and 256 the shadow ones.
constexpr int kBatch = 64;
constexpr int kShadowBatch = 128;
// A pool smaller than this many tasks claims smaller batches (32 primary rays, 64 shadow
// tasks per warp), so that its few tasks per warp still spread evenly over the warps:
// measured on open256 at 32 rays per probe (262 k rays and about 140 k shadow tasks per slab),
// 0.293 -> 0.263 ms per update; the 256-ray update's pools are larger and unchanged.
constexpr uint32_t kSmallPool = 1u << 19;
// Threads per CTA of the persistent trace kernels: two warps, 32 CTAs resident per SM for the
// same 64 warps. As a pool drains, its CTAs leave a warp pair at a time, so the next kernel
// (the other slab's traces, the next stage) takes over freed slots sooner than from CTAs of
// eight warps that wait for their slowest ray.
constexpr int kTraceThreads = 64;
constexpr size_t kSmallShadowRays = (size_t)1 << 19;  // launches below this take the small-pool shadow kernel


// A voxel-volume trace runs in voxel coordinates: o is the origin's voxel coordinate
// ((p - lo)/h - 1/2, voxel centres at integers), t and tlimit are in voxels (d is the same
// unit direction). A trace of primitives runs in world units.
struct TraceState {
    float3 o, d;
    float t, tlimit;
    float last;    // the previous sample's distance (scenes of primitives: bounds the next query)
    float moved;   // how far the trace moved since that sample (scenes of primitives)
    float prev_r;  // over-relaxed stepping: the previous sample's distance,
    float step;    //   the last step taken,
    float omega;   //   and the relaxation factor (1: plain sphere tracing)
    int s;
    uint32_t aux;  // task payload kept for the completion handler
    float tstop;   // plain voxel-volume traces: min(tlimit, the distance at which the ray leaves the box)
};

// Voxel coordinate o lies in the volume box [-1/2, n - 1/2] (the negated test puts NaN outside).
__device__ __forceinline__ bool in_box(const VolumeView& v, float3 o) {
    return o.x >= -0.5f && o.x <= v.gmax[0] && o.y >= -0.5f && o.y <= v.gmax[1] && o.z >= -0.5f && o.z <= v.gmax[2];
}

// The distance along unit direction d (voxel units) at which a ray from o, inside the volume
// box, reaches the face it moves toward; a zero component never reaches its faces. The fast
// quotient (within 2 ulp) moves the distance by rounding only: it decides only when the ray
// leaves the box, and a sample taken up to that distance stays well inside the store's
// half-voxel apron.
__device__ __forceinline__ float box_exit(const VolumeView& v, float3 o, float3 d) {
    const float tx = d.x != 0.f ? __fdividef((d.x > 0.f ? v.gmax[0] : -0.5f) - o.x, d.x) : INFINITY;
    const float ty = d.y != 0.f ? __fdividef((d.y > 0.f ? v.gmax[1] : -0.5f) - o.y, d.y) : INFINITY;
    const float tz = d.z != 0.f ? __fdividef((d.z > 0.f ? v.gmax[2] : -0.5f) - o.z, d.z) : INFINITY;
    return fminf(tx, fminf(ty, tz));
}

// The SDF at p on a sphere trace. For a scene of primitives the query starts from the last
// distance plus the distance moved since (the field is 1-Lipschitz; a plain step moved by the
// last distance, so the bound is twice it; the slack covers float rounding), and falls back to
// a full query if nothing lies below that bound, so the result is always the minimum over all
// primitives.
template <typename T>
__device__ __forceinline__ float trace_sample(const VolumeView& v, TraceState& st, float3 p) {
    if constexpr (std::is_same<T, Analytic>::value) {
        const float bound = st.last < INFINITY ? fmaf(1.001f, st.last + st.moved, 1e-4f * v.h) : INFINITY;
        float sd = analytic_sdf(v, p, bound);
        if (!(sd < bound)) sd = analytic_sdf(v, p, INFINITY);
        st.last = sd;
        return sd;
    } else {
        return sample_sdf<T>(v, p);
    }
}

// Advances a sphere trace by one step. The tests come in the order leave the box, hit, pass
// the limit, spend the budget. Returns the event, or -1 while the trace continues; on an
// event *steps and *t_end receive the step count and the recorded distance.
// With omega > 1 the steps are over-relaxed (the paper's accelerated sphere tracing, Sec. 3.3,
// after Keinert et al.'s enhanced sphere tracing): step omega * sdf; when the sphere of the new
// sample and that of the previous one do not overlap (sdf + previous sdf < step), or when the
// step left the volume box, the step may have passed a surface, so the trace goes back to the
// previous point's plain step and stays plain (omega = 1) for the rest of the ray; the
// discarded sample counts as a step.
template <typename T, bool Relax, bool Idx64>
__device__ __forceinline__ int trace_step(const VolumeView& v, TraceState& st, float eps, int max_steps,
                                          int* steps, float* t_end) {
    constexpr bool kVox = !std::is_same<T, Analytic>::value;
    if constexpr (kVox && !Relax) {
        // A plain voxel-volume trace tests the box once per ray: it started inside, and it
        // leaves where t passes the exit distance, folded with the limit into tstop. The events
        // keep their order (past the limit, then the budget, then leaving the box), and the
        // negated test ends a trace whose t is not a number.
        const float sd = sample_sdf_vox<T, Idx64>(v, fma3(st.t, st.d, st.o));
        if (sd < eps) {
            *steps = st.s + 1;
            *t_end = st.t;
            return kHit;
        }
        st.t = fmaf(sd, v.inv_h, st.t);
        const int s1 = ++st.s;
        if (!(st.t <= st.tstop)) {
            if (st.t > st.tlimit) {
                *steps = s1;
                *t_end = st.tlimit;
                return kPastLimit;
            }
            *steps = s1;
            *t_end = s1 == max_steps ? st.t : st.tlimit;
            return s1 == max_steps ? kExhausted : kLeftVolume;
        }
        if (s1 == max_steps) {
            *steps = max_steps;
            *t_end = st.t;
            return kExhausted;
        }
        return -1;
    }
    const float3 p = fma3(st.t, st.d, st.o);  // voxel coordinate (volumes) or world point (primitives)
    // outside the box, or not a number (the negated test sends NaN out of the volume too)
    const bool outside =
        kVox ? !(p.x >= -0.5f && p.x <= v.gmax[0] && p.y >= -0.5f && p.y <= v.gmax[1] && p.z >= -0.5f &&
                 p.z <= v.gmax[2])
             : (p.x < v.lo[0] || p.x > v.hi[0] || p.y < v.lo[1] || p.y > v.hi[1] || p.z < v.lo[2] || p.z > v.hi[2]);
    if (outside && !(Relax && st.omega > 1.f)) {
        *steps = st.s;
        *t_end = st.tlimit;
        return kLeftVolume;
    }
    // a relaxed step that left the box failed like one whose spheres do not overlap
    float sd = 0.f;
    if (!outside) {
        if constexpr (kVox)
            sd = sample_sdf_vox<T, Idx64>(v, p);
        else
            sd = trace_sample<T>(v, st, p);
    }
    // the step in the trace's units (the SDF holds world distances)
    const float sdu = kVox ? sd * v.inv_h : sd;
    if constexpr (Relax) {
        if (st.omega > 1.f && (outside || sdu + st.prev_r < st.step)) {
            const float back = st.prev_r - st.step;
            st.t += back;
            st.moved = -back;
            st.step = st.prev_r;
            st.omega = 1.f;
            if (++st.s == max_steps) {
                *steps = max_steps;
                *t_end = st.t;
                return kExhausted;
            }
            return -1;
        }
    }
    if (sd < eps) {
        *steps = st.s + 1;
        *t_end = st.t;
        return kHit;
    }
    if constexpr (Relax) {
        st.prev_r = sdu;
        st.step = st.omega * sdu;
        st.moved = st.step;
        st.t += st.step;
    } else if constexpr (kVox) {
        st.t = fmaf(sd, v.inv_h, st.t);
    } else {
        st.moved = sd;
        st.t += sd;
    }
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

// Device-wide pool of sphere traces. Tasks 0..n-1 are claimed from *counter by whole
// warps in batches of kBatch and handed to lanes as they finish their current trace;
// claim(b) runs on every lane of the warp when it has claimed tasks b..b+batch-1 (work
// shared by the whole batch is done there once), init(k, st) sets the origin, direction and
// limit in world units or returns false for a task that needs no trace (it is then
// complete), done(st, event, steps, t) consumes a finished trace (t in world units). A
// voxel-volume trace runs in voxel coordinates between the two. Every lane of the warp must
// take part (full-warp votes).
// A warp hands out new tasks only once at least `refill` of its lanes wait for one (or no
// lane is tracing): a ray lasts a few steps, so refilling lanes one by one would run the
// hand-out on nearly every step for one or two lanes at a time. STEPS: trace steps a lane
// takes per iteration, between two of the warp's votes (one or two). Two made open256's
// primary traces 5 % faster, though a lane whose ray ends after the first step idles for the
// second; they cost cascade512's volumes, and the large shadow pools spill with them at 32
// registers.
template <typename T, bool Relax, bool Idx64, int STEPS = 1, typename Claim, typename Init, typename Done>
__device__ __forceinline__ void trace_pool(const VolumeView& v, uint32_t n, uint32_t* counter, float eps,
                                           int max_steps, float omega, uint32_t batch, int refill, Claim claim,
                                           Init init, Done done) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    uint32_t batch_next = 0, batch_end = 0;  // warp-uniform
    bool need = true, busy = false, dry = false;
    unsigned tracing = 0;  // lanes with a trace in progress, as of the last vote
    TraceState st;
    for (;;) {
        const unsigned want = __ballot_sync(full, need && !dry);
        if (want && (__popc(want) >= refill || !tracing)) {
            if (batch_next >= batch_end) {
                uint32_t b = 0;
                if (lane == 0) b = atomicAdd(counter, batch);
                b = __shfl_sync(full, b, 0);
                batch_next = b;
                batch_end = b + batch;
                claim(b);
            }
            const uint32_t avail = batch_end - batch_next;
            const uint32_t rank = __popc(want & ((1u << lane) - 1u));
            if (need && !dry && rank < avail) {
                const uint32_t k = batch_next + rank;
                need = false;
                if (k >= n) {
                    dry = true;  // the pool is exhausted for this lane
                } else if (init(k, st)) {
                    if constexpr (!std::is_same<T, Analytic>::value) {  // into voxel coordinates
                        st.o = f3(fmaf(st.o.x - v.lo[0], v.inv_h, -0.5f), fmaf(st.o.y - v.lo[1], v.inv_h, -0.5f),
                                  fmaf(st.o.z - v.lo[2], v.inv_h, -0.5f));
                        st.tlimit *= v.inv_h;
                    }
                    st.t = 0.f;
                    st.s = 0;
                    st.last = INFINITY;
                    st.moved = 0.f;
                    st.prev_r = 0.f;
                    st.step = 0.f;
                    st.omega = omega;
                    busy = true;
                    if constexpr (!std::is_same<T, Analytic>::value && !Relax) {
                        if (in_box(v, st.o)) {
                            st.tstop = fminf(st.tlimit, box_exit(v, st.o, st.d));
                        } else {  // outside the volume from the start: it leaves before any sample
                            done(st, kLeftVolume, 0, st.tlimit * v.h);
                            busy = false;
                            need = true;
                        }
                    }
                } else {
                    need = true;  // nothing to trace for this task: take another
                }
            }
            batch_next += min((uint32_t)__popc(want), avail);
        }
        tracing = __ballot_sync(full, busy);
        if (!tracing) {
            if (!__any_sync(full, need && !dry)) break;
            continue;  // every lane waits for a task (its last ones needed no trace): hand out more
        }
        if (busy) {
            int steps;
            float t_end;
            int ev = trace_step<T, Relax, Idx64>(v, st, eps, max_steps, &steps, &t_end);
            if constexpr (STEPS > 1) {
                if (ev < 0) ev = trace_step<T, Relax, Idx64>(v, st, eps, max_steps, &steps, &t_end);
            }
            static_assert(STEPS == 1 || STEPS == 2, "one or two steps between votes");
            if (ev >= 0) {
                if constexpr (!std::is_same<T, Analytic>::value) t_end *= v.h;  // back to world units
                done(st, ev, steps, t_end);
                busy = false;
                need = true;
            }
        }
    }
}

__device__ __forceinline__ uint32_t pool_batch(const UpdateParams& P, int fallback = kBatch) {
    return P.sched.pool_batch > 0 ? (uint32_t)P.sched.pool_batch : (uint32_t)fallback;
}

#ifndef SDFDDGI_REFILL_DEFAULT
#define SDFDDGI_REFILL_DEFAULT 12  // measured on open256 (256 and 32 rays): 1, 4, 8, 12, 16, 24 idle lanes
#endif
__device__ __forceinline__ int pool_refill(const UpdateParams& P) {
    return P.sched.refill > 0 ? min(P.sched.refill, 32) : SDFDDGI_REFILL_DEFAULT;
}

// Direction of ray i of the frame (shared by every probe), stored by the weights stage.
__device__ __forceinline__ float3 ray_dir(const UpdateParams& P, int i) {
    const float4 d = __ldg(P.dirs + i);
    return f3(d.x, d.y, d.z);
}

__device__ __forceinline__ float3 probe_origin(const UpdateParams& P, int p, uint32_t* flags) {
    if (P.states) {
        const sdfddgi_probe_state st = P.states[p];
        *flags = st.flags;
        return f3(st.pos[0], st.pos[1], st.pos[2]);
    }
    const int g = p + P.p_begin;  // grid positions follow the volume's index (a slab starts at p_begin)
    const int ix = g % P.gdims[0], iy = (g / P.gdims[0]) % P.gdims[1], iz = g / (P.gdims[0] * P.gdims[1]);
    *flags = SDFDDGI_PROBE_ACTIVE;
    return f3(fmaf((float)ix, P.gspacing[0], P.gorigin[0]), fmaf((float)iy, P.gspacing[1], P.gorigin[1]),
              fmaf((float)iz, P.gspacing[2], P.gorigin[2]));
}

// Light l's contribution factor at x with normal n: cos for a directional light,
// cos * window / d^2 for a point light; *gate tells whether the light can reach x.
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

// A test that never rejects a light light_scale would gate at x: a point light can reach x
// only if the normal faces it (n . (L - x) > 0 is the sign of light_scale's cosine, its
// distance being positive) and x lies inside the window's range (beyond 1.01 range^2 of squared
// distance the window's q^4 exceeds 1 whatever the float rounding, so the window is 0). The
// hit preparation computes the full factor only for the lights that pass: the same gate bits
// for a fraction of the square roots and divisions.
__device__ __forceinline__ bool light_may_reach(const LightDev& li, float3 x, float3 n) {
    if (li.type == SDFDDGI_LIGHT_DIRECTIONAL) return true;
    const float3 Lv = f3(li.v[0], li.v[1], li.v[2]) - x;
    return dot(n, Lv) > 0.f && dot(Lv, Lv) <= 1.01f * li.range * li.range;
}

// ------------------------------------------------------------------ 1. primary traces
// A claimed batch of tasks lies within one probe whenever R is a multiple of the batch
// size, so the probe's origin and flags are decoded once per batch, by lane 0 into its
// warp's slot; a task outside the slot's probe decodes its own.
template <typename T, bool Relax, bool Idx64, int STEPS>
__global__ void __launch_bounds__(kTraceThreads, 32) primary_kernel(const __grid_constant__ UpdateParams P) {
    __shared__ float4 s_origin[kTraceThreads / 32];  // probe origin, its first task index (bits)
    __shared__ uint32_t s_flags[kTraceThreads / 32];
    const uint32_t n = (uint32_t)P.P * (uint32_t)P.R;
    const int warp = threadIdx.x >> 5;
    trace_pool<T, Relax, Idx64, STEPS>(
        P.vol, n, &P.counters[kPrimaryPool], P.eps_w, P.max_steps, P.omega_primary,
        pool_batch(P, n < kSmallPool ? kBatch / 2 : kBatch), pool_refill(P),
        [&](uint32_t b) {
            __syncwarp();  // every lane has read the previous batch's slot
            if ((threadIdx.x & 31) == 0 && b < n) {
                const uint32_t p = b / (uint32_t)P.R;
                uint32_t flags;
                const float3 o = probe_origin(P, (int)p, &flags);
                s_origin[warp] = make_float4(o.x, o.y, o.z, __uint_as_float(p * (uint32_t)P.R));
                s_flags[warp] = flags;
            }
            __syncwarp();
        },
        [&](uint32_t k, TraceState& st) {
            const float4 so = s_origin[warp];
            const uint32_t rel = k - __float_as_uint(so.w);
            int i;
            uint32_t flags;
            if (rel < (uint32_t)P.R) {
                i = (int)rel;
                flags = s_flags[warp];
                st.o = f3(so.x, so.y, so.z);
            } else {
                i = (int)(k % (uint32_t)P.R);
                st.o = probe_origin(P, (int)(k / (uint32_t)P.R), &flags);
            }
            if (!(flags & SDFDDGI_PROBE_ACTIVE)) {
                P.ray_es[k] = kNoRay;
                return false;
            }
            st.d = ray_dir(P, i);
            st.tlimit = P.tmax_w;
            st.aux = k;
            return true;
        },
        [&](const TraceState& st, int ev, int steps, float t_end) {
            const uint32_t k = checked(st.aux, n, P.vol.fail);
            P.ray_t[k] = t_end;
            P.ray_es[k] = (uint32_t)ev | ((uint32_t)steps << 8);
        });
}

// The ray's record, when records were asked for.
__device__ __forceinline__ void write_record(const UpdateParams& P, uint32_t k, uint32_t es, float4 v, uint32_t lit,
                                             uint32_t owner, uint32_t shadow_steps) {
    const int ev = (int)(es & 0xffu);
    sdfddgi_ray_record rec = {};
    rec.event = (uint8_t)ev;
    if (ev != kNoRay) {
        rec.t = P.ray_t[k];
        rec.L[0] = v.x;
        rec.L[1] = v.y;
        rec.L[2] = v.z;
        rec.lit_mask = lit;
        rec.shadow_steps = is_miss(ev) ? 0u : shadow_steps;
        rec.steps = (uint16_t)(es >> 8);
        rec.material_owner = is_miss(ev) ? 0u : owner;
    }
    P.records[k] = rec;
}

// ------------------------------------------------------------------ 2. hit preparation
constexpr int kPrepRays = 2048;  // rays per hit-preparation CTA, at most
// Rays per hit-preparation CTA for a launch of n rays: the largest power of two from 512 to
// kPrepRays that still gives every SM ctas_per_sm CTAs, so that a small launch (a 32-ray
// update's slab: 128 CTAs of 2048 rays for 148 SMs) fills the GPU with smaller CTAs instead of
// leaving most SMs with one. Measured on open256 (two slab branches): at 32 rays per probe
// 0.344 -> 0.315 ms with 512-ray CTAs; 256 rays per probe unchanged. Asking for two CTAs per
// SM keeps the cascade's 1 M-ray volumes at 2048 rays, where 1024 ran their plain updates
// 1.7 % slower.
inline uint32_t prep_rays(size_t n, int sms, int ctas_per_sm) {
    uint32_t r = (uint32_t)kPrepRays;
    while (r > 512u && n < (size_t)r * (size_t)sms * (size_t)ctas_per_sm) r >>= 1;
    return r;
}

#ifndef SDFDDGI_PREP_CTAS
#define SDFDDGI_PREP_CTAS 4
#endif
// Rays block * rays .. + rays - 1 of one launch's probes.
template <typename T>
__device__ __forceinline__ void prep_body(const UpdateParams& P, uint32_t block, uint32_t rays) {  // rays <= kPrepRays
    // The CTA's rays to shade (hit, or step budget spent) are first gathered into shared
    // memory, so that the shading below runs in full warps instead of one thread per ray
    // with the misses idle.
    __shared__ uint32_t s_rays[kPrepRays];
    __shared__ int s_count;
    const uint32_t n = (uint32_t)P.P * (uint32_t)P.R;
    const uint32_t first = block * rays;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    for (int r = threadIdx.x; r < (int)rays; r += kThreads) {
        const uint32_t k = first + (uint32_t)r;
        bool shade = false;
        if (k < n) {
            const uint32_t es = P.ray_es[k];
            const int ev = (int)(es & 0xffu);
            shade = ev != kNoRay && !is_miss(ev);
            if (!shade) {  // a miss, or a ray of an inactive probe: its value for the gather is final
                const float4 v = ev == kNoRay ? make_float4(0.f, 0.f, 0.f, 0.f)
                                              : make_float4(P.sky[0], P.sky[1], P.sky[2], P.tmax_w);
                P.ray_val[k] = v;
                if (P.records) write_record(P, k, es, v, 0u, 0u, 0u);
            }
        }
        const unsigned want = __ballot_sync(0xffffffffu, shade);
        int base = 0;
        if (lane == 0 && want) base = atomicAdd(&s_count, __popc(want));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (shade) s_rays[base + __popc(want & ((1u << lane) - 1u))] = k;
    }
    __syncthreads();
    const int n_shade = s_count;
    const float inv_pi = 0.318309886183790671538f;
    for (int j0 = 0; j0 < n_shade; j0 += kThreads) {
        const int j = j0 + threadIdx.x;
        uint32_t gate = 0, k = 0;
        float3 x = f3(0.f, 0.f, 0.f), nr = f3(0.f, 0.f, 0.f);  // the hit and its normal
        float4 alb = make_float4(0.f, 0.f, 0.f, 0.f), b = alb;    // albedo + owner bits, base
        if (j < n_shade) {
            k = s_rays[j];
            const VolumeView& V = P.vol;
            const int p = (int)(k / (uint32_t)P.R), i = (int)(k % (uint32_t)P.R);
            uint32_t flags;
            const float3 o = probe_origin(P, p, &flags);
            const float3 d = ray_dir(P, i);
            const float t = P.ray_t[k];
            x = fma3(t, d, o);
            const float hh = 0.5f * V.h;
            const float gx = sample_sdf<T>(V, f3(x.x + hh, x.y, x.z)) - sample_sdf<T>(V, f3(x.x - hh, x.y, x.z));
            const float gy = sample_sdf<T>(V, f3(x.x, x.y + hh, x.z)) - sample_sdf<T>(V, f3(x.x, x.y - hh, x.z));
            const float gz = sample_sdf<T>(V, f3(x.x, x.y, x.z + hh)) - sample_sdf<T>(V, f3(x.x, x.y, x.z - hh));
            const float glen = sqrtf(gx * gx + gy * gy + gz * gz);
            // a gradient that is zero or not finite (an SDF holding infinities or NaN near the
            // hit) gives no normal: the reversed ray direction stands in
            nr = glen > 0.f && glen < INFINITY ? f3(gx / glen, gy / glen, gz / glen) : f3(-d.x, -d.y, -d.z);
            float3 albedo, emission;
            uint32_t owner = 0;  // scenes of primitives: the caller's index + 1 of the material's primitive
            if constexpr (std::is_same<T, Analytic>::value) {
                int slot;
                analytic_sdf(V, x, INFINITY, nullptr, &slot);
                const PrimDev& q = V.prims[slot];
                albedo = f3(q.albedo[0], q.albedo[1], q.albedo[2]);
                emission = f3(q.emission[0], q.emission[1], q.emission[2]);
                owner = (uint32_t)q.index + 1u;
            } else {
                sample_material(V, x, &albedo, &emission);
            }
            float3 ind = f3(0.f, 0.f, 0.f);
            if (P.k_bounce != 0.f)
                ind = interpolate_irradiance(P.gdims, P.gorigin, P.gspacing, P.look_irr, P.look_valid, x, nr,
                                             P.vol.fail);
            for (int l = 0; l < P.n_lights; ++l) {
                if (!light_may_reach(P.lights[l], x, nr)) continue;
                bool g;
                light_scale(P.lights[l], x, nr, &g);
                if (g) gate |= 1u << l;
            }
            alb = make_float4(albedo.x, albedo.y, albedo.z, __uint_as_float(owner));
            b = make_float4(emission.x + albedo.x * P.k_bounce * ind.x, emission.y + albedo.y * P.k_bounce * ind.y,
                            emission.z + albedo.z * P.k_bounce * ind.z, 0.f);
            if (!gate) {  // no light can reach the hit: its value (the finalize rule's with no light) is final
                const float4 v = make_float4(fmaf(alb.x * inv_pi, 0.f, b.x), fmaf(alb.y * inv_pi, 0.f, b.y),
                                             fmaf(alb.z * inv_pi, 0.f, b.z), fminf(t, P.tmax_w));
                P.ray_val[k] = v;
                if (P.records) write_record(P, k, P.ray_es[k], v, 0u, owner, 0u);
            }
        }
        // append this warp's (ray, light) pairs to the task list with one atomic, and its rays
        // with tasks to the finalize list with another
        const int cnt = __popc(gate);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (total == 0) continue;
        const unsigned fin = __ballot_sync(0xffffffffu, gate != 0u);
        uint32_t base = 0, fbase = 0;
        if (lane == 31) {
            base = atomicAdd(&P.counters[kTaskCount], (uint32_t)total);
            fbase = atomicAdd(&P.counters[kFinCount], (uint32_t)__popc(fin));
        }
        base = __shfl_sync(0xffffffffu, base, 31);
        fbase = __shfl_sync(0xffffffffu, fbase, 31);
        uint32_t pos = base + (uint32_t)(incl - cnt);
        if (base + (uint32_t)total > P.task_capacity) {  // cannot happen with capacity P*R*lights
            if (lane == 31) atomicOr(&P.counters[kFailWord], kFailTasks);
            gate = 0;  // no task: the ray is finalized with no light (the update is flagged invalid)
            pos = 0;
        }
        uint32_t entry = 0;  // the ray's finalize-list position, which its shadow tasks carry
        if (fin & (1u << lane)) {  // the finalize list's entry: the ray, and its shading in list order
            const uint32_t f = checked(fbase + (uint32_t)__popc(fin & ((1u << lane) - 1u)), n, P.vol.fail);
            P.fin_list[f] = k;
            P.ray_alb[f] = make_float4(alb.x, alb.y, alb.z, __uint_as_float(gate));
            P.ray_base[f] = make_float4(b.x, b.y, b.z, __uint_as_float(pos));
            P.ray_lit[f] = 0;  // the shadow traces set the visible lights' bits
            if (P.records) {
                P.ray_ssteps[f] = 0;
                P.ray_n[k] = make_float4(alb.w, 0.f, 0.f, 0.f);  // the owner, for the record
            }
            entry = f;
        }
        const float3 so = fma3(P.bias_w, nr, x);  // the shadow rays' origin: the hit lifted off the surface
        while (gate) {
            const int l = __ffs(gate) - 1;
            gate &= gate - 1;
            bool g;
            P.task_scale[pos] = light_scale(P.lights[l], x, nr, &g);  // the factor the gating saw
            P.tasks[pos++] = make_float4(so.x, so.y, so.z, __uint_as_float((entry << 5) | (uint32_t)l));
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads, SDFDDGI_PREP_CTAS) prep_kernel(const __grid_constant__ UpdateParams P,
                                                                          uint32_t rays) {
    prep_body<T>(P, blockIdx.x, min(rays, (uint32_t)kPrepRays));
}

// ------------------------------------------------------------------ 3. shadow traces
// SMALL: a launch of fewer than kSmallShadowRays rays, whose small pool runs 24 CTAs per SM
// of up to 40 registers and takes two trace steps between the warps' votes (with 32 CTAs
// of 32 registers two steps spill): 32-ray updates' shadow stage 0.0775 -> 0.0716 ms, while
// 256-ray updates were slower that way (0.2014 -> 0.209 ms).
template <typename T, bool Relax, bool Idx64, bool SMALL>
__global__ void __launch_bounds__(kTraceThreads, SMALL ? 24 : 32) shadow_kernel(const __grid_constant__ UpdateParams P) {
    const uint32_t n = min(P.counters[kTaskCount], P.task_capacity);
    trace_pool<T, Relax, Idx64, SMALL ? 2 : 1>(
        P.vol, n, &P.counters[kShadowPool], P.eps_w, P.max_steps, P.omega_shadow,
        pool_batch(P, n < kSmallPool ? kShadowBatch / 2 : kShadowBatch),  // n: the tasks the preparation made
        pool_refill(P),
        [](uint32_t) {},
        [&](uint32_t j, TraceState& st) {
            const float4 task = P.tasks[j];
            const uint32_t tk = __float_as_uint(task.w);
            const int l = (int)(tk & 31u);
            st.o = f3(task.x, task.y, task.z);
            const LightDev& li = P.lights[l];
            if (li.type == SDFDDGI_LIGHT_DIRECTIONAL) {
                st.d = f3(li.v[0], li.v[1], li.v[2]);
                st.tlimit = P.tmax_w;
            } else {
                const float3 Ls = f3(li.v[0], li.v[1], li.v[2]) - st.o;
                const float ds = sqrtf(dot(Ls, Ls));
                st.d = (1.f / ds) * Ls;
                st.tlimit = ds;
            }
            st.aux = tk;
            return true;
        },
        [&](const TraceState& st, int ev, int steps, float) {
            const uint32_t f = checked(st.aux >> 5, (size_t)P.P * P.R, P.vol.fail);  // the hit's finalize entry
            if (P.records) atomicAdd(&P.ray_ssteps[f], (uint32_t)steps);
            if (is_miss(ev)) atomicOr(&P.ray_lit[f], 1u << (st.aux & 31u));  // hit or exhausted: occluded
        });
}

// ------------------------------------------------------------------ merged launches (batched form)
// The part of a merged launch that x (a task, CTA or block index) falls in: the last volume
// whose part begins at or before x (an empty part is skipped, as the next one begins where it
// ends).
__device__ __forceinline__ int merged_part(const uint32_t* begin, int n, uint32_t x) {
    int v = 0;
#pragma unroll
    for (int i = 1; i < kMaxMerged; ++i) v += (i < n && x >= begin[i]) ? 1 : 0;
    return v;
}

// Primary traces of every volume from one pool. A claimed batch lies within one volume (the
// parts are padded to the batch); its volume and, as in primary_kernel, its probe are decoded
// once per claim. A ray's payload is its merged task index, from which the completion finds
// the volume again.
template <typename T, bool Relax, bool Idx64>
__global__ void __launch_bounds__(kTraceThreads, 32) primary_merged_kernel(const __grid_constant__ MergedParams M) {
    __shared__ float4 s_origin[kTraceThreads / 32];  // probe origin, its first merged task index (bits)
    __shared__ uint32_t s_flags[kTraceThreads / 32];
    __shared__ int s_vol[kTraceThreads / 32];
    const UpdateParams& P0 = M.p[0];
    const uint32_t n = M.ray_begin[M.n];
    const int warp = threadIdx.x >> 5;
    trace_pool<T, Relax, Idx64>(
        P0.vol, n, &P0.counters[kPrimaryPool], P0.eps_w, P0.max_steps, P0.omega_primary, M.primary_batch,
        pool_refill(P0),
        [&](uint32_t b) {
            __syncwarp();
            if ((threadIdx.x & 31) == 0 && b < n) {
                const int v = merged_part(M.ray_begin, M.n, b);
                const UpdateParams& P = M.p[v];
                const uint32_t k = b - M.ray_begin[v];
                uint32_t flags = 0;
                float3 o = f3(0.f, 0.f, 0.f);
                const uint32_t p = k / (uint32_t)P.R;
                if (k < (uint32_t)P.P * (uint32_t)P.R) o = probe_origin(P, (int)p, &flags);
                s_origin[warp] = make_float4(o.x, o.y, o.z, __uint_as_float(M.ray_begin[v] + p * (uint32_t)P.R));
                s_flags[warp] = flags;
                s_vol[warp] = v;
            }
            __syncwarp();
        },
        [&](uint32_t kg, TraceState& st) {
            const int v = s_vol[warp];
            const UpdateParams& P = M.p[v];
            const uint32_t k = kg - M.ray_begin[v];
            if (k >= (uint32_t)P.P * (uint32_t)P.R) return false;  // padding of the volume's part
            const float4 so = s_origin[warp];
            const uint32_t rel = kg - __float_as_uint(so.w);
            int i;
            uint32_t flags;
            if (rel < (uint32_t)P.R) {
                i = (int)rel;
                flags = s_flags[warp];
                st.o = f3(so.x, so.y, so.z);
            } else {
                i = (int)(k % (uint32_t)P.R);
                st.o = probe_origin(P, (int)(k / (uint32_t)P.R), &flags);
            }
            if (!(flags & SDFDDGI_PROBE_ACTIVE)) {
                P.ray_es[k] = kNoRay;
                return false;
            }
            st.d = ray_dir(P, i);
            st.tlimit = P.tmax_w;
            st.aux = kg;
            return true;
        },
        [&](const TraceState& st, int ev, int steps, float t_end) {
            const int v = merged_part(M.ray_begin, M.n, st.aux);
            const UpdateParams& P = M.p[v];
            const uint32_t k = checked(st.aux - M.ray_begin[v], (size_t)P.P * P.R, P.vol.fail);
            P.ray_t[k] = t_end;
            P.ray_es[k] = (uint32_t)ev | ((uint32_t)steps << 8);
        });
}

// Shadow traces of every volume from one pool: volume v's tasks follow the earlier volumes'
// (each part padded to the batch), laid out by every CTA from the task counts the hit
// preparation left. A task's payload is its merged index; the completion reads the task's
// ray and light from the volume's list again.
template <typename T, bool Relax, bool Idx64>
__global__ void __launch_bounds__(kTraceThreads, 32) shadow_merged_kernel(const __grid_constant__ MergedParams M) {
    __shared__ uint32_t s_begin[kMaxMerged + 1], s_count[kMaxMerged];
    if (threadIdx.x == 0) {
        uint32_t b = 0;
        for (int v = 0; v < M.n; ++v) {
            const uint32_t c = min(M.p[v].counters[kTaskCount], M.p[v].task_capacity);
            s_begin[v] = b;
            s_count[v] = c;
            b += (c + M.shadow_batch - 1) / M.shadow_batch * M.shadow_batch;
        }
        s_begin[M.n] = b;
    }
    __syncthreads();
    const UpdateParams& P0 = M.p[0];
    const uint32_t n = s_begin[M.n];
    trace_pool<T, Relax, Idx64>(
        P0.vol, n, &P0.counters[kShadowPool], P0.eps_w, P0.max_steps, P0.omega_shadow, M.shadow_batch,
        pool_refill(P0),
        [](uint32_t) {},
        [&](uint32_t jg, TraceState& st) {
            const int v = merged_part(s_begin, M.n, jg);
            const uint32_t j = jg - s_begin[v];
            if (j >= s_count[v]) return false;  // padding of the volume's part
            const UpdateParams& P = M.p[v];
            const float4 task = P.tasks[j];
            const int l = (int)(__float_as_uint(task.w) & 31u);
            st.o = f3(task.x, task.y, task.z);
            const LightDev& li = P.lights[l];
            if (li.type == SDFDDGI_LIGHT_DIRECTIONAL) {
                st.d = f3(li.v[0], li.v[1], li.v[2]);
                st.tlimit = P.tmax_w;
            } else {
                const float3 Ls = f3(li.v[0], li.v[1], li.v[2]) - st.o;
                const float ds = sqrtf(dot(Ls, Ls));
                st.d = (1.f / ds) * Ls;
                st.tlimit = ds;
            }
            st.aux = jg;
            return true;
        },
        [&](const TraceState& st, int ev, int steps, float) {
            const int v = merged_part(s_begin, M.n, st.aux);
            const UpdateParams& P = M.p[v];
            const uint32_t j = checked(st.aux - s_begin[v], P.task_capacity, P.vol.fail);
            const uint32_t tk = __float_as_uint(P.tasks[j].w);
            const uint32_t f = checked(tk >> 5, (size_t)P.P * P.R, P.vol.fail);  // the hit's finalize entry
            if (P.records) atomicAdd(&P.ray_ssteps[f], (uint32_t)steps);
            if (is_miss(ev)) atomicOr(&P.ray_lit[f], 1u << (tk & 31u));  // hit or exhausted: occluded
        });
}

template <typename T>
__global__ void __launch_bounds__(kThreads, SDFDDGI_PREP_CTAS) prep_merged_kernel(const __grid_constant__ MergedParams M) {
    const int v = merged_part(M.prep_begin, M.n, blockIdx.x);
    prep_body<T>(M.p[v], blockIdx.x - M.prep_begin[v], min(M.prep_rays[v], (uint32_t)kPrepRays));
}

// ------------------------------------------------------------------ 4. gather (Eq. 3)
// The texel weights max(0, u_j . d_i)^e depend on the frame's ray set only, so they are
// computed once per update: row i (ray) x column j (texel, irradiance first), plus each
// column's sum, in ray order. Directions and cosines are taken in double-float arithmetic
// (csrc/dfloat.cuh) and each weight rounded to float once, so that a weight keeps its
// relative accuracy down to the cosine cutoff; the traces read the directions rounded to
// float from the same computation.
template <int PEXP, bool Dirs>
__device__ __forceinline__ void weights_body(const UpdateParams& P, int i) {  // ray i, one texel per thread
    __shared__ dfloat s_d[3];
    const int j = threadIdx.x;
    if (j == 0) {
        dfloat d[3];
        df_ray_direction(i, P.R, P.rot_dev ? P.rot_dev : P.rot, d);
        s_d[0] = d[0];
        s_d[1] = d[1];
        s_d[2] = d[2];
        if (Dirs) P.dirs[i] = make_float4(d[0].hi, d[1].hi, d[2].hi, 0.f);
    }
    __syncthreads();
    if (j >= kTexels) return;
    const bool irr = j < kIrrTexels;
    const int jj = irr ? j : j - kIrrTexels, n = irr ? kIrrN : kDepN;
    dfloat u[3];
    df_texel_direction(jj % n, jj / n, n, u);
    const dfloat d[3] = {s_d[0], s_d[1], s_d[2]};
    const dfloat c = df_dot(u, d);
    float w = 0.f;
    if (c.hi > 0.f) w = irr ? c.hi : df_pow(c, PEXP == 50 ? 50 : P.depth_exp).hi;
    P.weights[(size_t)i * kTexels + j] = w;
}

template <int PEXP, bool Dirs>
__global__ void __launch_bounds__(kThreads) weights_kernel(const __grid_constant__ UpdateParams P) {
    weights_body<PEXP, Dirs>(P, blockIdx.x);  // one ray per block
}

// The frame's R ray directions alone (what the traces need of stage 0), for updates whose
// texel weights are computed beside the traces; the same rounding as weights_kernel's.
__global__ void __launch_bounds__(kThreads) ray_dirs_kernel(const __grid_constant__ UpdateParams P) {
    const int i = blockIdx.x * kThreads + threadIdx.x;
    if (i >= P.R) return;
    dfloat d[3];
    df_ray_direction(i, P.R, P.rot_dev ? P.rot_dev : P.rot, d);
    P.dirs[i] = make_float4(d[0].hi, d[1].hi, d[2].hi, 0.f);
}

// Column sums of the texel weights, accumulated in double-float in ray order.
__global__ void __launch_bounds__(kThreads) weight_sums_kernel(const __grid_constant__ UpdateParams P) {
    const int j = threadIdx.x;
    if (j >= kTexels) return;
    dfloat sw = df(0.f);
    for (int i = 0; i < P.R; ++i) sw = sw + df(P.weights[(size_t)i * kTexels + j]);
    P.weights[(size_t)P.R * kTexels + j] = sw.hi;
}

// The hits with shadow tasks (the finalize list, written by the hit preparation, which
// completes every other ray): radiance = base + albedo / pi * the sum over visible lights, in
// light order, of the light's factor at the hit (stored with its task) times its rgb, and the
// clamped distance; written over the ray's slot of the gather's values, and the ray's record
// when records were asked for. Grid-stride over the list.
__device__ __forceinline__ void finalize_body(const UpdateParams& P) {
    const uint32_t n = (uint32_t)P.P * (uint32_t)P.R;
    const uint32_t count = min(P.counters[kFinCount], n);
    const float inv_pi = 0.318309886183790671538f;
    for (uint32_t j = blockIdx.x * kThreads + threadIdx.x; j < count; j += gridDim.x * kThreads) {
        const uint32_t k = checked(P.fin_list[j], n, P.vol.fail);
        const float4 a = P.ray_alb[j], b = P.ray_base[j];  // in list order: albedo + gate mask, base + first task
        uint32_t gate = __float_as_uint(a.w), pos = __float_as_uint(b.w);
        const uint32_t lit = P.ray_lit[j];
        float3 direct = f3(0.f, 0.f, 0.f);
        while (gate) {
            const int l = __ffs(gate) - 1;
            gate &= gate - 1;
            if ((lit >> l) & 1u) {
                const float sc = P.task_scale[checked(pos, P.task_capacity, P.vol.fail)];
                direct = fma3(sc, f3(P.lights[l].rgb[0], P.lights[l].rgb[1], P.lights[l].rgb[2]), direct);
            }
            ++pos;
        }
        const uint32_t owner = P.records ? __float_as_uint(P.ray_n[k].x) : 0u;  // read before ray_val overwrites it
        const float4 v = make_float4(fmaf(a.x * inv_pi, direct.x, b.x), fmaf(a.y * inv_pi, direct.y, b.y),
                                     fmaf(a.z * inv_pi, direct.z, b.z), fminf(P.ray_t[k], P.tmax_w));
        P.ray_val[k] = v;
        if (P.records) write_record(P, k, P.ray_es[k], v, lit, owner, P.ray_ssteps[j]);
    }
}

__global__ void __launch_bounds__(kThreads) finalize_kernel(const __grid_constant__ UpdateParams P) { finalize_body(P); }

// The merged launches of the texel weights (one block per ray of every volume, all with the
// same depth exponent) and of the finalize stage (each volume's list in turn, grid-stride).
template <int PEXP>
__global__ void __launch_bounds__(kThreads) weights_merged_kernel(const __grid_constant__ MergedParams M) {
    const int v = merged_part(M.dir_begin, M.n, blockIdx.x);
    weights_body<PEXP, true>(M.p[v], (int)(blockIdx.x - M.dir_begin[v]));
}

__global__ void __launch_bounds__(kThreads) finalize_merged_kernel(const __grid_constant__ MergedParams M) {
    for (int v = 0; v < M.n; ++v) finalize_body(M.p[v]);
}

// G probes per CTA. Stage a: the rays' values of the G probes go to shared memory (one
// float4 per ray and probe). Stage b: thread j owns texel j of all G probes and
// accumulates sum_i W[i][j] v_i over the rays, reading W coalesced and each v_i as a
// shared-memory broadcast. Stage c: normalise by the column sum, mix with last frame's
// texel, fill the borders, store each map contiguously.
template <int G>
__global__ void __launch_bounds__(kThreads) gather_kernel(const __grid_constant__ UpdateParams P) {
    extern __shared__ float4 s_val[];  // [R][G]
    __shared__ float4 s_irr[G][kIrrT * kIrrT];
    __shared__ __align__(16) float2 s_dep[G][kDepT * kDepT];  // stored out as float4 pairs
    __shared__ float s_hyst[G];
    __shared__ uint32_t s_flags[G];
    __shared__ float3 s_o[G];

    const int tid = threadIdx.x, nt = blockDim.x;
    const int p0 = blockIdx.x * G;
    const int ng = min(G, P.P - p0);
    if (tid < G) {
        uint32_t flags = 0;
        float3 o = f3(0.f, 0.f, 0.f);
        if (tid < ng) o = probe_origin(P, p0 + tid, &flags);
        s_o[tid] = o;
        s_flags[tid] = flags;
        s_hyst[tid] = (tid < ng && P.prev_valid[p0 + tid] && !(flags & SDFDDGI_PROBE_REJECT_HISTORY)) ? P.hyst : 0.f;
    }
    __syncthreads();

    // a. the rays' values, [ray][probe]
    for (int e = tid; e < P.R * G; e += nt) {
        const int i = e / G, g = e % G;
        s_val[e] = g < ng ? P.ray_val[(size_t)(p0 + g) * P.R + i] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();

    // b. texel j of every probe: sum over rays of W[i][j] * value
    if (tid < kTexels) {
        const int j = tid;
        const bool irr = j < kIrrTexels;
        float acc[G][3];
#pragma unroll
        for (int g = 0; g < G; ++g) acc[g][0] = acc[g][1] = acc[g][2] = 0.f;
        const float* W = P.weights + j;
        if (irr) {
            for (int i = 0; i < P.R; ++i) {
                const float w = __ldg(W + (size_t)i * kTexels);
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const float4 v = s_val[i * G + g];
                    acc[g][0] = fmaf(w, v.x, acc[g][0]);
                    acc[g][1] = fmaf(w, v.y, acc[g][1]);
                    acc[g][2] = fmaf(w, v.z, acc[g][2]);
                }
            }
        } else {
            for (int i = 0; i < P.R; ++i) {
                const float w = __ldg(W + (size_t)i * kTexels);
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const float t = s_val[i * G + g].w;
                    acc[g][0] = fmaf(w, t, acc[g][0]);
                    acc[g][1] = fmaf(w, t * t, acc[g][1]);
                }
            }
        }
        // c. normalise and mix with the previous texel
        const float sw = __ldg(P.weights + (size_t)P.R * kTexels + j);
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (g >= ng) break;
            const size_t p = (size_t)(p0 + g);
            const float hyst = s_hyst[g], keep = 1.f - hyst;
            if (irr) {
                const int a = j % kIrrN, b = j / kIrrN, k = (b + 1) * kIrrT + (a + 1);
                float4 out = __ldg(P.prev_irr + p * (kIrrT * kIrrT) + k);
                if ((s_flags[g] & SDFDDGI_PROBE_ACTIVE) && sw > 0.f) {
                    const float inv = 1.f / sw;
                    out.x = fmaf(hyst, out.x, keep * (acc[g][0] * inv));
                    out.y = fmaf(hyst, out.y, keep * (acc[g][1] * inv));
                    out.z = fmaf(hyst, out.z, keep * (acc[g][2] * inv));
                    out.w = 1.f;
                }
                s_irr[g][k] = out;
            } else {
                const int jj = j - kIrrTexels, a = jj % kDepN, b = jj / kDepN, k = (b + 1) * kDepT + (a + 1);
                float2 out = __ldg(P.prev_depth + p * (kDepT * kDepT) + k);
                if ((s_flags[g] & SDFDDGI_PROBE_ACTIVE) && sw > 0.f) {
                    const float inv = 1.f / sw;
                    out.x = fmaf(hyst, out.x, keep * (acc[g][0] * inv));
                    out.y = fmaf(hyst, out.y, keep * (acc[g][1] * inv));
                }
                s_dep[g][k] = out;
            }
        }
    }
    __syncthreads();

    // borders from the interior (inactive probes: copy of the old map, borders included)
    for (int e = tid; e < ng * kIrrT * kIrrT; e += nt) {
        const int g = e / (kIrrT * kIrrT), k = e % (kIrrT * kIrrT);
        const int y = k / kIrrT, x = k % kIrrT;
        const int2 s = border_source(y, x, kIrrN);
        if (!(s_flags[g] & SDFDDGI_PROBE_ACTIVE)) {
            s_irr[g][k] = __ldg(P.prev_irr + (size_t)(p0 + g) * (kIrrT * kIrrT) + k);
        } else if (s.x != y || s.y != x) {
            s_irr[g][k] = s_irr[g][s.x * kIrrT + s.y];
        }
    }
    for (int e = tid; e < ng * kDepT * kDepT; e += nt) {
        const int g = e / (kDepT * kDepT), k = e % (kDepT * kDepT);
        const int y = k / kDepT, x = k % kDepT;
        const int2 s = border_source(y, x, kDepN);
        if (!(s_flags[g] & SDFDDGI_PROBE_ACTIVE)) {
            s_dep[g][k] = __ldg(P.prev_depth + (size_t)(p0 + g) * (kDepT * kDepT) + k);
        } else if (s.x != y || s.y != x) {
            s_dep[g][k] = s_dep[g][s.x * kDepT + s.y];
        }
    }
    __syncthreads();
    float4* cur_i = P.cur_irr + (size_t)p0 * (kIrrT * kIrrT);
    for (int e = tid; e < ng * kIrrT * kIrrT; e += nt) cur_i[e] = (&s_irr[0][0])[e];
    float4* cur_d4 = reinterpret_cast<float4*>(P.cur_depth + (size_t)p0 * (kDepT * kDepT));
    const float4* sd4 = reinterpret_cast<const float4*>(&s_dep[0][0]);
    for (int e = tid; e < ng * kDepT * kDepT / 2; e += nt) cur_d4[e] = sd4[e];
    if (tid < ng) P.cur_valid[p0 + tid] = (s_flags[tid] & SDFDDGI_PROBE_ACTIVE) ? 1 : P.prev_valid[p0 + tid];
}

// ------------------------------------------------------------------ launch
// One-time set-up per device, made outside any stream capture (volume creation calls it):
// the SM count, the occupancy limits of the persistent pool kernels and the dynamic
// shared-memory limits of the gathers. Updates then make no such calls, so that they can
// be captured into a graph.
struct DeviceSetup {
    bool done = false;
    cudaError_t err = cudaSuccess;
    int sms = 0;
    int occ_primary[2][3] = {};  // [plain, relaxed][float, __half, Analytic]
    int occ_shadow[2][3] = {};
    int occ_shadow_small[2] = {};  // [float, __half], plain traces
    int occ_primary_merged[2][2] = {};  // [plain, relaxed][float, __half]
    int occ_shadow_merged[2][2] = {};
};

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
DeviceSetup g_setup[kMaxDevices];

template <typename T>
constexpr int type_slot() { return std::is_same<T, float>::value ? 0 : (std::is_same<T, __half>::value ? 1 : 2); }

int occupancy(const void* kernel, int threads = kThreads) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, 0) != cudaSuccess) return 1;
    return max(1, occ);
}

}  // namespace

cudaError_t prepare_update_kernels(const DeviceSetup** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup& s = g_setup[dev];
    if (!s.done) {
        s.err = cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, dev);
        s.occ_primary[0][0] = occupancy((const void*)primary_kernel<float, false, false, 2>, kTraceThreads);
        s.occ_primary[0][1] = occupancy((const void*)primary_kernel<__half, false, false, 2>, kTraceThreads);
        s.occ_primary[0][2] = occupancy((const void*)primary_kernel<Analytic, false, false, 1>, kTraceThreads);
        s.occ_shadow[0][0] = occupancy((const void*)shadow_kernel<float, false, false, false>, kTraceThreads);
        s.occ_shadow[0][1] = occupancy((const void*)shadow_kernel<__half, false, false, false>, kTraceThreads);
        s.occ_shadow[0][2] = occupancy((const void*)shadow_kernel<Analytic, false, false, false>, kTraceThreads);
        s.occ_shadow_small[0] = occupancy((const void*)shadow_kernel<float, false, false, true>, kTraceThreads);
        s.occ_shadow_small[1] = occupancy((const void*)shadow_kernel<__half, false, false, true>, kTraceThreads);
        s.occ_primary[1][0] = occupancy((const void*)primary_kernel<float, true, false, 1>, kTraceThreads);
        s.occ_primary[1][1] = occupancy((const void*)primary_kernel<__half, true, false, 1>, kTraceThreads);
        s.occ_primary[1][2] = occupancy((const void*)primary_kernel<Analytic, true, false, 1>, kTraceThreads);
        s.occ_shadow[1][0] = occupancy((const void*)shadow_kernel<float, true, false, false>, kTraceThreads);
        s.occ_shadow[1][1] = occupancy((const void*)shadow_kernel<__half, true, false, false>, kTraceThreads);
        s.occ_shadow[1][2] = occupancy((const void*)shadow_kernel<Analytic, true, false, false>, kTraceThreads);
        s.occ_primary_merged[0][0] = occupancy((const void*)primary_merged_kernel<float, false, false>, kTraceThreads);
        s.occ_primary_merged[0][1] = occupancy((const void*)primary_merged_kernel<__half, false, false>, kTraceThreads);
        s.occ_primary_merged[1][0] = occupancy((const void*)primary_merged_kernel<float, true, false>, kTraceThreads);
        s.occ_primary_merged[1][1] = occupancy((const void*)primary_merged_kernel<__half, true, false>, kTraceThreads);
        s.occ_shadow_merged[0][0] = occupancy((const void*)shadow_merged_kernel<float, false, false>, kTraceThreads);
        s.occ_shadow_merged[0][1] = occupancy((const void*)shadow_merged_kernel<__half, false, false>, kTraceThreads);
        s.occ_shadow_merged[1][0] = occupancy((const void*)shadow_merged_kernel<float, true, false>, kTraceThreads);
        s.occ_shadow_merged[1][1] = occupancy((const void*)shadow_merged_kernel<__half, true, false>, kTraceThreads);
        // the SIMT gathers stage [R][G] values: at most 32 KiB for the G chosen per R
        for (const void* k : {(const void*)gather_kernel<8>, (const void*)gather_kernel<4>, (const void*)gather_kernel<2>})
            if (s.err == cudaSuccess) s.err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 32 << 10);
        if (s.err == cudaSuccess) s.err = prepare_gather_tc();
        s.done = true;
    }
    if (out) *out = &s;
    return s.err;
}

// Grid of a persistent pool kernel: resident CTAs per SM (the occupancy limit, or fewer
// when the schedule asks) times the SM count.
static int persistent_blocks(const DeviceSetup& s, int occ, int want_per_sm) {
    const int per_sm = want_per_sm > 0 ? min(occ, want_per_sm) : occ;
    return max(1, s.sms * per_sm);
}

template <int G>
static cudaError_t launch_gather(const UpdateParams& p, cudaStream_t stream) {
    const size_t smem = (size_t)p.R * G * sizeof(float4);  // at most 32 KiB for the G chosen below
    gather_kernel<G><<<(p.P + G - 1) / G, kThreads, smem, stream>>>(p);
    return cudaGetLastError();
}

// Stage s (0 primary traces, 1 hit preparation, 2 shadow traces, 3 finalize + gather) of one
// launch's probes (the volume, or one slab of it) on `stream`, followed by stage event s + 2
// when ev is given. With pack, the tensor-core gather first packs the weight image (slab
// branches find it packed before the fork).
template <typename T>
static cudaError_t launch_stage(const UpdateParams& p, const DeviceSetup& setup, int s, cudaStream_t stream,
                                cudaEvent_t const* ev, bool pack) {
    const int rp = p.omega_primary > 1.f ? 1 : 0, rs = p.omega_shadow > 1.f ? 1 : 0;
    const uint32_t n = (uint32_t)p.P * (uint32_t)p.R;
    cudaError_t e = cudaSuccess;
    // the quad-index arithmetic of the traces (same addresses): the 32-bit row form unless the
    // schedule asks for the 64-bit one (the batch autotuner tries both)
    const bool i64 = p.sched.index == 2;
    if (s == 0) {
        const int g = persistent_blocks(setup, setup.occ_primary[rp][type_slot<T>()], p.sched.blocks_per_sm);
        // plain voxel traces take two steps between votes unless the schedule asks for one
        constexpr int kTwo = std::is_same<T, Analytic>::value ? 1 : 2;
        if (rp)
            i64 ? primary_kernel<T, true, true, 1><<<g, kTraceThreads, 0, stream>>>(p)
                : primary_kernel<T, true, false, 1><<<g, kTraceThreads, 0, stream>>>(p);
        else if (p.sched.steps != 1)
            i64 ? primary_kernel<T, false, true, kTwo><<<g, kTraceThreads, 0, stream>>>(p)
                : primary_kernel<T, false, false, kTwo><<<g, kTraceThreads, 0, stream>>>(p);
        else
            i64 ? primary_kernel<T, false, true, 1><<<g, kTraceThreads, 0, stream>>>(p)
                : primary_kernel<T, false, false, 1><<<g, kTraceThreads, 0, stream>>>(p);
    } else if (s == 1) {
        const uint32_t rays = prep_rays(n, setup.sms, 2);
        prep_kernel<T><<<(n + rays - 1) / rays, kThreads, 0, stream>>>(p, rays);
    } else if (s == 2) {
        // a launch of fewer than kSmallShadowRays rays with plain voxel traces takes the shadow
        // kernel of 24 CTAs per SM and two steps between votes
        constexpr bool kVoxel = !std::is_same<T, Analytic>::value;
        if (kVoxel && !rs && (size_t)p.P * (size_t)p.R < kSmallShadowRays) {
            if constexpr (kVoxel) {
                const int g = persistent_blocks(setup, setup.occ_shadow_small[type_slot<T>()], p.sched.blocks_per_sm);
                i64 ? shadow_kernel<T, false, true, true><<<g, kTraceThreads, 0, stream>>>(p)
                    : shadow_kernel<T, false, false, true><<<g, kTraceThreads, 0, stream>>>(p);
            }
        } else {
            const int g = persistent_blocks(setup, setup.occ_shadow[rs][type_slot<T>()], p.sched.blocks_per_sm);
            if (rs)
                i64 ? shadow_kernel<T, true, true, false><<<g, kTraceThreads, 0, stream>>>(p)
                    : shadow_kernel<T, true, false, false><<<g, kTraceThreads, 0, stream>>>(p);
            else
                i64 ? shadow_kernel<T, false, true, false><<<g, kTraceThreads, 0, stream>>>(p)
                    : shadow_kernel<T, false, false, false><<<g, kTraceThreads, 0, stream>>>(p);
        }
    } else {
        finalize_kernel<<<max(1, min((int)((n + kThreads - 1) / kThreads), 8 * setup.sms)), kThreads, 0, stream>>>(p);
        if (gather_tc_supported(p) && p.sched.gather != 2)
            e = launch_gather_tc(p, stream, pack);
        else if (p.R <= 256)  // probes per gather CTA: as many as keep [R][G] values within 32 KiB
            e = launch_gather<8>(p, stream);
        else if (p.R <= 512)
            e = launch_gather<4>(p, stream);
        else
            e = launch_gather<2>(p, stream);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[s + 2], stream);
    return e;
}

// Slab c of K: the z-layers [c*gz/K, (c+1)*gz/K) of the probe grid, with every per-probe and
// per-ray pointer moved to its first probe, its own counters and its own part of the task list.
static UpdateParams slab_params(const UpdateParams& p, int c, int K) {
    UpdateParams q = p;
    const int layer = p.gdims[0] * p.gdims[1];
    const int z0 = c * p.gdims[2] / K, z1 = (c + 1) * p.gdims[2] / K;
    const size_t p0 = (size_t)layer * z0, k0 = p0 * (size_t)p.R;
    const size_t lights = (size_t)(p.n_lights > 0 ? p.n_lights : 1);
    q.P = layer * (z1 - z0);
    q.p_begin = p.p_begin + (int)p0;
    if (p.states) q.states = p.states + p0;
    q.prev_irr = p.prev_irr + p0 * (kIrrT * kIrrT);
    q.prev_depth = p.prev_depth + p0 * (kDepT * kDepT);
    q.prev_valid = p.prev_valid + p0;
    q.cur_irr = p.cur_irr + p0 * (kIrrT * kIrrT);
    q.cur_depth = p.cur_depth + p0 * (kDepT * kDepT);
    q.cur_valid = p.cur_valid + p0;
    if (p.records) q.records = p.records + k0;
    q.ray_t = p.ray_t + k0;
    q.ray_es = p.ray_es + k0;
    q.ray_n = p.ray_n + k0;
    q.ray_alb = p.ray_alb + k0;
    q.ray_base = p.ray_base + k0;
    q.ray_lit = p.ray_lit + k0;
    q.ray_ssteps = p.ray_ssteps + k0;
    q.ray_val = p.ray_val + k0;
    q.tasks = p.tasks + k0 * lights;
    q.task_scale = p.task_scale + k0 * lights;
    q.fin_list = p.fin_list + k0;
    const size_t cap = (size_t)q.P * (size_t)p.R * lights;
    q.task_capacity = (uint32_t)(cap < 0xffffffffu ? cap : 0xffffffffu);
    q.counters = p.counters + (size_t)c * kSlabCounterStride;
    q.vol.fail = q.counters + kFailWord;
    return q;
}

template <typename T>
static cudaError_t launch_stages(const UpdateParams& p, cudaStream_t stream, cudaEvent_t const* ev,
                                 const SlabLanes* lanes, int slabs) {
    const DeviceSetup* setup = nullptr;
    cudaError_t e = prepare_update_kernels(&setup);
    if (e != cudaSuccess) return e;
    auto mark = [&](int k) { return ev ? cudaEventRecord(ev[k], stream) : cudaSuccess; };
    e = mark(0);
    // the pools and counts of every slab start at zero; the failure bits are sticky until read
    for (int c = 0; c < slabs && e == cudaSuccess; ++c)
        e = cudaMemsetAsync(p.counters + (size_t)c * kSlabCounterStride, 0, kFailWord * sizeof(uint32_t), stream);
    if (e != cudaSuccess) return e;
    const bool tc = gather_tc_supported(p) && p.sched.gather != 2;
    // the texel weights (with the frame's directions when dirs is set); the column sums serve
    // the SIMT gather, the tensor-core gather sums a column of ones
    auto weights = [&](cudaStream_t s, bool dirs) {
        if (p.depth_exp == 50) {
            if (dirs)
                weights_kernel<50, true><<<p.R, kThreads, 0, s>>>(p);
            else
                weights_kernel<50, false><<<p.R, kThreads, 0, s>>>(p);
        } else {
            if (dirs)
                weights_kernel<0, true><<<p.R, kThreads, 0, s>>>(p);
            else
                weights_kernel<0, false><<<p.R, kThreads, 0, s>>>(p);
        }
        if (!tc) weight_sums_kernel<<<1, kThreads, 0, s>>>(p);
    };
    if (slabs == 1) {
        weights(stream, true);
        if ((e = mark(1)) != cudaSuccess) return e;
        for (int s = 0; s < 4 && e == cudaSuccess; ++s) e = launch_stage<T>(p, *setup, s, stream, ev, true);
        return e;
    }
    // Slab branches: while one slab's pools drain (their last, longest rays keep few lanes
    // busy), the other slabs' kernels fill the SMs. Slab c runs on its own stream (slab 0 on
    // `stream`). Only the directions come before the fork: the texel weights and their image,
    // which only the gathers read, run on a stream of their own (a spare side stream, else
    // the last slab's), and every other slab's gather waits for them.
    ray_dirs_kernel<<<(p.R + kThreads - 1) / kThreads, kThreads, 0, stream>>>(p);
    if ((e = cudaEventRecord(lanes->fork, stream)) != cudaSuccess) return e;
    const int n_side = slabs < kMaxSlabs ? slabs : slabs - 1;  // side streams in use
    for (int c = 0; c < n_side && e == cudaSuccess; ++c) e = cudaStreamWaitEvent(lanes->side[c], lanes->fork, 0);
    if (e != cudaSuccess) return e;
    UpdateParams q[kMaxSlabs];
    for (int c = 0; c < slabs; ++c) q[c] = slab_params(p, c, slabs);
    auto lane = [&](int c) { return c == 0 ? stream : lanes->side[c - 1]; };
    const cudaStream_t ws = lanes->side[n_side - 1];
    const int w_slab = slabs < kMaxSlabs ? -1 : slabs - 1;  // the slab sharing that stream, if any
    weights(ws, false);
    if (tc) e = launch_pack_weights(p, ws);
    if (e == cudaSuccess) e = cudaEventRecord(lanes->weights_ready, ws);
    for (int c = 0; c < slabs; ++c)
        for (int s = 0; s < 4 && e == cudaSuccess; ++s) {
            if (s == 3 && c != w_slab) e = cudaStreamWaitEvent(lane(c), lanes->weights_ready, 0);
            if (e == cudaSuccess) e = launch_stage<T>(q[c], *setup, s, lane(c), nullptr, false);
        }
    // join even after a failed launch, so that no branch is left unjoined
    cudaError_t j = cudaSuccess;
    for (int c = 0; c < n_side && j == cudaSuccess; ++c) {  // the slabs' streams and the weights' stream
        j = cudaEventRecord(lanes->join[c], lanes->side[c]);
        if (j == cudaSuccess) j = cudaStreamWaitEvent(stream, lanes->join[c], 0);
    }
    return e != cudaSuccess ? e : j;
}

template <typename T>
static cudaError_t launch_merged_stages(const MergedParams& m, const DeviceSetup& setup, cudaStream_t stream) {
    // the merged pools span every volume, so they take the default shapes rather than one
    // volume's tuned schedule: the occupancy limit of CTAs and the 32-bit index form
    const UpdateParams& p0 = m.p[0];
    const int rp = p0.omega_primary > 1.f ? 1 : 0, rs = p0.omega_shadow > 1.f ? 1 : 0;
    constexpr bool i64 = false;
    cudaError_t e = cudaSuccess;
    if (p0.depth_exp == 50)
        weights_merged_kernel<50><<<m.dir_begin[m.n], kThreads, 0, stream>>>(m);
    else
        weights_merged_kernel<0><<<m.dir_begin[m.n], kThreads, 0, stream>>>(m);
    const int gp = persistent_blocks(setup, setup.occ_primary_merged[rp][type_slot<T>()], 0);
    if (rp)
        i64 ? primary_merged_kernel<T, true, true><<<gp, kTraceThreads, 0, stream>>>(m)
            : primary_merged_kernel<T, true, false><<<gp, kTraceThreads, 0, stream>>>(m);
    else
        i64 ? primary_merged_kernel<T, false, true><<<gp, kTraceThreads, 0, stream>>>(m)
            : primary_merged_kernel<T, false, false><<<gp, kTraceThreads, 0, stream>>>(m);
    prep_merged_kernel<T><<<m.prep_begin[m.n], kThreads, 0, stream>>>(m);
    const int gs = persistent_blocks(setup, setup.occ_shadow_merged[rs][type_slot<T>()], 0);
    if (rs)
        i64 ? shadow_merged_kernel<T, true, true><<<gs, kTraceThreads, 0, stream>>>(m)
            : shadow_merged_kernel<T, true, false><<<gs, kTraceThreads, 0, stream>>>(m);
    else
        i64 ? shadow_merged_kernel<T, false, true><<<gs, kTraceThreads, 0, stream>>>(m)
            : shadow_merged_kernel<T, false, false><<<gs, kTraceThreads, 0, stream>>>(m);
    uint32_t rays = 0;
    for (int v = 0; v < m.n; ++v) rays += (uint32_t)m.p[v].P * (uint32_t)m.p[v].R;
    finalize_merged_kernel<<<max(1, min((int)((rays + kThreads - 1) / kThreads), 8 * setup.sms)), kThreads, 0, stream>>>(m);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_gather_tc_merged(m, stream, true);
    return e;
}

cudaError_t launch_merged(const UpdateParams* p, int n, MergedParams* m, cudaStream_t stream) {
    if (!merged_supported(p, n, nullptr)) return cudaErrorInvalidValue;
    const DeviceSetup* setup = nullptr;
    cudaError_t e = prepare_update_kernels(&setup);
    if (e != cudaSuccess) return e;
    std::memset(m, 0, sizeof *m);
    m->n = n;
    m->primary_batch = (uint32_t)kBatch;
    m->shadow_batch = (uint32_t)kShadowBatch;
    uint64_t rb = 0, pb = 0, gb = 0, db = 0;
    for (int v = 0; v < n; ++v) {
        m->p[v] = prepared_params(p[v]);
        const uint64_t rays = (uint64_t)p[v].P * (uint64_t)p[v].R;
        m->ray_begin[v] = (uint32_t)rb;
        m->prep_begin[v] = (uint32_t)pb;
        m->gather_begin[v] = (uint32_t)gb;
        m->dir_begin[v] = (uint32_t)db;
        rb += (rays + m->primary_batch - 1) / m->primary_batch * m->primary_batch;
        m->prep_rays[v] = prep_rays(rays, setup->sms, 2);
        pb += (rays + m->prep_rays[v] - 1) / m->prep_rays[v];
        gb += ((uint64_t)p[v].P + kGatherTcProbes - 1) / kGatherTcProbes;
        db += (uint64_t)(p[v].P > 0 ? p[v].R : 0);
    }
    if (rb >= 0xffffffffull - 2 * kShadowBatch) return cudaErrorInvalidValue;  // merged task indices are 32-bit
    m->ray_begin[n] = (uint32_t)rb;
    m->prep_begin[n] = (uint32_t)pb;
    m->gather_begin[n] = (uint32_t)gb;
    m->dir_begin[n] = (uint32_t)db;
    // every volume's pools and counts start at zero (the merged pools are volume 0's words)
    for (int v = 0; v < n && e == cudaSuccess; ++v)
        e = cudaMemsetAsync(m->p[v].counters, 0, kFailWord * sizeof(uint32_t), stream);
    if (e != cudaSuccess || rb == 0) return e;
    return p[0].vol.dtype == SDFDDGI_F16 ? launch_merged_stages<__half>(*m, *setup, stream)
                                         : launch_merged_stages<float>(*m, *setup, stream);
}

int slab_count(const UpdateParams& p, bool have_lanes, bool stage_events) {
    if (!have_lanes || stage_events || p.P <= 0) return 1;
    int k = p.sched.slabs;
    // automatic: two slabs once an update is large enough for its pool tails to matter
    // (measured on open256: from 2^19 rays, 32 rays per probe, two slabs are ahead)
    if (k <= 0) k = (size_t)p.P * (size_t)p.R >= ((size_t)1 << 19) ? 2 : 1;
    return max(1, min(min(k, kMaxSlabs), p.gdims[2]));
}

bool merged_supported(const UpdateParams* p, int n, const char** why) {
    auto no = [&](const char* m) {
        if (why) *why = m;
        return false;
    };
    if (n < 1 || n > kMaxMerged) return no("the merged form takes 1 to 8 volumes");
    for (int i = 0; i < n; ++i) {
        const UpdateParams& a = p[i];
        const UpdateParams& b = p[0];
        if (a.vol.dtype != SDFDDGI_F32 && a.vol.dtype != SDFDDGI_F16) return no("the merged form needs a voxel SDF");
        if (a.vol.quads != b.vol.quads) return no("the volumes must share one scene");
        if (a.eps_w != b.eps_w || a.max_steps != b.max_steps)
            return no("the volumes must share the hit threshold and the step budget");
        if ((a.omega_primary > 1.f) != (b.omega_primary > 1.f) || (a.omega_shadow > 1.f) != (b.omega_shadow > 1.f) ||
            (a.omega_primary > 1.f && a.omega_primary != b.omega_primary) ||
            (a.omega_shadow > 1.f && a.omega_shadow != b.omega_shadow))
            return no("the volumes must share the relaxation of their traces");
        if (a.depth_exp != b.depth_exp || a.blend_bf16 != b.blend_bf16)
            return no("the volumes must share the depth exponent and the gather precision");
        if (!gather_tc_supported(a) || a.sched.gather == 2)
            return no("the merged form needs the tensor-core gather (rays per probe a multiple of 16)");
        if (a.records || a.test_stall) return no("the merged form records no rays");
    }
    if (why) *why = nullptr;
    return true;
}

UpdateParams prepared_params(const UpdateParams& params) {
    UpdateParams p = params;
    if (!(p.omega_primary > 1.f)) p.omega_primary = 1.f;  // plain sphere tracing unless relaxation was asked for
    if (!(p.omega_shadow > 1.f)) p.omega_shadow = 1.f;
    if (!p.look_irr) p.look_irr = p.prev_irr;
    if (!p.look_valid) p.look_valid = p.prev_valid;
    p.dirs = reinterpret_cast<float4*>(p.weights + (size_t)(p.R + 1) * kTexels);  // after the weights
    p.ray_val = p.ray_n;  // the gather's values replace the normals, dead after the shadow stage
    p.vol.fail = p.counters + kFailWord;
    return p;
}

cudaError_t launch_update(const UpdateParams& params, cudaStream_t stream, cudaEvent_t const* stage_events,
                          const SlabLanes* lanes) {
    if (params.P == 0) return cudaSuccess;
    const UpdateParams p = prepared_params(params);
    const int slabs = slab_count(p, lanes != nullptr, stage_events != nullptr);
    if (p.vol.dtype == kAnalytic) return launch_stages<Analytic>(p, stream, stage_events, lanes, slabs);
    return p.vol.dtype == SDFDDGI_F16 ? launch_stages<__half>(p, stream, stage_events, lanes, slabs)
                                      : launch_stages<float>(p, stream, stage_events, lanes, slabs);
}

}  // namespace sdfddgi
