// device.cuh -- device building blocks of the probe update (FP32 arithmetic).
//
// Sampling rule of the signed-distance and material volumes: voxel centres sit at
// integer coordinates g = (p - lo)/h - 1/2; the trilinear cell is clamped to the
// volume and the fractions to [0, 1]. Sphere tracing, shading and the octahedral
// map follow Sec. 3.3 of Hu et al. (arXiv 2007.14394); see the host header for
// the full statement of each step.
#pragma once

#include "internal.h"

namespace sdfddgi {

__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 fma3(float s, float3 d, float3 o) {
    return f3(fmaf(s, d.x, o.x), fmaf(s, d.y, o.y), fmaf(s, d.z, o.z));
}

// The index i of a buffer of n elements; in the bounds-checked build an index outside
// [0, n) sets kFailBounds in *fail (when given) and becomes 0.
template <typename I>
__device__ __forceinline__ I checked(I i, size_t n, uint32_t* fail) {
    if constexpr (kChecked) {
        if (!((size_t)i < n)) {
            if (fail) atomicOr(fail, kFailBounds);
            return (I)0;
        }
    }
    return i;
}

// ------------------------------------------------------------------ volume sampling
struct Cell {
    size_t base;  // linear index of corner (0,0,0)
    int ix, iy, iz;
    float fx, fy, fz;
};

__device__ __forceinline__ int clamp_index(float g, int n, float* frac) {
    int i = (int)floorf(g);
    i = max(0, min(i, n - 2));
    *frac = fminf(fmaxf(g - (float)i, 0.0f), 1.0f);
    return i;
}

__device__ __forceinline__ Cell cell_of(const VolumeView& v, float3 p) {
    Cell c;
    int ix = clamp_index(fmaf(p.x - v.lo[0], v.inv_h, -0.5f), v.nx, &c.fx);
    int iy = clamp_index(fmaf(p.y - v.lo[1], v.inv_h, -0.5f), v.ny, &c.fy);
    int iz = clamp_index(fmaf(p.z - v.lo[2], v.inv_h, -0.5f), v.nz, &c.fz);
    c.base = ((size_t)iz * v.ny + iy) * v.nx + ix;
    c.ix = ix;
    c.iy = iy;
    c.iz = iz;
    return c;
}

__device__ __forceinline__ float lerp(float a, float b, float t) { return fmaf(t, b - a, a); }

// The four corners (x,y) (x+1,y) (x,y+1) (x+1,y+1) of one z slice of a cell, from the
// xy-quad store (one vector load).
template <typename T>
__device__ __forceinline__ float4 ld_quad(const void* quads, size_t i);
template <>
__device__ __forceinline__ float4 ld_quad<float>(const void* quads, size_t i) {
    return __ldg(static_cast<const float4*>(quads) + i);
}
template <>
__device__ __forceinline__ float4 ld_quad<__half>(const void* quads, size_t i) {
    const uint2 r = __ldg(static_cast<const uint2*>(quads) + i);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&r.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&r.y));
    return make_float4(a.x, a.y, b.x, b.y);
}

// Trilinear interpolation of a cell from its two quads (slices z and z + 1).
__device__ __forceinline__ float trilinear_quads(float4 q0, float4 q1, float fx, float fy, float fz) {
    const float x00 = lerp(q0.x, q0.y, fx), x10 = lerp(q0.z, q0.w, fx);
    const float x01 = lerp(q1.x, q1.y, fx), x11 = lerp(q1.z, q1.w, fx);
    return lerp(lerp(x00, x10, fy), lerp(x01, x11, fy), fz);
}

// The SDF at world point p by the sampling rule (cell and fractions clamped).
template <typename T>
__device__ __forceinline__ float sample_sdf(const VolumeView& v, float3 p) {
    const Cell c = cell_of(v, p);
    const int z = c.iz + 1;  // padded slice of the cell's lower corner
    const size_t i0 = quad_index((size_t)c.ix + 1, (size_t)c.iy + 1, (size_t)z, (size_t)v.qx, (size_t)v.qy);
    // slice z + 1: the next entry for even z, else the first of the next pair
    const size_t i1 = (z & 1) ? i0 + (size_t)2 * v.qx * v.qy - 1 : i0 + 1;
    return trilinear_quads(ld_quad<T>(v.quads, checked(i0, v.n_quads, v.fail)),
                           ld_quad<T>(v.quads, checked(i1, v.n_quads, v.fail)), c.fx, c.fy, c.fz);
}

// The SDF at voxel coordinate g (voxel centres at integers, g = (p - lo)/h - 1/2) for a point
// inside the volume box, g in [-1/2, n - 1/2] on every axis: the cell floor(g) lies in
// [-1, n - 1], which the apron of the quad store covers, so neither the cell nor the
// fractions need clamping; where the clamped rule would clamp, the apron's copies of the
// edge values give the same value. The two forms of the quad index (Idx64: all in 64 bits,
// else the z-pair row in 32 bits) give the same addresses; which one runs faster depends on
// the store (measured: the 32-bit form on a 275 MB float32 store, the 64-bit form on a 1 GB
// binary16 one).
template <typename T, bool Idx64>
__device__ __forceinline__ float sample_sdf_vox(const VolumeView& v, float3 g) {
    const int ix = __float2int_rd(g.x), iy = __float2int_rd(g.y), iz = __float2int_rd(g.z);
    const float fx = g.x - (float)ix, fy = g.y - (float)iy, fz = g.z - (float)iz;
    const int z = iz + 1;  // padded slice of the cell's lower corner
    size_t i0;
    if constexpr (Idx64) {
        i0 = quad_index((size_t)ix + 1, (size_t)iy + 1, (size_t)z, (size_t)v.qx, (size_t)v.qy);
    } else {
        const uint32_t row = (uint32_t)(z >> 1) * (uint32_t)v.qy + (uint32_t)(iy + 1);
        i0 = ((size_t)row * (uint32_t)v.qx + (uint32_t)(ix + 1)) * 2 + (uint32_t)(z & 1);
    }
    const size_t i1 = (z & 1) ? i0 + (size_t)2 * v.qx * v.qy - 1 : i0 + 1;
    return trilinear_quads(ld_quad<T>(v.quads, checked(i0, v.n_quads, v.fail)),
                           ld_quad<T>(v.quads, checked(i1, v.n_quads, v.fail)), fx, fy, fz);
}

// ------------------------------------------------------------------ analytic scene (Sec. 3.1)
struct Analytic {};  // the SDF-type tag of a scene made of primitives

// Exact Euclidean distance to one primitive (negative inside), float32.
__device__ __forceinline__ float prim_distance(const PrimDev& q, float3 x) {
    switch (q.type) {
        case SDFDDGI_PRIM_SPHERE: {
            const float3 v = x - f3(q.p[0], q.p[1], q.p[2]);
            return sqrtf(dot(v, v)) - q.p[3];
        }
        case SDFDDGI_PRIM_BOX: {
            const float ex = fabsf(x.x - q.p[0]) - q.p[3], ey = fabsf(x.y - q.p[1]) - q.p[4],
                        ez = fabsf(x.z - q.p[2]) - q.p[5];
            const float ox = fmaxf(ex, 0.f), oy = fmaxf(ey, 0.f), oz = fmaxf(ez, 0.f);
            return sqrtf(ox * ox + oy * oy + oz * oz) + fminf(fmaxf(ex, fmaxf(ey, ez)), 0.f);
        }
        case SDFDDGI_PRIM_CAPSULE: {
            const float3 a = f3(q.p[0], q.p[1], q.p[2]), ab = f3(q.p[3], q.p[4], q.p[5]) - a, ax = x - a;
            const float l2 = dot(ab, ab);
            const float s = l2 > 0.f ? fminf(fmaxf(dot(ax, ab) / l2, 0.f), 1.f) : 0.f;
            const float3 r = ax - s * ab;
            return sqrtf(dot(r, r)) - q.p[6];
        }
        case SDFDDGI_PRIM_PLANE_Y:
            return x.y - q.p[0];
        case SDFDDGI_PRIM_INV_SPHERE: {
            const float3 v = x - f3(q.p[0], q.p[1], q.p[2]);
            return q.p[3] - sqrtf(dot(v, v));
        }
        default:
            return INFINITY;
    }
}

__device__ __forceinline__ void take(const PrimDev& q, float d, float* best, int* who) {
    if (d < *best || (d == *best && q.index < *who)) {
        *best = d;
        *who = q.index;
    }
}

// Distance of the union of primitives at p (the paper's cluster query): the unbounded
// primitives, then every cluster whose box lies no farther than the best distance so far
// (or contains p, once p is inside a primitive),
// starting from `bound` (an upper bound known beforehand: +inf, or about twice the last
// distance of a sphere trace). The result is the minimum over all primitives whenever
// bound is one. *who (optional) receives the caller's index of the primitive attaining
// it (the lowest among equals), *slot its position in the primitive array.
__device__ __forceinline__ float analytic_sdf(const VolumeView& v, float3 p, float bound, int* who = nullptr,
                                              int* slot = nullptr) {
    float best = bound;
    int idx = 0x7fffffff, at = -1;
    for (int k = 0; k < v.n_unbounded; ++k) {
        const PrimDev& q = v.prims[k];
        const int before = idx;
        take(q, prim_distance(q, p), &best, &idx);
        if (idx != before) at = k;
    }
    for (int c = 0; c < v.n_clusters; ++c) {
        const ClusterDev cl = v.clusters[c];
        const float dx = fmaxf(fmaxf(cl.lo[0] - p.x, p.x - cl.hi[0]), 0.f);
        const float dy = fmaxf(fmaxf(cl.lo[1] - p.y, p.y - cl.hi[1]), 0.f);
        const float dz = fmaxf(fmaxf(cl.lo[2] - p.z, p.z - cl.hi[2]), 0.f);
        // every primitive inside lies at least the box distance away; a point already inside a
        // primitive (best < 0) must still visit each box that contains it
        if (sqrtf(dx * dx + dy * dy + dz * dz) > fmaxf(best, 0.f)) continue;
        for (int k = cl.first; k < cl.first + cl.count; ++k) {
            const PrimDev& q = v.prims[k];
            const int before = idx;
            take(q, prim_distance(q, p), &best, &idx);
            if (idx != before) at = k;
        }
    }
    if (who) *who = idx;
    if (slot) *slot = at;
    return best;
}

template <>
__device__ __forceinline__ float sample_sdf<Analytic>(const VolumeView& v, float3 p) {
    return analytic_sdf(v, p, INFINITY);
}

// Albedo and emission: the material volume under the same trilinear rule.
__device__ __forceinline__ void sample_material(const VolumeView& v, float3 p, float3* albedo, float3* emission) {
    *albedo = f3(0.f, 0.f, 0.f);
    *emission = f3(0.f, 0.f, 0.f);
    if (!v.material) return;
    const Cell c = cell_of(v, p);
    const size_t sy = (size_t)v.nx, sz = (size_t)v.nx * v.ny;
    float a[3] = {0.f, 0.f, 0.f}, e[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int dx = k & 1, dy = (k >> 1) & 1, dz = (k >> 2) & 1;
        const float w = (dx ? c.fx : 1.f - c.fx) * (dy ? c.fy : 1.f - c.fy) * (dz ? c.fz : 1.f - c.fz);
        const uint4 raw = __ldg(v.material + checked(c.base + dz * sz + dy * sy + dx, sz * v.nz, v.fail));
        const __half2 h01 = *reinterpret_cast<const __half2*>(&raw.x);
        const __half2 h23 = *reinterpret_cast<const __half2*>(&raw.y);
        const __half2 h45 = *reinterpret_cast<const __half2*>(&raw.z);
        const __half2 h67 = *reinterpret_cast<const __half2*>(&raw.w);
        const float2 m01 = __half22float2(h01), m23 = __half22float2(h23);
        const float2 m45 = __half22float2(h45), m67 = __half22float2(h67);
        a[0] = fmaf(w, m01.x, a[0]);
        a[1] = fmaf(w, m01.y, a[1]);
        a[2] = fmaf(w, m23.x, a[2]);
        e[0] = fmaf(w, m45.x, e[0]);
        e[1] = fmaf(w, m45.y, e[1]);
        e[2] = fmaf(w, m67.x, e[2]);
    }
    *albedo = f3(a[0], a[1], a[2]);
    *emission = f3(e[0], e[1], e[2]);
}

// ------------------------------------------------------------------ sphere tracing
struct Trace {
    float t;
    int steps;
    int event;
};

__device__ __forceinline__ bool is_miss(int event) { return event == kLeftVolume || event == kPastLimit; }

// Sphere tracing (Sec. 3.3, accelerated sphere tracing of the scene SDF): step by the
// sampled distance until it drops below eps (hit), the point leaves the volume box,
// t passes `tlimit`, or the budget is spent (taken as a hit at the final t).
template <typename T>
__device__ __forceinline__ Trace sphere_trace(const VolumeView& v, float3 o, float3 d, float eps, float tlimit,
                                              int max_steps) {
    float t = 0.0f;
    for (int s = 0; s < max_steps; ++s) {
        const float3 p = fma3(t, d, o);
        if (p.x < v.lo[0] || p.x > v.hi[0] || p.y < v.lo[1] || p.y > v.hi[1] || p.z < v.lo[2] || p.z > v.hi[2])
            return {tlimit, s, kLeftVolume};
        const float sd = sample_sdf<T>(v, p);
        if (sd < eps) return {t, s + 1, kHit};
        t += sd;
        if (t > tlimit) return {tlimit, s + 1, kPastLimit};
    }
    return {t, max_steps, kExhausted};
}

// ------------------------------------------------------------------ octahedral map
__device__ __forceinline__ float sign_nz(float x) { return x >= 0.f ? 1.f : -1.f; }

// Octahedral parameterisation of the sphere (pole +z), uv in [0,1]^2.
__device__ __forceinline__ float2 oct_encode(float3 v) {
    const float inv_l1 = 1.0f / (fabsf(v.x) + fabsf(v.y) + fabsf(v.z));
    float qx = v.x * inv_l1, qy = v.y * inv_l1;
    if (v.z < 0.f) {
        const float ox = (1.f - fabsf(qy)) * sign_nz(qx);
        const float oy = (1.f - fabsf(qx)) * sign_nz(qy);
        qx = ox;
        qy = oy;
    }
    return make_float2(fmaf(0.5f, qx, 0.5f), fmaf(0.5f, qy, 0.5f));
}

__device__ __forceinline__ float3 oct_decode(float u, float w) {
    const float qx = fmaf(2.f, u, -1.f), qy = fmaf(2.f, w, -1.f);
    const float z = 1.f - fabsf(qx) - fabsf(qy);
    float x = qx, y = qy;
    if (z < 0.f) {
        x = (1.f - fabsf(qy)) * sign_nz(qx);
        y = (1.f - fabsf(qx)) * sign_nz(qy);
    }
    const float inv = rsqrtf(x * x + y * y + z * z);
    return f3(x * inv, y * inv, z * inv);
}

// Direction of interior texel (a, b) of an n x n octahedral map.
__device__ __forceinline__ float3 texel_dir(int a, int b, int n) {
    const float inv_n = 1.0f / (float)n;
    return oct_decode(((float)a + 0.5f) * inv_n, ((float)b + 0.5f) * inv_n);
}

// Source texel of bordered-map texel (y, x) for an (n+2)^2 map: interior texels map to
// themselves; each edge row/column mirrors the adjacent interior row/column about its
// midpoint, and each corner takes the diagonally opposite interior corner (the
// octahedron's fold puts those texels next to each other on the sphere).
__device__ __forceinline__ int2 border_source(int y, int x, int n) {
    const int last = n + 1;
    const bool top = y == 0, bottom = y == last, left = x == 0, right = x == last;
    if ((top || bottom) && (left || right)) return make_int2(top ? n : 1, left ? n : 1);  // corners
    if (top) return make_int2(1, last - x);
    if (bottom) return make_int2(n, last - x);
    if (left) return make_int2(last - y, 1);
    if (right) return make_int2(last - y, n);
    return make_int2(y, x);
}

// Texel (y, x) of border texel b (0 <= b < 4n + 4) of an (n+2)^2 map: the top row, the bottom
// row, then the left and right columns between them. Every border texel's source
// (border_source) is an interior texel, so the border copies are independent of one another.
__device__ __forceinline__ int2 border_texel(int b, int n) {
    const int w = n + 2;
    if (b < w) return make_int2(0, b);
    if (b < 2 * w) return make_int2(n + 1, b - w);
    b -= 2 * w;
    return b < n ? make_int2(b + 1, 0) : make_int2(b - n + 1, n + 1);
}

// ------------------------------------------------------------------ probe interpolation
// Normalised irradiance at world point x for unit normal nrm from an irradiance atlas:
// trilinear over the 8 probes of the grid cell (clamped), weighted by trilinear weight
// times the probe's history flag, each probe contributing its map's bilinear value at
// oct(nrm); weights renormalised, 0 when they all vanish.
__device__ __forceinline__ float3 interpolate_irradiance(const int gd[3], const float go[3], const float gs[3],
                                                         const float4* irr, const uint8_t* valid, float3 x,
                                                         float3 nrm, uint32_t* fail = nullptr) {
    const float xs[3] = {x.x, x.y, x.z};
    int base[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float c = fminf(fmaxf((xs[a] - go[a]) / gs[a], 0.f), (float)(gd[a] - 1));
        int b = (int)floorf(c);
        b = max(0, min(b, gd[a] - 2));
        base[a] = b;
        f[a] = gd[a] > 1 ? c - (float)b : 0.f;
    }
    const float2 uv = oct_encode(nrm);
    const float cx = fmaf(uv.x, (float)kIrrN, 0.5f), cy = fmaf(uv.y, (float)kIrrN, 0.5f);  // 1 + uv*n - 1/2
    const int x0 = min((int)floorf(cx), kIrrN), y0 = min((int)floorf(cy), kIrrN);
    const float fx = cx - (float)x0, fy = cy - (float)y0;
    float sw = 0.f, r = 0.f, g = 0.f, bl = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int dx = k & 1, dy = (k >> 1) & 1, dz = (k >> 2) & 1;
        const int ix = min(base[0] + dx, gd[0] - 1), iy = min(base[1] + dy, gd[1] - 1), iz = min(base[2] + dz, gd[2] - 1);
        const size_t p = checked(((size_t)iz * gd[1] + iy) * gd[0] + ix, (size_t)gd[0] * gd[1] * gd[2], fail);
        float w = (dx ? f[0] : 1.f - f[0]) * (dy ? f[1] : 1.f - f[1]) * (dz ? f[2] : 1.f - f[2]);
        if (!__ldg(valid + p)) w = 0.f;
        if (!(w > 0.f)) continue;
        const float4* m = irr + p * (kIrrT * kIrrT);
        const int t0 = checked(y0 * kIrrT + x0, kIrrT * kIrrT - kIrrT - 1, fail);  // the 2x2 texels stay in the map
        const float4 t00 = __ldg(m + t0), t01 = __ldg(m + t0 + 1);
        const float4 t10 = __ldg(m + t0 + kIrrT), t11 = __ldg(m + t0 + kIrrT + 1);
        const float w00 = (1.f - fx) * (1.f - fy), w01 = fx * (1.f - fy), w10 = (1.f - fx) * fy, w11 = fx * fy;
        r = fmaf(w, w00 * t00.x + w01 * t01.x + w10 * t10.x + w11 * t11.x, r);
        g = fmaf(w, w00 * t00.y + w01 * t01.y + w10 * t10.y + w11 * t11.y, g);
        bl = fmaf(w, w00 * t00.z + w01 * t01.z + w10 * t10.z + w11 * t11.z, bl);
        sw += w;
    }
    if (!(sw > 0.f)) return f3(0.f, 0.f, 0.f);
    const float inv = 1.0f / sw;
    return f3(r * inv, g * inv, bl * inv);
}

// ------------------------------------------------------------------ probe visibility
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

// The interpolation of interpolate_irradiance with each probe's weight times its visibility
// from x; probes at their grid positions or at V.states' positions.
template <typename T>
__device__ float3 interpolate_irradiance_visible(const int gd[3], const float go[3], const float gs[3],
                                                 const float4* irr, const uint8_t* valid, const VisParams& V,
                                                 float3 x, float3 nrm) {
    const float xs[3] = {x.x, x.y, x.z};
    int base[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float c = fminf(fmaxf((xs[a] - go[a]) / gs[a], 0.f), (float)(gd[a] - 1));
        int b = (int)floorf(c);
        b = max(0, min(b, gd[a] - 2));
        base[a] = b;
        f[a] = gd[a] > 1 ? c - (float)b : 0.f;
    }
    const float2 uv = oct_encode(nrm);
    const float cx = fmaf(uv.x, (float)kIrrN, 0.5f), cy = fmaf(uv.y, (float)kIrrN, 0.5f);
    const int x0 = min((int)floorf(cx), kIrrN), y0 = min((int)floorf(cy), kIrrN);
    const float fx = cx - (float)x0, fy = cy - (float)y0;
    float sw = 0.f, r = 0.f, g = 0.f, bl = 0.f;
    for (int k = 0; k < 8; ++k) {
        const int dx = k & 1, dy = (k >> 1) & 1, dz = (k >> 2) & 1;
        const int ix = min(base[0] + dx, gd[0] - 1), iy = min(base[1] + dy, gd[1] - 1), iz = min(base[2] + dz, gd[2] - 1);
        const size_t p = ((size_t)iz * gd[1] + iy) * gd[0] + ix;
        float w = (dx ? f[0] : 1.f - f[0]) * (dy ? f[1] : 1.f - f[1]) * (dz ? f[2] : 1.f - f[2]);
        if (!__ldg(valid + p)) w = 0.f;
        if (!(w > 0.f)) continue;
        float3 q;
        if (V.states) {
            q = f3(V.states[p].pos[0], V.states[p].pos[1], V.states[p].pos[2]);
        } else {
            q = f3(fmaf((float)ix, gs[0], go[0]), fmaf((float)iy, gs[1], go[1]), fmaf((float)iz, gs[2], go[2]));
        }
        w *= probe_visibility<T>(V, x, nrm, q);
        if (!(w > 0.f)) continue;
        const float4* m = irr + p * (kIrrT * kIrrT);
        const float4 t00 = __ldg(m + y0 * kIrrT + x0), t01 = __ldg(m + y0 * kIrrT + x0 + 1);
        const float4 t10 = __ldg(m + (y0 + 1) * kIrrT + x0), t11 = __ldg(m + (y0 + 1) * kIrrT + x0 + 1);
        const float w00 = (1.f - fx) * (1.f - fy), w01 = fx * (1.f - fy), w10 = (1.f - fx) * fy, w11 = fx * fy;
        r = fmaf(w, w00 * t00.x + w01 * t01.x + w10 * t10.x + w11 * t11.x, r);
        g = fmaf(w, w00 * t00.y + w01 * t01.y + w10 * t10.y + w11 * t11.y, g);
        bl = fmaf(w, w00 * t00.z + w01 * t01.z + w10 * t10.z + w11 * t11.z, bl);
        sw += w;
    }
    if (!(sw > 0.f)) return f3(0.f, 0.f, 0.f);
    const float inv = 1.0f / sw;
    return f3(r * inv, g * inv, bl * inv);
}

}  // namespace sdfddgi
