// cascade.cu -- irradiance at points from a cascade of probe volumes (Sec. 3.5): the finest
// volume whose probe box holds the point, blended toward the next coarser volume across the
// finer one's outermost cell layer with a weight from mean value coordinates (Floater, Kos
// and Reimers 2005; Ju, Schaefer and Warren 2005). One lane per point; the integrals of the
// points that blend are spread over half-warps.
//
// The weight is the sum of the mean value coordinates of the inner box's 8 corners over the
// closed shell between the probe box and that box shrunk by one spacing (inner faces facing
// into the hole). Mean value coordinates are lambda_j = W_j / sum W, W_j the integral over
// the shell's surface of phi_j(p) h(p) / |p - x|^4 dA, phi_j the piecewise-linear hat of
// corner j and h(p) = n(p) . (p - x) the signed distance of the surface's plane at p. Over a
// whole face the hats of its 4 corners sum to 1, so the inner corners' total is
//     w = sum over the 6 inner faces of I_F / sum over all 12 faces of I_F,
//     I_F = h_F * integral over F of dA / |p - x|^4,
// the same number as the per-triangle closed form of Ju et al., but a float evaluation of
// that form loses up to 1e-3 in the weight (the per-triangle term cancels near the faces'
// planes, where every point of the shell lies), while I_F has a closed form that keeps full
// float accuracy (shell_terms below).
#include <algorithm>
#include <cmath>

#include "device.cuh"
#include "handles.h"

using namespace sdfddgi;

namespace {

constexpr int kMaxCascade = 8;
constexpr float kPi = 3.14159265358979f;

struct CascadeVol {
    int gdims[3];
    float gorigin[3];
    float gspacing[3];
    const float4* irr;
    const uint8_t* valid;
    bool visible;  // weight each probe by its visibility from the point (Sec. 3.4)
    VisParams vis;
};

struct CascadeArgs {
    CascadeVol v[kMaxCascade];
    int n;
    const float* points;
    const float* normals;
    float* out;
    int32_t* level;
    float* weight;
    int64_t n_pts;
};
static_assert(sizeof(CascadeArgs) <= 4096, "cascade parameters must stay within 4 KiB");

__device__ __forceinline__ float sgnf(float v) { return (float)((v > 0.f) - (v < 0.f)); }

// T(s) = atan(s h^2 / E) / h^2, finite as h -> 0.
__device__ __forceinline__ float atan_over(float s, float E, float h2) {
    const float q = __fdividef(s, E), z = q * h2;
    return fabsf(z) < 1e-3f ? q * fmaf(-z * z, 1.f / 3.f, 1.f) : q * __fdividef(atanf(z), z);
}

// The face integrals as sums over edges. In polar coordinates about the foot of x on the
// face's plane, I_F = h * integral of dA / (h^2 + rho^2)^2 becomes, edge by edge along the
// face's boundary (counter-clockwise in the plane's coordinates),
//     I_F = pi S / h - (h / 2) sum over edges of sigma [dA / (R (R + p)) + (p / R) dT],
// for an edge at in-plane distance p from the foot, R = sqrt(h^2 + p^2), endpoints at s1 < s2
// along it from the foot's projection, sigma = +-1 its orientation about the foot,
//     dA = atan(s2 / p) - atan(s1 / p) = atan2(p (s2 - s1), p^2 + s1 s2),
//     dT = T(s2) - T(s1),  T(s) = atan(s h^2 / E(s)) / h^2,  E(s) = (R + p)(p R + s^2),
// and S = 1 with the foot inside the face (1/2 on an edge, 1/4 at a corner, 0 outside). It
// follows from integrating rho d rho / (h^2 + rho^2)^2 along each direction and splitting
// (p / R) atan(s / R) into atan(s / p) (whose sum over the edges is the angle 2 pi S) and
// terms carrying h^2: nothing cancels as h -> 0 (x next to a face's plane) or as h and p
// both -> 0 (x next to an edge's line), the two places where every point of the shell can
// lie. Each box edge (12 per box) is shared by two faces, which share R, s1 and s2.
struct ShellBox {
    float lo[3], hi[3], ilo[3], ihi[3];
};

// Lane slot c (0..31) of a warp: for c < 24 the two face terms of box edge c (0..11 outer,
// 12..23 inner; axis e = (c % 12) / 4, at the corner bits (c & 1, (c >> 1) & 1) of axes e + 1,
// e + 2), for c < 12 also the pi S / h term of face c (0..5 outer, 6..11 inner; axis
// (c % 6) / 2, side c & 1). Adds them to num (inner faces) and den (all faces).
__device__ __forceinline__ void shell_terms(const ShellBox& B, const float x[3], int c, float& num, float& den) {
    if (c < 24) {
        const bool inner = c >= 12;
        const int r = c % 12, e = r >> 2, u = e == 2 ? 0 : e + 1, v = e == 0 ? 2 : (e == 1 ? 0 : 1);
        const int bits[2] = {r & 1, (r >> 1) & 1};
        const float* L = inner ? B.ilo : B.lo;
        const float* H = inner ? B.ihi : B.hi;
        const float du = (bits[0] ? H[u] : L[u]) - x[u], dv = (bits[1] ? H[v] : L[v]) - x[v];
        const float s1 = L[e] - x[e], s2 = H[e] - x[e];
        const float R = sqrtf(fmaf(du, du, dv * dv));
        float t = 0.f;
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            const float dax = f ? dv : du, dw = f ? du : dv;
            const int b_ax = bits[f], b_w = bits[f ^ 1];
            const float sigma = (b_w ? 1.f : -1.f) * sgnf(dw);
            if (dax == 0.f || sigma == 0.f) continue;  // h = 0: no integral; p = 0: no term
            const float p = fabsf(dw), h2 = dax * dax;
            // h = n . (corner - x), n the shell's outward normal: away from the probe box's
            // centre on the outer faces, into the hole on the inner ones
            const float h = (b_ax ? 1.f : -1.f) * (inner ? -1.f : 1.f) * dax;
            const float dA = atan2f(p * (s2 - s1), fmaf(p, p, s1 * s2));
            const float rp = R + p;
            const float dT = atan_over(s2, rp * fmaf(p, R, s2 * s2), h2) - atan_over(s1, rp * fmaf(p, R, s1 * s1), h2);
            t = fmaf(-0.5f * h * sigma, __fdividef(dA, R * rp) + __fdividef(p, R) * dT, t);
        }
        if (inner) num += t;
        den += t;
    }
    if (c < 12) {
        const bool fin = c >= 6;
        const int ax = (c % 6) >> 1, side = c & 1, p = ax == 0 ? 1 : 0, q = ax == 2 ? 1 : 2;
        const float* FL = fin ? B.ilo : B.lo;
        const float* FH = fin ? B.ihi : B.hi;
        const float S = 0.25f * (sgnf(FH[p] - x[p]) - sgnf(FL[p] - x[p])) * (sgnf(FH[q] - x[q]) - sgnf(FL[q] - x[q]));
        if (S != 0.f) {  // never with h = 0: x on a face is settled before
            const float n = (side ? 1.f : -1.f) * (fin ? -1.f : 1.f);
            const float h = n * ((side ? FH[ax] : FL[ax]) - x[ax]);
            const float fv = S * kPi / h;
            if (fin) num += fv;
            den += fv;
        }
    }
}

__device__ __forceinline__ float box_hi(const CascadeVol& V, int a) {
    return fmaf((float)(V.gdims[a] - 1), V.gspacing[a], V.gorigin[a]);
}

__device__ __forceinline__ bool in_box(const CascadeVol& V, const float xs[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (xs[a] < V.gorigin[a] || xs[a] > box_hi(V, a)) return false;
    return true;
}

__device__ __forceinline__ void shell_box(const CascadeVol& V, ShellBox& B) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        B.lo[a] = V.gorigin[a];
        B.hi[a] = box_hi(V, a);
        B.ilo[a] = B.lo[a] + V.gspacing[a];
        B.ihi[a] = B.hi[a] - V.gspacing[a];
    }
}

// The weight where it needs no integral: 1 without an inner box of positive volume or on and
// inside the inner box, 0 on the probe box's faces; -1 where the shell's integrals decide.
__device__ __forceinline__ float shell_limit(const CascadeVol& V, const float xs[3]) {
    ShellBox B;
    shell_box(V, B);
    bool inner = true, boundary = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (V.gdims[a] < 4) return 1.f;
        if (xs[a] < B.ilo[a] || xs[a] > B.ihi[a]) inner = false;
        if (xs[a] == B.lo[a] || xs[a] == B.hi[a]) boundary = true;
    }
    return inner ? 1.f : (boundary ? 0.f : -1.f);
}

// E_i of one level: the plain interpolation, or the one with probe visibility.
template <bool Visible>
__device__ __forceinline__ float3 level_irradiance(const CascadeVol& V, float3 x, float3 n) {
    if (Visible && V.visible) {
        if (V.vis.vol.dtype == kAnalytic)
            return interpolate_irradiance_visible<Analytic>(V.gdims, V.gorigin, V.gspacing, V.irr, V.valid, V.vis, x, n);
        if (V.vis.vol.dtype == SDFDDGI_F16)
            return interpolate_irradiance_visible<__half>(V.gdims, V.gorigin, V.gspacing, V.irr, V.valid, V.vis, x, n);
        return interpolate_irradiance_visible<float>(V.gdims, V.gorigin, V.gspacing, V.irr, V.valid, V.vis, x, n);
    }
    return interpolate_irradiance(V.gdims, V.gorigin, V.gspacing, V.irr, V.valid, x, n);
}

constexpr unsigned kFull = 0xffffffffu;

// One warp handles 32 consecutive points. The points whose weight needs the shell's integrals
// are taken one at a time by the whole warp, one box edge per lane (the 48 edge terms and 12
// face terms of a point spread over 24 lanes instead of running in one lane while the warp's
// other lanes idle), and the warp's sums are reduced by shuffles.
template <bool Visible>
__global__ void __launch_bounds__(256) cascade_kernel(const __grid_constant__ CascadeArgs A) {
    const int lane = threadIdx.x & 31;
    const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < A.n_pts;
         base += n_warps * 32) {
        const int64_t i = base + lane;
        const bool live = i < A.n_pts;
        float xs[3] = {0.f, 0.f, 0.f};
        float3 nrm = f3(0.f, 0.f, 1.f);
        int k = A.n - 1;
        float w = 1.f;
        if (live) {
            xs[0] = A.points[3 * i];
            xs[1] = A.points[3 * i + 1];
            xs[2] = A.points[3 * i + 2];
            nrm = f3(A.normals[3 * i], A.normals[3 * i + 1], A.normals[3 * i + 2]);
            for (int j = 0; j < A.n - 1; ++j)
                if (in_box(A.v[j], xs)) {
                    k = j;
                    break;
                }
            if (k < A.n - 1) w = shell_limit(A.v[k], xs);
        }
        unsigned todo = __ballot_sync(kFull, live && w < 0.f);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const float px[3] = {__shfl_sync(kFull, xs[0], src), __shfl_sync(kFull, xs[1], src),
                                 __shfl_sync(kFull, xs[2], src)};
            ShellBox B;
            shell_box(A.v[__shfl_sync(kFull, k, src)], B);
            float num = 0.f, den = 0.f;
            shell_terms(B, px, lane, num, den);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                num += __shfl_xor_sync(kFull, num, o);
                den += __shfl_xor_sync(kFull, den, o);
            }
            if (lane == src) w = fminf(fmaxf(num / den, 0.f), 1.f);
        }
        if (!live) continue;
        const CascadeVol& V = A.v[k];
        const float3 x = f3(xs[0], xs[1], xs[2]);
        float3 e = level_irradiance<Visible>(V, x, nrm);
        if (w < 1.f) {
            const float3 c = level_irradiance<Visible>(A.v[k + 1], x, nrm);
            const float u = 1.f - w;
            e = f3(fmaf(w, e.x, u * c.x), fmaf(w, e.y, u * c.y), fmaf(w, e.z, u * c.z));
        }
        A.out[3 * i] = e.x;
        A.out[3 * i + 1] = e.y;
        A.out[3 * i + 2] = e.z;
        if (A.level) A.level[i] = k;
        if (A.weight) A.weight[i] = w;
    }
}

}  // namespace

extern "C" SDFDDGI_API int sdfddgi_sample_irradiance_cascade(const sdfddgi_volume* const* volumes, int32_t n,
                                                             const float* points, const float* normals, int64_t n_pts,
                                                             float softness, const sdfddgi_probe_state* const* states,
                                                             float* out_rgb, int32_t* out_level, float* out_weight,
                                                             void* stream) {
    if (!volumes) return report_error(SDFDDGI_ERR_INVALID_ARG, "sample_irradiance_cascade: volumes is NULL");
    if (n < 1 || n > kMaxCascade)
        return report_error(SDFDDGI_ERR_INVALID_ARG, "sample_irradiance_cascade: n must be in [1, 8]");
    if (n_pts < 0 || n_pts > ((int64_t)1 << 38))
        return report_error(SDFDDGI_ERR_INVALID_ARG, "sample_irradiance_cascade: n_pts out of range");
    if (n_pts > 0 && (!points || !normals || !out_rgb))
        return report_error(SDFDDGI_ERR_INVALID_ARG, "sample_irradiance_cascade: NULL array");
    if (!(softness >= 0.f) || !std::isfinite(softness))
        return report_error(SDFDDGI_ERR_INVALID_ARG, "sample_irradiance_cascade: softness must be >= 0 and finite");
    CascadeArgs a{};
    a.n = n;
    const bool visible = softness > 0.f;
    for (int j = 0; j < n; ++j) {
        const sdfddgi_volume* v = volumes[j];
        if (!v) return report_error(SDFDDGI_ERR_INVALID_ARG, "sample_irradiance_cascade: a volume is NULL");
        CascadeVol& c = a.v[j];
        for (int k = 0; k < 3; ++k) {
            c.gdims[k] = v->desc.dims[k];
            c.gorigin[k] = v->desc.origin[k];
            c.gspacing[k] = v->desc.spacing[k];
        }
        c.irr = v->irr[v->cur];
        c.valid = v->valid[v->cur];
        // the farthest level is never tested for visibility (Sec. 3.5)
        c.visible = visible && j < n - 1;
        if (c.visible) {
            const sdfddgi_scene* s = v->scene;
            if (!s || !s->has_sdf)
                return report_error(SDFDDGI_ERR_STATE, "sample_irradiance_cascade: a volume's scene holds no SDF yet");
            scene_view(s, &c.vis.vol);
            c.vis.softness = softness;
            c.vis.eps_w = v->desc.eps * s->h;
            c.vis.bias_w = v->desc.normal_bias * s->h;
            c.vis.max_steps = v->desc.max_steps;
            c.vis.states = states ? states[j] : nullptr;
        }
    }
    if (n_pts == 0) return SDFDDGI_OK;
    a.points = points;
    a.normals = normals;
    a.out = out_rgb;
    a.level = out_level;
    a.weight = out_weight;
    a.n_pts = n_pts;
    const int64_t blocks = std::min<int64_t>((n_pts + 255) / 256, 148 * 32);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (visible)
        cascade_kernel<true><<<(unsigned)blocks, 256, 0, st>>>(a);
    else
        cascade_kernel<false><<<(unsigned)blocks, 256, 0, st>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return report_error(SDFDDGI_ERR_CUDA, cudaGetErrorString(e));
    return SDFDDGI_OK;
}
