// relocate.cu -- probe relocation (Sec. 3.2, the procedure UpdateProbePos), one thread
// per probe. A probe whose grid position lies nearer than the clearance to a surface
// takes Gauss-Newton steps on (c - sdf(p))^2 / 2 toward the level set sdf = c,
//     p <- p + (c - sdf(p)) g / |g|^2,  g = central differences of the trilinear SDF at
//     +-h/2 divided by h (the shading normal's rule),
// each followed by a clamp of every coordinate to within max_offset * spacing of the grid
// position; it stops once sdf(p) >= c, when the gradient vanishes, or after
// max_iterations steps. The probe ends active iff its SDF then exceeds the minimum
// clearance, and its history is rejected iff it lies farther than the rejection distance
// from last frame's position.
#include <cmath>

#include "device.cuh"
#include "handles.h"

using namespace sdfddgi;

namespace {

struct RelocArgs {
    VolumeView vol;
    int gdims[3];
    float gorigin[3];
    float gspacing[3];
    float c;          // clearance, world units
    float reject;     // rejection distance, world units (<= 0: never)
    float lim[3];     // per-axis displacement limit, world units
    float min_c;      // minimum clearance, world units
    int max_iters;
    int P;
    const sdfddgi_probe_state* last;
    sdfddgi_probe_state* out;
};

template <typename T>
__global__ void __launch_bounds__(256) relocate_kernel(const __grid_constant__ RelocArgs a) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.P) return;
    const int ix = p % a.gdims[0], iy = (p / a.gdims[0]) % a.gdims[1], iz = p / (a.gdims[0] * a.gdims[1]);
    const float3 home = f3(fmaf((float)ix, a.gspacing[0], a.gorigin[0]), fmaf((float)iy, a.gspacing[1], a.gorigin[1]),
                           fmaf((float)iz, a.gspacing[2], a.gorigin[2]));
    float3 last = home;
    if (a.last) last = f3(a.last[p].pos[0], a.last[p].pos[1], a.last[p].pos[2]);
    float3 pos = home;
    const float hh = 0.5f * a.vol.h;
    if (a.c > 0.f) {
        for (int it = 0; it < a.max_iters; ++it) {
            const float s = sample_sdf<T>(a.vol, pos);
            if (s >= a.c) break;
            const float gx = (sample_sdf<T>(a.vol, f3(pos.x + hh, pos.y, pos.z)) -
                              sample_sdf<T>(a.vol, f3(pos.x - hh, pos.y, pos.z))) * a.vol.inv_h;
            const float gy = (sample_sdf<T>(a.vol, f3(pos.x, pos.y + hh, pos.z)) -
                              sample_sdf<T>(a.vol, f3(pos.x, pos.y - hh, pos.z))) * a.vol.inv_h;
            const float gz = (sample_sdf<T>(a.vol, f3(pos.x, pos.y, pos.z + hh)) -
                              sample_sdf<T>(a.vol, f3(pos.x, pos.y, pos.z - hh))) * a.vol.inv_h;
            const float g2 = gx * gx + gy * gy + gz * gz;
            if (!(g2 > 0.f)) break;
            const float k = (a.c - s) / g2;
            pos.x = fminf(fmaxf(fmaf(k, gx, pos.x), home.x - a.lim[0]), home.x + a.lim[0]);
            pos.y = fminf(fmaxf(fmaf(k, gy, pos.y), home.y - a.lim[1]), home.y + a.lim[1]);
            pos.z = fminf(fmaxf(fmaf(k, gz, pos.z), home.z - a.lim[2]), home.z + a.lim[2]);
        }
    }
    uint32_t flags = sample_sdf<T>(a.vol, pos) > a.min_c ? (uint32_t)SDFDDGI_PROBE_ACTIVE : 0u;
    const float3 dv = pos - last;
    if (a.reject > 0.f && sqrtf(dot(dv, dv)) > a.reject) flags |= SDFDDGI_PROBE_REJECT_HISTORY;
    sdfddgi_probe_state o;
    o.pos[0] = pos.x;
    o.pos[1] = pos.y;
    o.pos[2] = pos.z;
    o.flags = flags;
    a.out[p] = o;
}

bool finite_nonneg(float x) { return std::isfinite(x) && x >= 0.f; }

}  // namespace

extern "C" SDFDDGI_API int sdfddgi_relocate_probes(const sdfddgi_volume* v, const sdfddgi_relocation* r,
                                                   const sdfddgi_probe_state* last, sdfddgi_probe_state* out,
                                                   void* stream) {
    if (!v || !r || !out) return report_error(SDFDDGI_ERR_INVALID_ARG, "relocate_probes: NULL argument");
    if (!std::isfinite(r->clearance) || !std::isfinite(r->reject_distance) || !finite_nonneg(r->min_clearance) ||
        !(r->max_offset >= 0.f && r->max_offset <= 0.5f) || r->max_iterations < 0 || r->max_iterations > 64)
        return report_error(SDFDDGI_ERR_INVALID_ARG,
                            "relocate_probes: clearance and reject_distance finite, min_clearance >= 0, "
                            "max_offset in [0, 0.5], max_iterations in [0, 64]");
    const sdfddgi_scene* s = v->scene;
    if (!s || !s->has_sdf) return report_error(SDFDDGI_ERR_STATE, "relocate_probes: the scene holds no SDF yet");
    if (v->P == 0) return SDFDDGI_OK;
    RelocArgs a{};
    scene_view(s, &a.vol);
    for (int k = 0; k < 3; ++k) {
        a.gdims[k] = v->desc.dims[k];
        a.gorigin[k] = v->desc.origin[k];
        a.gspacing[k] = v->desc.spacing[k];
        a.lim[k] = r->max_offset * v->desc.spacing[k];
    }
    a.c = r->clearance * s->h;
    a.reject = r->reject_distance;
    a.min_c = r->min_clearance * s->h;
    a.max_iters = r->max_iterations;
    a.P = (int)v->P;
    a.last = last;
    a.out = out;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned blocks = (unsigned)((a.P + 255) / 256);
    if (s->dtype == kAnalytic)
        relocate_kernel<Analytic><<<blocks, 256, 0, st>>>(a);
    else if (s->dtype == SDFDDGI_F16)
        relocate_kernel<__half><<<blocks, 256, 0, st>>>(a);
    else
        relocate_kernel<float><<<blocks, 256, 0, st>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return report_error(SDFDDGI_ERR_CUDA, cudaGetErrorString(e));
    return SDFDDGI_OK;
}
