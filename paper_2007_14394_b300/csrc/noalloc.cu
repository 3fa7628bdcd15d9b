// noalloc.cu -- the probe update for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc once they are running: a renderer or game engine
// that reserves all device memory up front and hands out sub-ranges of its own pools, a
// plug-in living inside another framework's memory manager, or a real-time loop where an
// allocation (which may synchronise the device) would break the frame budget. For them,
// sdfddgi_update_probes_noalloc runs the same kernels as sdfddgi_update_probes (the stages
// serially on the caller's stream, which gives the same maps bit for bit as the slab
// branches), taking every input and output buffer from the caller; the stages' scratch (the
// SDF's xy-quad copy, per-ray buffers, shadow-task list, texel weights and their tensor-core
// image, pool counters) lives in one file-scope __device__ array of kScratchBytes that
// every GPU loading this library holds until the process exits.
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "internal.h"

using namespace sdfddgi;

namespace {

constexpr size_t kScratchBytes = (size_t)32 << 20;  // 32 MiB per device
constexpr int kMaxDevices = 64;

// In host code this name is only a stand-in for the device array: kernels get the
// device address obtained from cudaGetSymbolAddress below, never &g_scratch.
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Failures are reported through sdfddgi_last_error(), like every other entry point.
int nofail(int code, const char* fmt, ...) {
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    return report_error(code, msg);
}

// Device address of the scratch array on the current device, looked up once per device.
int scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return nofail(SDFDDGI_ERR_CUDA, "update_probes_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return nofail(SDFDDGI_ERR_CUDA, "update_probes_noalloc: device %d not supported", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return nofail(SDFDDGI_ERR_CUDA, "update_probes_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
        e = prepare_update_kernels();  // the kernels' one-time set-up, on the same first call
        if (e != cudaSuccess)
            return nofail(SDFDDGI_ERR_CUDA, "update_probes_noalloc: kernel set-up: %s", cudaGetErrorString(e));
    }
    *out = g_scratch_ptr[dev];
    return SDFDDGI_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool pos_finite(float x) { return std::isfinite(x) && x > 0.f; }

// Do the byte ranges [a, a + na) and [b, b + nb) share a byte?
bool overlap(const void* a, size_t na, const void* b, size_t nb) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

constexpr uint32_t kAcceptedFlags = SDFDDGI_FLAG_BLEND_BF16 | SDFDDGI_FLAG_RELAXED_SHADOW | SDFDDGI_FLAG_RELAXED_PRIMARY;

}  // namespace

extern "C" {

SDFDDGI_API int sdfddgi_update_probes_noalloc(
    const sdfddgi_volume_desc* d, const void* sdf, const int32_t dims[3], float voxel_size, const float origin[3],
    int32_t dtype, const void* material, const sdfddgi_light* lights, int32_t n_lights, const float sky_rgb[3],
    uint32_t frame, const float* rotation, const sdfddgi_probe_state* states, const float* prev_irr,
    const float* prev_depth, const uint8_t* prev_valid, float* cur_irr, float* cur_depth, uint8_t* cur_valid,
    sdfddgi_ray_record* records, void* stream) {
    // ---- arguments (all checked before any device work)
    if (!d || !sdf || !dims || !origin || !prev_irr || !prev_depth || !prev_valid || !cur_irr || !cur_depth ||
        !cur_valid)
        return nofail(SDFDDGI_ERR_INVALID_ARG, "update_probes_noalloc: NULL argument");
    if (dtype != SDFDDGI_F32 && dtype != SDFDDGI_F16)
        return nofail(SDFDDGI_ERR_INVALID_ARG, "update_probes_noalloc: dtype must be F32 or F16");
    if (!pos_finite(voxel_size)) return nofail(SDFDDGI_ERR_INVALID_ARG, "update_probes_noalloc: voxel_size must be > 0");
    int64_t P = 1;
    for (int a = 0; a < 3; ++a) {
        if (dims[a] < 2 || dims[a] > 16384 || !std::isfinite(origin[a]))
            return nofail(SDFDDGI_ERR_INVALID_ARG, "update_probes_noalloc: SDF dims must be in [2, 16384]");
        if (d->dims[a] < 1 || !pos_finite(d->spacing[a]) || !std::isfinite(d->origin[a]))
            return nofail(SDFDDGI_ERR_INVALID_ARG, "update_probes_noalloc: invalid probe grid");
        P *= d->dims[a];  // each factor < 2^31 and P <= 2^31 - 1 so far: no overflow
        if (P > INT32_MAX)
            return nofail(SDFDDGI_ERR_INVALID_ARG, "update_probes_noalloc: more than 2^31-1 probes");
    }
    const int R = d->rays_per_probe;
    if (R < 1 || R > SDFDDGI_MAX_RAYS || d->max_steps < 1 || d->max_steps > SDFDDGI_MAX_STEPS ||
        d->depth_exponent < 1 || d->depth_exponent > 1024 || !pos_finite(d->eps) || !std::isfinite(d->t_max) ||
        !(d->hysteresis >= 0.f && d->hysteresis <= 1.f) || !(d->multibounce_k >= 0.f && d->multibounce_k <= 1.f) ||
        !(d->normal_bias >= 0.f) || !std::isfinite(d->normal_bias))
        return nofail(SDFDDGI_ERR_INVALID_ARG, "update_probes_noalloc: invalid volume description");
    if (d->flags & ~kAcceptedFlags)
        return nofail(SDFDDGI_ERR_INVALID_ARG,
                      "update_probes_noalloc: flags 0x%x: only BLEND_BF16 and the RELAXED_* flags are accepted",
                      (unsigned)d->flags);
    if (P * R > ((int64_t)1 << 27))
        return nofail(SDFDDGI_ERR_INVALID_ARG, "update_probes_noalloc: more than 2^27 probe rays");
    if (n_lights < 0 || n_lights > SDFDDGI_MAX_LIGHTS || (n_lights > 0 && !lights))
        return nofail(SDFDDGI_ERR_INVALID_ARG, "update_probes_noalloc: n_lights must be in [0, 32]");
    if (rotation)
        for (int k = 0; k < 9; ++k)
            if (!std::isfinite(rotation[k]))
                return nofail(SDFDDGI_ERR_INVALID_ARG, "update_probes_noalloc: rotation not finite");
    {  // the new maps must not share memory with the previous ones, nor with each other
        const size_t irr_b = (size_t)P * kIrrT * kIrrT * 16, dep_b = (size_t)P * kDepT * kDepT * 8, val_b = (size_t)P;
        const void* in[3] = {prev_irr, prev_depth, prev_valid};
        const void* out[3] = {cur_irr, cur_depth, cur_valid};
        const size_t nb[3] = {irr_b, dep_b, val_b};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                if (overlap(out[i], nb[i], in[j], nb[j]) || (j > i && overlap(out[i], nb[i], out[j], nb[j])))
                    return nofail(SDFDDGI_ERR_INVALID_ARG,
                                  "update_probes_noalloc: the cur_* maps overlap the prev_* maps or each other");
    }

    // ---- scratch layout and its limit
    const size_t n_vox = (size_t)dims[0] * dims[1] * dims[2];
    const size_t n_rays = (size_t)P * R;
    const size_t sizes[] = {quad_bytes(dtype, dims),
                            n_rays * 4,   // ray_t
                            n_rays * 4,   // ray_es
                            n_rays * 16,  // ray_n
                            n_rays * 16,  // ray_alb
                            n_rays * 16,  // ray_base
                            n_rays * 4,   // ray_lit
                            n_rays * 4,   // ray_ssteps
                            n_rays * 16 * (size_t)(n_lights > 0 ? n_lights : 1),  // tasks
                            kCounterWords * 4,  // counters
                            weights_bytes(R),   // texel weights, their sums, ray directions
                            wimage_bytes(R),    // the weights as the tensor-core gather's operand
                            n_rays * 4 * (size_t)(n_lights > 0 ? n_lights : 1),  // task light factors
                            n_rays * 4};        // finalize list
    size_t off[sizeof sizes / sizeof sizes[0]], total = 0;
    for (size_t k = 0; k < sizeof sizes / sizeof sizes[0]; ++k) {
        off[k] = total;
        total += align256(sizes[k]);
    }
    if (total > kScratchBytes)
        return nofail(SDFDDGI_ERR_INVALID_ARG,
                      "update_probes_noalloc: this update needs %zu bytes of scratch; the fixed scratch holds %zu "
                      "(%zu voxels, %zu probe rays, %d lights)",
                      total, kScratchBytes, n_vox, n_rays, n_lights);

    UpdateParams p;
    std::memset(&p, 0, sizeof p);
    for (int l = 0; l < n_lights; ++l) {
        const sdfddgi_light& li = lights[l];
        if (li.type != SDFDDGI_LIGHT_DIRECTIONAL && li.type != SDFDDGI_LIGHT_POINT)
            return nofail(SDFDDGI_ERR_INVALID_ARG, "update_probes_noalloc: light %d has an unknown type", l);
        if (li.type == SDFDDGI_LIGHT_POINT && !pos_finite(li.range))
            return nofail(SDFDDGI_ERR_INVALID_ARG, "update_probes_noalloc: light %d range must be > 0", l);
        p.lights[l].type = li.type;
        for (int a = 0; a < 3; ++a) {
            p.lights[l].v[a] = li.v[a];
            p.lights[l].rgb[a] = li.rgb[a];
        }
        p.lights[l].range = li.range;
    }
    p.n_lights = n_lights;
    if (rotation) {
        for (int k = 0; k < 9; ++k) p.rot[k] = rotation[k];
    } else {
        sdfddgi_frame_rotation(d->seed, frame, d->volume_id, p.rot);
    }

    // ---- the scratch array (first call on a device looks its address up)
    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    unsigned char* s = static_cast<unsigned char*>(base);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = build_quads(sdf, s + off[0], dtype, dims, st);
    if (e != cudaSuccess) return nofail(SDFDDGI_ERR_CUDA, "update_probes_noalloc: %s", cudaGetErrorString(e));

    VolumeView& vol = p.vol;
    vol.quads = s + off[0];
    vol.material = static_cast<const uint4*>(material);
    vol.nx = dims[0];
    vol.ny = dims[1];
    vol.nz = dims[2];
    vol.dtype = dtype;
    vol.h = voxel_size;
    vol.inv_h = 1.0f / voxel_size;
    set_trace_constants(&vol);
    for (int a = 0; a < 3; ++a) {
        vol.lo[a] = origin[a];
        vol.hi[a] = origin[a] + (float)dims[a] * voxel_size;
        p.sky[a] = sky_rgb ? sky_rgb[a] : 0.f;
        p.gdims[a] = d->dims[a];
        p.gorigin[a] = d->origin[a];
        p.gspacing[a] = d->spacing[a];
    }
    p.P = (int)P;
    p.R = R;
    p.max_steps = d->max_steps;
    p.depth_exp = d->depth_exponent;
    p.eps_w = d->eps * voxel_size;
    const double diag = std::sqrt((double)dims[0] * dims[0] + (double)dims[1] * dims[1] + (double)dims[2] * dims[2]);
    p.tmax_w = (d->t_max > 0.f ? d->t_max : (float)diag) * voxel_size;
    p.hyst = d->hysteresis;
    p.k_bounce = d->multibounce_k;
    p.bias_w = d->normal_bias * voxel_size;
    p.states = states;
    p.prev_irr = reinterpret_cast<const float4*>(prev_irr);
    p.prev_depth = reinterpret_cast<const float2*>(prev_depth);
    p.prev_valid = prev_valid;
    p.cur_irr = reinterpret_cast<float4*>(cur_irr);
    p.cur_depth = reinterpret_cast<float2*>(cur_depth);
    p.cur_valid = cur_valid;
    p.records = records;
    p.ray_t = reinterpret_cast<float*>(s + off[1]);
    p.ray_es = reinterpret_cast<uint32_t*>(s + off[2]);
    p.ray_n = reinterpret_cast<float4*>(s + off[3]);
    p.ray_alb = reinterpret_cast<float4*>(s + off[4]);
    p.ray_base = reinterpret_cast<float4*>(s + off[5]);
    p.ray_lit = reinterpret_cast<uint32_t*>(s + off[6]);
    p.ray_ssteps = reinterpret_cast<uint32_t*>(s + off[7]);
    p.tasks = reinterpret_cast<float4*>(s + off[8]);
    p.task_capacity = (uint32_t)(n_rays * (size_t)(n_lights > 0 ? n_lights : 1));
    p.counters = reinterpret_cast<uint32_t*>(s + off[9]);
    p.weights = reinterpret_cast<float*>(s + off[10]);
    p.wimage = s + off[11];
    p.task_scale = reinterpret_cast<float*>(s + off[12]);
    p.fin_list = reinterpret_cast<uint32_t*>(s + off[13]);
    p.blend_bf16 = (d->flags & SDFDDGI_FLAG_BLEND_BF16) ? 1 : 0;
    p.omega_primary = (d->flags & SDFDDGI_FLAG_RELAXED_PRIMARY) ? SDFDDGI_RELAX_OMEGA : 1.f;
    p.omega_shadow = (d->flags & SDFDDGI_FLAG_RELAXED_SHADOW) ? SDFDDGI_RELAX_OMEGA : 1.f;
    e = cudaMemsetAsync(p.counters, 0, kCounterWords * sizeof(uint32_t), st);  // the scratch is shared: no sticky bits
    if (e == cudaSuccess) e = launch_update(p, st);
    if (e != cudaSuccess) return nofail(SDFDDGI_ERR_CUDA, "update_probes_noalloc: launch failed: %s", cudaGetErrorString(e));
    return SDFDDGI_OK;
}

}  // extern "C"
