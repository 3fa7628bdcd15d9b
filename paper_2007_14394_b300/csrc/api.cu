// api.cu -- host side of the C ABI declared in include/sdfddgi.h.
//
// Owns the scene storage (SDF + material volume, lights) and the probe volumes'
// ping-pong maps in device memory, validates every argument before enqueuing
// work, and turns CUDA failures into status codes with a thread-local message.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "handles.h"

using namespace sdfddgi;

namespace {

thread_local char g_error[1024] = "";

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_error, sizeof g_error, fmt, ap);
    va_end(ap);
    return code;
}

#define CUDA_TRY(call)                                                                            \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return fail(SDFDDGI_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

int alloc(void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(SDFDDGI_ERR_OOM, "cudaMalloc of %zu bytes failed: out of device memory", bytes);
    }
    if (e != cudaSuccess) return fail(SDFDDGI_ERR_CUDA, "cudaMalloc: %s", cudaGetErrorString(e));
    return SDFDDGI_OK;
}

bool finite_pos(float x) { return std::isfinite(x) && x > 0.f; }

constexpr size_t kIrrBytes = sizeof(float4) * kIrrT * kIrrT;
constexpr size_t kDepBytes = sizeof(float2) * kDepT * kDepT;

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

void free_volume_buffers(sdfddgi_volume* v) {
    for (int k = 0; k < 2; ++k) {
        cudaFree(v->irr[k]);
        cudaFree(v->depth[k]);
        cudaFree(v->valid[k]);
        v->irr[k] = nullptr;
        v->depth[k] = nullptr;
        v->valid[k] = nullptr;
    }
    cudaFree(v->states);
    v->states = nullptr;
    void* scratch[] = {v->ray_t, v->ray_es, v->ray_n, v->ray_alb, v->ray_base, v->ray_lit, v->ray_ssteps,
                       v->counters, v->tasks, v->task_scale, v->fin_list, v->weights, v->wimage};
    for (void* q : scratch) cudaFree(q);
    for (int c = 0; c < kMaxSlabs - 1; ++c) {
        if (v->lanes.side[c]) cudaStreamDestroy(v->lanes.side[c]);
        if (v->lanes.join[c]) cudaEventDestroy(v->lanes.join[c]);
    }
    if (v->lanes.fork) cudaEventDestroy(v->lanes.fork);
    if (v->lanes.weights_ready) cudaEventDestroy(v->lanes.weights_ready);
    v->lanes = {};
    if (v->copy) cudaStreamDestroy(v->copy);
    if (v->read_order) cudaEventDestroy(v->read_order);
    for (int b = 0; b < 2; ++b)
        if (v->read_done[b]) cudaEventDestroy(v->read_done[b]);
    v->copy = nullptr;
    v->read_order = v->read_done[0] = v->read_done[1] = nullptr;
    v->weights = nullptr;
    v->wimage = nullptr;
    v->ray_t = nullptr;
    v->ray_es = nullptr;
    v->ray_n = v->ray_alb = v->ray_base = nullptr;
    v->ray_lit = v->ray_ssteps = v->counters = nullptr;
    v->tasks = nullptr;
    v->task_scale = nullptr;
    v->fin_list = nullptr;
    v->task_capacity = 0;
}

int alloc_scratch(sdfddgi_volume* v) {
    const size_t n = (size_t)v->P * v->desc.rays_per_probe;
    int rc = alloc((void**)&v->ray_t, n * sizeof(float));
    if (!rc) rc = alloc((void**)&v->ray_es, n * sizeof(uint32_t));
    if (!rc) rc = alloc((void**)&v->ray_n, n * sizeof(float4));
    if (!rc) rc = alloc((void**)&v->ray_alb, n * sizeof(float4));
    if (!rc) rc = alloc((void**)&v->ray_base, n * sizeof(float4));
    if (!rc) rc = alloc((void**)&v->ray_lit, n * sizeof(uint32_t));
    if (!rc) rc = alloc((void**)&v->ray_ssteps, n * sizeof(uint32_t));
    if (!rc) rc = alloc((void**)&v->fin_list, n * sizeof(uint32_t));
    if (!rc) rc = alloc((void**)&v->counters, kMaxSlabs * kSlabCounterStride * sizeof(uint32_t));
    if (!rc) rc = alloc((void**)&v->weights, weights_bytes(v->desc.rays_per_probe));
    if (!rc) rc = alloc(&v->wimage, wimage_bytes(v->desc.rays_per_probe));
    return rc;
}

// The shadow-task list holds at most one task per (ray, light) pair.
int ensure_task_capacity(sdfddgi_volume* v, int n_lights) {
    const size_t need = (size_t)v->P * v->desc.rays_per_probe * (size_t)(n_lights > 0 ? n_lights : 1);
    if (need <= v->task_capacity) return SDFDDGI_OK;
    cudaFree(v->tasks);
    cudaFree(v->task_scale);
    v->tasks = nullptr;
    v->task_scale = nullptr;
    v->task_capacity = 0;
    int rc = alloc((void**)&v->tasks, need * sizeof(float4));
    if (!rc) rc = alloc((void**)&v->task_scale, need * sizeof(float));
    if (!rc) v->task_capacity = need;
    return rc;
}

uint64_t splitmix64_next(uint64_t* state) {
    *state += 0x9E3779B97F4A7C15ull;
    uint64_t z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

int sdfddgi::report_error(int code, const char* msg) { return fail(code, "%s", msg); }

extern "C" {

SDFDDGI_API const char* sdfddgi_last_error(void) { return g_error; }

// ------------------------------------------------------------------------------ scene
SDFDDGI_API int sdfddgi_create_scene(sdfddgi_scene** out) {
    if (!out) return fail(SDFDDGI_ERR_INVALID_ARG, "create_scene: out is NULL");
    *out = nullptr;
    sdfddgi_scene* s = new (std::nothrow) sdfddgi_scene();
    if (!s) return fail(SDFDDGI_ERR_OOM, "create_scene: host allocation failed");
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) {
        delete s;
        return fail(SDFDDGI_ERR_CUDA, "create_scene: cudaGetDevice: %s", cudaGetErrorString(e));
    }
    *out = s;
    return SDFDDGI_OK;
}

SDFDDGI_API void sdfddgi_destroy_scene(sdfddgi_scene* s) {
    if (!s) return;
    cudaFree(s->sdf);
    cudaFree(s->quads);
    cudaFree(s->material);
    cudaFree(s->prims);
    cudaFree(s->clusters);
    delete s;
}

SDFDDGI_API int sdfddgi_upload_sdf(sdfddgi_scene* s, const void* sdf, const int32_t dims[3], float voxel_size,
                                   const float origin[3], int32_t dtype, const void* material,
                                   int32_t is_device_ptr, void* stream) {
    if (!s || !sdf || !dims || !origin) return fail(SDFDDGI_ERR_INVALID_ARG, "upload_sdf: NULL argument");
    if (dtype != SDFDDGI_F32 && dtype != SDFDDGI_F16)
        return fail(SDFDDGI_ERR_INVALID_ARG, "upload_sdf: dtype %d is neither F32 nor F16", dtype);
    for (int a = 0; a < 3; ++a) {
        if (dims[a] < 2 || dims[a] > 16384)
            return fail(SDFDDGI_ERR_INVALID_ARG, "upload_sdf: dims[%d] = %d outside [2, 16384]", a, dims[a]);
        if (!std::isfinite(origin[a])) return fail(SDFDDGI_ERR_INVALID_ARG, "upload_sdf: origin is not finite");
    }
    if (!finite_pos(voxel_size)) return fail(SDFDDGI_ERR_INVALID_ARG, "upload_sdf: voxel_size must be > 0");
    if (is_device_ptr != 0 && is_device_ptr != 1)
        return fail(SDFDDGI_ERR_INVALID_ARG, "upload_sdf: is_device_ptr must be 0 or 1");
    const size_t n = (size_t)dims[0] * dims[1] * dims[2];
    if (n > ((size_t)1 << 34)) return fail(SDFDDGI_ERR_INVALID_ARG, "upload_sdf: volume of %zu voxels too large", n);
    const size_t sdf_bytes = n * (dtype == SDFDDGI_F32 ? 4 : 2);
    const size_t mat_bytes = n * 16;
    cudaStream_t st = as_stream(stream);

    if (s->sdf_bytes != sdf_bytes) {
        cudaFree(s->sdf);
        s->sdf = nullptr;
        s->sdf_bytes = 0;
        s->has_sdf = false;
        int rc = alloc(&s->sdf, sdf_bytes);
        if (rc) return rc;
        s->sdf_bytes = sdf_bytes;
    }
    CUDA_TRY(cudaMemcpyAsync(s->sdf, sdf, sdf_bytes, cudaMemcpyDefault, st));
    const size_t qb = quad_bytes(dtype, dims);
    if (s->quads_bytes != qb) {
        cudaFree(s->quads);
        s->quads = nullptr;
        s->quads_bytes = 0;
        s->has_sdf = false;
        int rc = alloc(&s->quads, qb);
        if (rc) return rc;
        s->quads_bytes = qb;
    }
    CUDA_TRY(build_quads(s->sdf, s->quads, dtype, dims, st));
    if (material) {
        if (s->material_bytes != mat_bytes) {
            cudaFree(s->material);
            s->material = nullptr;
            s->material_bytes = 0;
            int rc = alloc(&s->material, mat_bytes);
            if (rc) return rc;
            s->material_bytes = mat_bytes;
        }
        CUDA_TRY(cudaMemcpyAsync(s->material, material, mat_bytes, cudaMemcpyDefault, st));
    }
    if (!is_device_ptr) CUDA_TRY(cudaStreamSynchronize(st));
    for (int a = 0; a < 3; ++a) {
        s->dims[a] = dims[a];
        s->origin[a] = origin[a];
    }
    s->dtype = dtype;
    s->h = voxel_size;
    s->has_sdf = true;
    s->has_material = material != nullptr;
    s->version++;
    return SDFDDGI_OK;
}

}  // extern "C"

void sdfddgi::scene_view(const sdfddgi_scene* s, VolumeView* v) {
    std::memset(v, 0, sizeof *v);
    v->dtype = s->dtype;
    v->nx = s->dims[0];
    v->ny = s->dims[1];
    v->nz = s->dims[2];
    v->h = s->h;
    v->inv_h = 1.0f / s->h;
    for (int a = 0; a < 3; ++a) {
        v->lo[a] = s->origin[a];
        v->hi[a] = s->origin[a] + (float)s->dims[a] * s->h;
    }
    set_trace_constants(v);
    if (s->dtype == kAnalytic) {
        v->prims = s->prims;
        v->clusters = s->clusters;
        v->n_unbounded = s->n_unbounded;
        v->n_clusters = s->n_clusters;
    } else {
        v->quads = s->quads;
        v->material = s->has_material ? static_cast<const uint4*>(s->material) : nullptr;
    }
}

extern "C" {

SDFDDGI_API int sdfddgi_set_lights(sdfddgi_scene* s, const sdfddgi_light* lights, int32_t n, const float sky_rgb[3]) {
    if (!s) return fail(SDFDDGI_ERR_INVALID_ARG, "set_lights: scene is NULL");
    if (n < 0 || n > SDFDDGI_MAX_LIGHTS)
        return fail(SDFDDGI_ERR_INVALID_ARG, "set_lights: %d lights outside [0, %d]", n, SDFDDGI_MAX_LIGHTS);
    if (n > 0 && !lights) return fail(SDFDDGI_ERR_INVALID_ARG, "set_lights: lights is NULL");
    LightDev tmp[SDFDDGI_MAX_LIGHTS] = {};
    for (int l = 0; l < n; ++l) {
        const sdfddgi_light& li = lights[l];
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(li.v[a]) || !std::isfinite(li.rgb[a]) || li.rgb[a] < 0.f)
                return fail(SDFDDGI_ERR_INVALID_ARG, "set_lights: light %d has a non-finite or negative field", l);
        if (li.type == SDFDDGI_LIGHT_DIRECTIONAL) {
            const double len = std::sqrt((double)li.v[0] * li.v[0] + (double)li.v[1] * li.v[1] + (double)li.v[2] * li.v[2]);
            if (std::fabs(len - 1.0) > 1e-3)
                return fail(SDFDDGI_ERR_INVALID_ARG, "set_lights: light %d direction is not a unit vector", l);
        } else if (li.type == SDFDDGI_LIGHT_POINT) {
            if (!finite_pos(li.range)) return fail(SDFDDGI_ERR_INVALID_ARG, "set_lights: light %d range must be > 0", l);
        } else {
            return fail(SDFDDGI_ERR_INVALID_ARG, "set_lights: light %d has unknown type %d", l, li.type);
        }
        tmp[l].type = li.type;
        for (int a = 0; a < 3; ++a) {
            tmp[l].v[a] = li.v[a];
            tmp[l].rgb[a] = li.rgb[a];
        }
        tmp[l].range = li.range;
    }
    float sky[3] = {0.f, 0.f, 0.f};
    if (sky_rgb)
        for (int a = 0; a < 3; ++a) {
            if (!std::isfinite(sky_rgb[a]) || sky_rgb[a] < 0.f)
                return fail(SDFDDGI_ERR_INVALID_ARG, "set_lights: sky radiance must be finite and >= 0");
            sky[a] = sky_rgb[a];
        }
    std::memcpy(s->lights, tmp, sizeof tmp);
    s->n_lights = n;
    std::memcpy(s->sky, sky, sizeof sky);
    s->version++;
    return SDFDDGI_OK;
}

// ------------------------------------------------------------------------------ volume
SDFDDGI_API int sdfddgi_create_volume(const sdfddgi_volume_desc* d, sdfddgi_scene* s, sdfddgi_volume** out) {
    if (!d || !s || !out) return fail(SDFDDGI_ERR_INVALID_ARG, "create_volume: NULL argument");
    *out = nullptr;
    int64_t P = 1;
    for (int a = 0; a < 3; ++a) {
        if (d->dims[a] < 1) return fail(SDFDDGI_ERR_INVALID_ARG, "create_volume: dims[%d] = %d < 1", a, d->dims[a]);
        if (!finite_pos(d->spacing[a])) return fail(SDFDDGI_ERR_INVALID_ARG, "create_volume: spacing must be > 0");
        if (!std::isfinite(d->origin[a])) return fail(SDFDDGI_ERR_INVALID_ARG, "create_volume: origin not finite");
        P *= d->dims[a];
    }
    if (P > INT32_MAX) return fail(SDFDDGI_ERR_INVALID_ARG, "create_volume: %lld probes exceed 2^31-1", (long long)P);
    if (P * (int64_t)(d->rays_per_probe > 0 ? d->rays_per_probe : 1) > ((int64_t)1 << 27))
        return fail(SDFDDGI_ERR_INVALID_ARG, "create_volume: probes x rays_per_probe exceeds 2^27");
    if (d->rays_per_probe < 1 || d->rays_per_probe > SDFDDGI_MAX_RAYS)
        return fail(SDFDDGI_ERR_INVALID_ARG, "create_volume: rays_per_probe %d outside [1, %d]", d->rays_per_probe,
                    SDFDDGI_MAX_RAYS);
    if (d->max_steps < 1 || d->max_steps > SDFDDGI_MAX_STEPS)
        return fail(SDFDDGI_ERR_INVALID_ARG, "create_volume: max_steps %d outside [1, %d]", d->max_steps,
                    SDFDDGI_MAX_STEPS);
    if (d->depth_exponent < 1 || d->depth_exponent > 1024)
        return fail(SDFDDGI_ERR_INVALID_ARG, "create_volume: depth_exponent %d outside [1, 1024]", d->depth_exponent);
    if (!finite_pos(d->eps)) return fail(SDFDDGI_ERR_INVALID_ARG, "create_volume: eps must be > 0");
    if (!std::isfinite(d->t_max)) return fail(SDFDDGI_ERR_INVALID_ARG, "create_volume: t_max not finite");
    if (!(d->hysteresis >= 0.f && d->hysteresis <= 1.f))
        return fail(SDFDDGI_ERR_INVALID_ARG, "create_volume: hysteresis outside [0, 1]");
    if (!(d->multibounce_k >= 0.f && d->multibounce_k <= 1.f))
        return fail(SDFDDGI_ERR_INVALID_ARG, "create_volume: multibounce_k outside [0, 1]");
    if (!(d->normal_bias >= 0.f) || !std::isfinite(d->normal_bias))
        return fail(SDFDDGI_ERR_INVALID_ARG, "create_volume: normal_bias must be >= 0");
    if (d->flags & ~(uint32_t)(SDFDDGI_FLAG_BLEND_BF16 | SDFDDGI_FLAG_RELAXED_SHADOW | SDFDDGI_FLAG_RELAXED_PRIMARY |
                               SDFDDGI_FLAG_TEST_GATHER_STALL))
        return fail(SDFDDGI_ERR_INVALID_ARG, "create_volume: unknown flags 0x%x", d->flags);

    sdfddgi_volume* v = new (std::nothrow) sdfddgi_volume();
    if (!v) return fail(SDFDDGI_ERR_OOM, "create_volume: host allocation failed");
    v->desc = *d;
    v->scene = s;
    v->P = P;
    int rc = SDFDDGI_OK;
    for (int k = 0; k < 2 && rc == SDFDDGI_OK; ++k) {
        if (!rc) rc = alloc((void**)&v->irr[k], P * kIrrBytes);
        if (!rc) rc = alloc((void**)&v->depth[k], P * kDepBytes);
        if (!rc) rc = alloc((void**)&v->valid[k], (size_t)P);
    }
    if (!rc) rc = alloc((void**)&v->states, sizeof(sdfddgi_probe_state) * P);
    if (!rc) rc = alloc_scratch(v);
    if (!rc) {
        cudaError_t e = cudaEventCreateWithFlags(&v->lanes.fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v->lanes.weights_ready, cudaEventDisableTiming);
        for (int c = 0; c < kMaxSlabs - 1 && e == cudaSuccess; ++c) {
            e = cudaStreamCreateWithFlags(&v->lanes.side[c], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v->lanes.join[c], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&v->copy, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v->read_order, cudaEventDisableTiming);
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaEventCreateWithFlags(&v->read_done[b], cudaEventDisableTiming);
        if (e != cudaSuccess) rc = fail(SDFDDGI_ERR_CUDA, "create_volume: %s", cudaGetErrorString(e));
    }
    if (rc) {
        free_volume_buffers(v);
        delete v;
        return rc;
    }
    rc = sdfddgi_reset(v, nullptr);
    if (!rc) {
        cudaError_t e = prepare_update_kernels();  // so that later updates can be captured
        if (e == cudaSuccess) e = cudaMemset(v->counters, 0, kMaxSlabs * kSlabCounterStride * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
        if (e != cudaSuccess) rc = fail(SDFDDGI_ERR_CUDA, "create_volume: %s", cudaGetErrorString(e));
    }
    if (rc) {
        free_volume_buffers(v);
        delete v;
        return rc;
    }
    *out = v;
    return SDFDDGI_OK;
}

SDFDDGI_API void sdfddgi_destroy_volume(sdfddgi_volume* v) {
    if (!v) return;
    free_volume_buffers(v);
    delete v;
}

SDFDDGI_API int sdfddgi_volume_probe_count(const sdfddgi_volume* v, int64_t* n) {
    if (!v || !n) return fail(SDFDDGI_ERR_INVALID_ARG, "volume_probe_count: NULL argument");
    *n = v->P;
    return SDFDDGI_OK;
}

SDFDDGI_API int sdfddgi_set_slabs(sdfddgi_volume* v, int32_t slabs) {
    if (!v) return fail(SDFDDGI_ERR_INVALID_ARG, "set_slabs: volume is NULL");
    if (slabs < 0 || slabs > SDFDDGI_MAX_SLABS)
        return fail(SDFDDGI_ERR_INVALID_ARG, "set_slabs: slabs must be in [0, %d]", SDFDDGI_MAX_SLABS);
    v->slabs = slabs;
    return SDFDDGI_OK;
}

SDFDDGI_API int sdfddgi_volume_slabs(const sdfddgi_volume* v, int32_t* slabs) {
    if (!v || !slabs) return fail(SDFDDGI_ERR_INVALID_ARG, "volume_slabs: NULL argument");
    UpdateParams p;
    std::memset(&p, 0, sizeof p);
    for (int a = 0; a < 3; ++a) p.gdims[a] = v->desc.dims[a];
    p.P = (int)v->P;
    p.R = v->desc.rays_per_probe;
    p.sched.slabs = v->slabs;
    *slabs = slab_count(p, true, v->has_stage_events);
    return SDFDDGI_OK;
}

SDFDDGI_API int sdfddgi_frame_rotation(uint32_t seed, uint32_t frame, uint32_t volume_id, float out[9]) {
    if (!out) return fail(SDFDDGI_ERR_INVALID_ARG, "frame_rotation: out is NULL");
    uint64_t state = (uint64_t)seed * 0x9E3779B97F4A7C15ull + (uint64_t)frame * 0xBF58476D1CE4E5B9ull +
                     (uint64_t)volume_id * 0x94D049BB133111EBull;
    double u[3];
    for (int k = 0; k < 3; ++k) u[k] = (double)(splitmix64_next(&state) >> 11) * (1.0 / 9007199254740992.0);
    const double two_pi = 6.283185307179586476925;
    const double a = std::sqrt(1.0 - u[0]), b = std::sqrt(u[0]);
    const double x = a * std::sin(two_pi * u[1]), y = a * std::cos(two_pi * u[1]);
    const double z = b * std::sin(two_pi * u[2]), w = b * std::cos(two_pi * u[2]);
    const double m[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - z * w),     2 * (x * z + y * w),
                         2 * (x * y + z * w),     1 - 2 * (x * x + z * z), 2 * (y * z - x * w),
                         2 * (x * z - y * w),     2 * (y * z + x * w),     1 - 2 * (x * x + y * y)};
    for (int k = 0; k < 9; ++k) out[k] = (float)m[k];
    return SDFDDGI_OK;
}

}  // extern "C"

cudaError_t sdfddgi::order_map_write(sdfddgi_volume* v, int buf, cudaStream_t stream) {
    if (!v->pending_read[buf]) return cudaSuccess;
    const cudaError_t e = cudaStreamWaitEvent(stream, v->read_done[buf], 0);
    if (e == cudaSuccess) v->pending_read[buf] = false;
    return e;
}

int sdfddgi::volume_params(sdfddgi_volume* v, UpdateParams* out) {
    sdfddgi_scene* s = v->scene;
    if (!s || !s->has_sdf) return fail(SDFDDGI_ERR_STATE, "update: the scene holds no SDF yet");
    const sdfddgi_volume_desc& d = v->desc;
    UpdateParams& p = *out;
    std::memset(&p, 0, sizeof p);
    scene_view(s, &p.vol);
    std::memcpy(p.lights, s->lights, sizeof p.lights);
    p.n_lights = s->n_lights;
    for (int a = 0; a < 3; ++a) {
        p.sky[a] = s->sky[a];
        p.gdims[a] = d.dims[a];
        p.gorigin[a] = d.origin[a];
        p.gspacing[a] = d.spacing[a];
    }
    p.P = (int)v->P;
    p.R = d.rays_per_probe;
    p.max_steps = d.max_steps;
    p.depth_exp = d.depth_exponent;
    p.eps_w = d.eps * s->h;
    const double diag = std::sqrt((double)s->dims[0] * s->dims[0] + (double)s->dims[1] * s->dims[1] +
                                  (double)s->dims[2] * s->dims[2]);
    p.tmax_w = (d.t_max > 0.f ? d.t_max : (float)diag) * s->h;
    p.hyst = d.hysteresis;
    p.k_bounce = d.multibounce_k;
    p.bias_w = d.normal_bias * s->h;
    const int prev = v->cur, next = v->cur ^ 1;
    p.prev_irr = v->irr[prev];
    p.prev_depth = v->depth[prev];
    p.prev_valid = v->valid[prev];
    p.cur_irr = v->irr[next];
    p.cur_depth = v->depth[next];
    p.cur_valid = v->valid[next];
    int rc = ensure_task_capacity(v, s->n_lights);
    if (rc) return rc;
    p.ray_t = v->ray_t;
    p.ray_es = v->ray_es;
    p.ray_n = v->ray_n;
    p.ray_alb = v->ray_alb;
    p.ray_base = v->ray_base;
    p.ray_lit = v->ray_lit;
    p.ray_ssteps = v->ray_ssteps;
    p.tasks = v->tasks;
    p.task_scale = v->task_scale;
    p.fin_list = v->fin_list;
    p.task_capacity = (uint32_t)(v->task_capacity < 0xffffffffu ? v->task_capacity : 0xffffffffu);
    p.counters = v->counters;
    p.weights = v->weights;
    p.wimage = v->wimage;
    p.blend_bf16 = (d.flags & SDFDDGI_FLAG_BLEND_BF16) ? 1 : 0;
    p.test_stall = (d.flags & SDFDDGI_FLAG_TEST_GATHER_STALL) ? 1 : 0;
    p.omega_primary = (d.flags & SDFDDGI_FLAG_RELAXED_PRIMARY) ? SDFDDGI_RELAX_OMEGA : 1.f;
    p.omega_shadow = (d.flags & SDFDDGI_FLAG_RELAXED_SHADOW) ? SDFDDGI_RELAX_OMEGA : 1.f;
    return SDFDDGI_OK;
}

extern "C" {

SDFDDGI_API int sdfddgi_update_probes(sdfddgi_volume* v, uint32_t frame, const float* rotation,
                                      const sdfddgi_probe_state* states, int32_t states_on_device,
                                      sdfddgi_ray_record* records, void* stream) {
    if (!v) return fail(SDFDDGI_ERR_INVALID_ARG, "update_probes: volume is NULL");
    if (states_on_device != 0 && states_on_device != 1)
        return fail(SDFDDGI_ERR_INVALID_ARG, "update_probes: states_on_device must be 0 or 1");
    if (rotation)
        for (int k = 0; k < 9; ++k)
            if (!std::isfinite(rotation[k])) return fail(SDFDDGI_ERR_INVALID_ARG, "update_probes: rotation not finite");
    cudaStream_t st = as_stream(stream);
    UpdateParams p;
    int rc = volume_params(v, &p);
    if (rc) return rc;
    if (rotation) {
        for (int k = 0; k < 9; ++k) p.rot[k] = rotation[k];
    } else {
        sdfddgi_frame_rotation(v->desc.seed, frame, v->desc.volume_id, p.rot);
    }
    if (states) {
        if (states_on_device) {
            p.states = states;
        } else {
            CUDA_TRY(cudaMemcpyAsync(v->states, states, sizeof(sdfddgi_probe_state) * v->P, cudaMemcpyHostToDevice, st));
            p.states = v->states;
        }
    }
    p.records = records;
    p.sched.slabs = v->slabs;
    cudaError_t e = order_map_write(v, v->cur ^ 1, st);  // the new maps replace a buffer being read?
    if (e != cudaSuccess) return fail(SDFDDGI_ERR_CUDA, "update_probes: %s", cudaGetErrorString(e));
    e = launch_update(p, st, v->has_stage_events ? v->stage_events : nullptr, &v->lanes);
    if (e != cudaSuccess) return fail(SDFDDGI_ERR_CUDA, "update_probes: launch failed: %s", cudaGetErrorString(e));
    v->cur ^= 1;
    return SDFDDGI_OK;
}

SDFDDGI_API int sdfddgi_set_stage_events(sdfddgi_volume* v, void* const* events, int32_t n) {
    if (!v) return fail(SDFDDGI_ERR_INVALID_ARG, "set_stage_events: volume is NULL");
    if (n == 0) {
        v->has_stage_events = false;
        return SDFDDGI_OK;
    }
    if (n != SDFDDGI_STAGE_EVENTS || !events)
        return fail(SDFDDGI_ERR_INVALID_ARG, "set_stage_events: pass %d events or none", SDFDDGI_STAGE_EVENTS);
    for (int k = 0; k < n; ++k) {
        if (!events[k]) return fail(SDFDDGI_ERR_INVALID_ARG, "set_stage_events: event %d is NULL", k);
        v->stage_events[k] = static_cast<cudaEvent_t>(events[k]);
    }
    v->has_stage_events = true;
    return SDFDDGI_OK;
}

SDFDDGI_API int sdfddgi_sample_irradiance(const sdfddgi_volume* v, const float* points, const float* normals,
                                          int64_t n, float* out_rgb, void* stream) {
    if (!v) return fail(SDFDDGI_ERR_INVALID_ARG, "sample_irradiance: volume is NULL");
    if (n < 0 || n > ((int64_t)1 << 38)) return fail(SDFDDGI_ERR_INVALID_ARG, "sample_irradiance: n out of range");
    if (n > 0 && (!points || !normals || !out_rgb))
        return fail(SDFDDGI_ERR_INVALID_ARG, "sample_irradiance: NULL array");
    SampleParams p;
    std::memset(&p, 0, sizeof p);
    for (int a = 0; a < 3; ++a) {
        p.gdims[a] = v->desc.dims[a];
        p.gorigin[a] = v->desc.origin[a];
        p.gspacing[a] = v->desc.spacing[a];
    }
    p.irr = v->irr[v->cur];
    p.valid = v->valid[v->cur];
    p.points = points;
    p.normals = normals;
    p.out = out_rgb;
    p.n = n;
    cudaError_t e = launch_sample(p, as_stream(stream));
    if (e != cudaSuccess) return fail(SDFDDGI_ERR_CUDA, "sample_irradiance: launch failed: %s", cudaGetErrorString(e));
    return SDFDDGI_OK;
}

SDFDDGI_API int sdfddgi_sample_irradiance_visible(const sdfddgi_volume* v, const float* points, const float* normals,
                                                  int64_t n, float softness, const sdfddgi_probe_state* states,
                                                  float* out_rgb, void* stream) {
    if (!v) return fail(SDFDDGI_ERR_INVALID_ARG, "sample_irradiance_visible: volume is NULL");
    if (n < 0 || n > ((int64_t)1 << 38))
        return fail(SDFDDGI_ERR_INVALID_ARG, "sample_irradiance_visible: n out of range");
    if (n > 0 && (!points || !normals || !out_rgb))
        return fail(SDFDDGI_ERR_INVALID_ARG, "sample_irradiance_visible: NULL array");
    if (!(softness > 0.f) || !std::isfinite(softness))
        return fail(SDFDDGI_ERR_INVALID_ARG, "sample_irradiance_visible: softness must be positive and finite");
    const sdfddgi_scene* s = v->scene;
    if (!s || !s->has_sdf) return fail(SDFDDGI_ERR_STATE, "sample_irradiance_visible: the scene holds no SDF yet");
    SampleParams p;
    std::memset(&p, 0, sizeof p);
    for (int a = 0; a < 3; ++a) {
        p.gdims[a] = v->desc.dims[a];
        p.gorigin[a] = v->desc.origin[a];
        p.gspacing[a] = v->desc.spacing[a];
    }
    p.irr = v->irr[v->cur];
    p.valid = v->valid[v->cur];
    p.points = points;
    p.normals = normals;
    p.out = out_rgb;
    p.n = n;
    VisParams vp;
    std::memset(&vp, 0, sizeof vp);
    scene_view(s, &vp.vol);
    vp.softness = softness;
    vp.eps_w = v->desc.eps * s->h;
    vp.bias_w = v->desc.normal_bias * s->h;
    vp.max_steps = v->desc.max_steps;
    vp.states = states;
    cudaError_t e = launch_sample_visible(p, vp, as_stream(stream));
    if (e != cudaSuccess)
        return fail(SDFDDGI_ERR_CUDA, "sample_irradiance_visible: launch failed: %s", cudaGetErrorString(e));
    return SDFDDGI_OK;
}

SDFDDGI_API int sdfddgi_get_maps(const sdfddgi_volume* v, const float** irr, const float** depth,
                                 const uint8_t** valid) {
    if (!v) return fail(SDFDDGI_ERR_INVALID_ARG, "get_maps: volume is NULL");
    if (irr) *irr = reinterpret_cast<const float*>(v->irr[v->cur]);
    if (depth) *depth = reinterpret_cast<const float*>(v->depth[v->cur]);
    if (valid) *valid = v->valid[v->cur];
    return SDFDDGI_OK;
}

SDFDDGI_API int sdfddgi_read_state(const sdfddgi_volume* v, float* irr, float* depth, uint8_t* valid,
                                   int32_t on_device, void* stream) {
    if (!v) return fail(SDFDDGI_ERR_INVALID_ARG, "read_state: volume is NULL");
    if (on_device != 0 && on_device != 1) return fail(SDFDDGI_ERR_INVALID_ARG, "read_state: on_device must be 0 or 1");
    cudaStream_t st = as_stream(stream);
    if (irr) CUDA_TRY(cudaMemcpyAsync(irr, v->irr[v->cur], v->P * kIrrBytes, cudaMemcpyDefault, st));
    if (depth) CUDA_TRY(cudaMemcpyAsync(depth, v->depth[v->cur], v->P * kDepBytes, cudaMemcpyDefault, st));
    if (valid) CUDA_TRY(cudaMemcpyAsync(valid, v->valid[v->cur], (size_t)v->P, cudaMemcpyDefault, st));
    if (!on_device) CUDA_TRY(cudaStreamSynchronize(st));
    return SDFDDGI_OK;
}

SDFDDGI_API int sdfddgi_read_state_async(sdfddgi_volume* v, float* irr, float* depth, uint8_t* valid, void* stream,
                                         void* done_event) {
    if (!v) return fail(SDFDDGI_ERR_INVALID_ARG, "read_state_async: volume is NULL");
    const int b = v->cur;
    // after everything enqueued on `stream` so far (the update that wrote buffer b)
    CUDA_TRY(cudaEventRecord(v->read_order, as_stream(stream)));
    CUDA_TRY(cudaStreamWaitEvent(v->copy, v->read_order, 0));
    if (irr) CUDA_TRY(cudaMemcpyAsync(irr, v->irr[b], v->P * kIrrBytes, cudaMemcpyDefault, v->copy));
    if (depth) CUDA_TRY(cudaMemcpyAsync(depth, v->depth[b], v->P * kDepBytes, cudaMemcpyDefault, v->copy));
    if (valid) CUDA_TRY(cudaMemcpyAsync(valid, v->valid[b], (size_t)v->P, cudaMemcpyDefault, v->copy));
    CUDA_TRY(cudaEventRecord(v->read_done[b], v->copy));
    v->pending_read[b] = true;
    if (done_event) CUDA_TRY(cudaEventRecord(static_cast<cudaEvent_t>(done_event), v->copy));
    return SDFDDGI_OK;
}

SDFDDGI_API int sdfddgi_write_state(sdfddgi_volume* v, const float* irr, const float* depth, const uint8_t* valid,
                                    int32_t on_device, void* stream) {
    if (!v) return fail(SDFDDGI_ERR_INVALID_ARG, "write_state: volume is NULL");
    if (!irr || !depth || !valid) return fail(SDFDDGI_ERR_INVALID_ARG, "write_state: NULL array");
    if (on_device != 0 && on_device != 1) return fail(SDFDDGI_ERR_INVALID_ARG, "write_state: on_device must be 0 or 1");
    cudaStream_t st = as_stream(stream);
    CUDA_TRY(order_map_write(v, v->cur, st));
    CUDA_TRY(cudaMemcpyAsync(v->irr[v->cur], irr, v->P * kIrrBytes, cudaMemcpyDefault, st));
    CUDA_TRY(cudaMemcpyAsync(v->depth[v->cur], depth, v->P * kDepBytes, cudaMemcpyDefault, st));
    CUDA_TRY(cudaMemcpyAsync(v->valid[v->cur], valid, (size_t)v->P, cudaMemcpyDefault, st));
    if (!on_device) CUDA_TRY(cudaStreamSynchronize(st));
    return SDFDDGI_OK;
}

SDFDDGI_API int sdfddgi_volume_status(sdfddgi_volume* v, uint32_t* flags) {
    if (flags) *flags = 0;
    if (!v) return fail(SDFDDGI_ERR_INVALID_ARG, "volume_status: volume is NULL");
    uint32_t words[kMaxSlabs * kSlabCounterStride];
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(cudaMemcpy(words, v->counters, sizeof words, cudaMemcpyDeviceToHost));
    uint32_t f = 0;  // the failure bits of every slab's counters
    for (int c = 0; c < kMaxSlabs; ++c) {
        f |= words[c * kSlabCounterStride + kFailWord];
        CUDA_TRY(cudaMemset(v->counters + c * kSlabCounterStride + kFailWord, 0, sizeof(uint32_t)));
    }
    if (flags) *flags = f;
    if (f & kFailWait) return fail(SDFDDGI_ERR_TIMEOUT, "volume_status: a bounded wait of the tensor-core gather gave up");
    if (f & kFailBounds)
        return fail(SDFDDGI_ERR_BOUNDS, "volume_status: the bounds-checked build found an index outside its buffer");
    return SDFDDGI_OK;
}

SDFDDGI_API int sdfddgi_reset(sdfddgi_volume* v, void* stream) {
    if (!v) return fail(SDFDDGI_ERR_INVALID_ARG, "reset: volume is NULL");
    cudaStream_t st = as_stream(stream);
    for (int k = 0; k < 2; ++k) {
        CUDA_TRY(order_map_write(v, k, st));
        CUDA_TRY(cudaMemsetAsync(v->irr[k], 0, v->P * kIrrBytes, st));
        CUDA_TRY(cudaMemsetAsync(v->depth[k], 0, v->P * kDepBytes, st));
        CUDA_TRY(cudaMemsetAsync(v->valid[k], 0, (size_t)v->P, st));
    }
    v->cur = 0;
    return SDFDDGI_OK;
}

}  // extern "C"
