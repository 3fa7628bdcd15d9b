/*
 * sdfddgi.h -- C ABI of the SDFDDGI probe-update library (CUDA, sm_103a).
 *
 * The library implements the per-frame probe update of "Signed Distance Fields
 * Dynamic Diffuse Global Illumination" (Hu et al., arXiv 2007.14394):
 *   Sec. 3.2 / Eq. 2  -- irradiance E(P, D) is sampled at probes P on a grid;
 *   Sec. 3.3 / Eq. 3  -- each probe traces low-discrepancy random rays through
 *                        the scene's signed-distance field, shades the hits
 *                        (direct light + emission + last frame's probes for
 *                        multi-bounce), and every octahedral texel gathers
 *                        E = integral of max(0, cos) L over the probe's samples,
 *                        mixed temporally with the previous frame;
 *   Sec. 3.4          -- shading points interpolate the probes.
 * The scene is a voxel signed-distance volume (the paper's primitives baked at
 * voxel centres); light visibility is an SDF shadow ray (in place of the
 * paper's reflective shadow map); depth/depth^2 moments are blended as well.
 *
 * Conventions
 *  - Every call returns SDFDDGI_OK (0) or a negative sdfddgi_status; the text
 *    of the last failure on the calling thread is sdfddgi_last_error().
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    All device work is enqueued on it and is asynchronous to the host unless
 *    the entry point says otherwise. Argument errors are reported before any
 *    work is enqueued; launch failures are reported by the call that launched.
 *  - World units throughout; parameters documented "in voxels" are multiples
 *    of the scene's voxel size.
 *  - The library owns the scene and volume storage (device memory obtained
 *    with cudaMalloc) and copies every input at call time; callers own every
 *    pointer they pass and may reuse it once the call's work on `stream` has
 *    completed.
 *  - Handles are not thread-safe: one host thread at a time per handle.
 */
#ifndef SDFDDGI_H
#define SDFDDGI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SDFDDGI_API __attribute__((visibility("default")))
#else
#define SDFDDGI_API
#endif

typedef enum {
    SDFDDGI_OK = 0,
    SDFDDGI_ERR_INVALID_ARG = -1, /* a pointer, size, enum or range is invalid   */
    SDFDDGI_ERR_OOM = -2,         /* a device or host allocation failed          */
    SDFDDGI_ERR_CUDA = -3,        /* a CUDA runtime call or launch failed        */
    SDFDDGI_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up          */
    SDFDDGI_ERR_STATE = -5,       /* the handle is not ready for this call       */
    SDFDDGI_ERR_BOUNDS = -6       /* the bounds-checked build found an index outside its buffer */
} sdfddgi_status;

typedef struct sdfddgi_scene sdfddgi_scene;   /* SDF + material volume + lights */
typedef struct sdfddgi_volume sdfddgi_volume; /* probe grid + ping-pong probe maps */
typedef struct sdfddgi_batch sdfddgi_batch;   /* volumes updated together (one graph launch) */
typedef struct sdfddgi_denoiser sdfddgi_denoiser; /* learned correction of low-ray updates */

enum { SDFDDGI_F32 = 0, SDFDDGI_F16 = 1 };                          /* SDF storage type  */
enum { SDFDDGI_LIGHT_DIRECTIONAL = 0, SDFDDGI_LIGHT_POINT = 1 };    /* light type        */
enum { SDFDDGI_PROBE_ACTIVE = 1u, SDFDDGI_PROBE_REJECT_HISTORY = 2u }; /* probe flags   */
enum { SDFDDGI_MAX_LIGHTS = 32, SDFDDGI_MAX_RAYS = 1024, SDFDDGI_MAX_STEPS = 65535 };
enum { SDFDDGI_STAGE_EVENTS = 6 };
#define SDFDDGI_MAX_SLABS 4
/* Volume flags. BLEND_BF16 -- the precision form of the gather (Eq. 3): texel weights and
 * ray values rounded to bf16, products accumulated in fp32 on the tensor cores, instead of
 * the default float32-accurate gather (three tf32 products per term). It applies when
 * rays_per_probe is a multiple of 16 (otherwise the float32 gather runs). Combine it with a
 * binary16 SDF (upload_sdf dtype SDFDDGI_F16; stepping stays float32) for the full
 * precision form. */
enum { SDFDDGI_FLAG_BLEND_BF16 = 1u };
/* RELAXED_PRIMARY, RELAXED_SHADOW -- the primary or the shadow traces take over-relaxed
 * steps (the paper's accelerated sphere tracing, Sec. 3.3, after enhanced sphere tracing): a
 * step is SDFDDGI_RELAX_OMEGA times the sampled distance; when the new sample's sphere and
 * the previous one's do not overlap (sdf + previous sdf < step), or the step left the volume
 * box, the trace returns to the previous point's plain step and stays plain for the rest of
 * the ray (the discarded sample counts toward max_steps). Hits are found with the same eps
 * test; the paths differ from plain sphere tracing, so hit distances differ within about eps.
 * Relaxation pays for rays that run far through free space (shadow rays toward the lights);
 * rays that meet a surface within a few steps pay a discarded step instead. */
enum { SDFDDGI_FLAG_RELAXED_SHADOW = 2u, SDFDDGI_FLAG_RELAXED_PRIMARY = 4u };
#define SDFDDGI_RELAX_OMEGA 1.6f
/* For tests of the failure detection only: the tensor-core gather leaves the first chunk's
 * weight copy out, so that its bounded waits run out (after about 0.2 s). The update then
 * reports SDFDDGI_ERR_TIMEOUT through sdfddgi_volume_status, and its maps are not valid. */
enum { SDFDDGI_FLAG_TEST_GATHER_STALL = 1u << 30 };

/* Octahedral map sizes (Sec. 3.3: octahedral mapping into the probe atlas):
 * irradiance 6x6 interior texels + 1-texel border = 8x8, RGBA float32 per texel
 * (A = 1 once the texel has received a ray); depth moments 14x14 + border = 16x16,
 * (mean distance, mean squared distance) float32 per texel. Probe-major layout:
 * irradiance [P][8][8][4], depth [P][16][16][2], row = octahedral v, column = u. */
enum { SDFDDGI_IRR_INTERIOR = 6, SDFDDGI_IRR_SIDE = 8, SDFDDGI_DEPTH_INTERIOR = 14, SDFDDGI_DEPTH_SIDE = 16 };

/* A light (Sec. 3.3 shading). DIRECTIONAL: v = unit direction toward the light,
 * rgb = irradiance on a surface facing it. POINT: v = position, rgb = radiant
 * intensity, range = distance at which its smooth window (1-(d/range)^4)^2 reaches 0. */
typedef struct {
    int32_t type;
    float v[3];
    float rgb[3];
    float range;
} sdfddgi_light;

/* Per-probe state (Sec. 3.2, probe choosing): world position and flags. A probe
 * without SDFDDGI_PROBE_ACTIVE casts no ray and keeps its maps; one with
 * SDFDDGI_PROBE_REJECT_HISTORY discards its history (no temporal mixing). */
typedef struct {
    float pos[3];
    uint32_t flags;
} sdfddgi_probe_state;

/* Probe volume description (Sec. 3.2 grid; Sec. 3.3 update parameters). */
typedef struct {
    int32_t dims[3];          /* probes along x, y, z (each >= 1); probe index = (z*dy + y)*dx + x */
    int32_t rays_per_probe;   /* R, 1..SDFDDGI_MAX_RAYS, spherical-Fibonacci set rotated per frame */
    float origin[3];          /* world position of probe (0,0,0) */
    float spacing[3];         /* world distance between neighbouring probes (each > 0) */
    int32_t max_steps;        /* sphere-trace step budget, 1..SDFDDGI_MAX_STEPS */
    int32_t depth_exponent;   /* p >= 1: depth texels weight rays by max(0, cos)^p */
    float eps;                /* hit threshold, voxels (> 0) */
    float t_max;              /* trace length limit, voxels; <= 0 selects the volume diagonal */
    float hysteresis;         /* temporal mixing weight of the old value, in [0, 1] */
    float multibounce_k;      /* gain of the last-frame probe term, in [0, 1] */
    float normal_bias;        /* shadow-ray origin offset along the normal, voxels (>= 0) */
    uint32_t seed;            /* seed of the per-frame ray rotation */
    uint32_t volume_id;       /* distinguishes rotations of volumes sharing a seed */
    uint32_t flags;           /* 0, or SDFDDGI_FLAG_BLEND_BF16 | SDFDDGI_FLAG_RELAXED_SHADOW |
                                 SDFDDGI_FLAG_RELAXED_PRIMARY (SDFDDGI_FLAG_TEST_GATHER_STALL: tests) */
} sdfddgi_volume_desc;

/* Per-ray record of one update (32 bytes), written only when requested:
 * the primary trace's exit event (0 left the volume, 1 hit, 2 passed t_max,
 * 3 step budget spent; 255 for rays of inactive probes), its step count, the
 * hit distance (t_max for misses), the radiance carried back, which lights were
 * visible, the total steps of the shadow rays, and (scenes of primitives) the caller's
 * index + 1 of the primitive whose material the hit took (0 otherwise). */
typedef struct {
    float t;
    float L[3];
    uint32_t lit_mask;
    uint32_t shadow_steps;
    uint16_t steps;
    uint8_t event;
    uint8_t reserved0;
    uint32_t material_owner;
} sdfddgi_ray_record;

/* An analytic SDF primitive (Sec. 3.1: the scene as a set of primitives, each with its
 * type, transform and material). params:
 *  SPHERE     centre x y z, radius
 *  BOX        centre x y z, half-extents x y z (axis-aligned)
 *  CAPSULE    end a x y z, end b x y z, radius
 *  PLANE_Y    y: solid below the plane y = params[0]
 *  INV_SPHERE centre x y z, radius: solid outside the ball (a hollow room)
 * The scene's SDF is the minimum over its primitives (exact Euclidean distances), and a
 * hit takes the albedo/emission of the primitive attaining it (the lowest index on ties). */
enum { SDFDDGI_PRIM_SPHERE = 0, SDFDDGI_PRIM_BOX = 1, SDFDDGI_PRIM_CAPSULE = 2, SDFDDGI_PRIM_PLANE_Y = 3,
       SDFDDGI_PRIM_INV_SPHERE = 4 };
typedef struct {
    int32_t type;
    float params[7];
    float albedo[3];
    float emission[3];
    float pad[2];
} sdfddgi_primitive;  /* 64 bytes */

/* Text of the last failure on this thread ("" if none). Never NULL. */
SDFDDGI_API const char* sdfddgi_last_error(void);

/* ---- scene (Sec. 3.1: the scene's SDF representation) ------------------- */

/* Creates an empty scene on the current CUDA device. *out receives the handle. */
SDFDDGI_API int sdfddgi_create_scene(sdfddgi_scene** out);
SDFDDGI_API void sdfddgi_destroy_scene(sdfddgi_scene* s);

/* Copies a signed-distance volume (and optionally its material volume) into the
 * scene, replacing any previous one. Voxel (x,y,z) holds the signed distance
 * (world units; negative inside geometry) at world point
 * origin + (x+1/2, y+1/2, z+1/2) * voxel_size; layout [z][y][x], x fastest.
 * dtype SDFDDGI_F32 (float) or SDFDDGI_F16 (IEEE binary16). dims each >= 2.
 * material: NULL (albedo 0, emission 0) or [z][y][x][8] binary16 values
 * (albedo r,g,b, unused, emission r,g,b, unused), sampled trilinearly.
 * is_device_ptr: 1 if sdf/material are device pointers, 0 for host memory.
 * Distances are not checked for being finite. An update stays inside its buffers
 * regardless: a trace meeting NaN ends as leaving the volume, +inf passes the limit,
 * -inf is a hit, and a hit whose gradient is not finite takes the reversed ray direction
 * as its normal.
 * Synchronous with respect to the host for host inputs. */
SDFDDGI_API int sdfddgi_upload_sdf(sdfddgi_scene* s, const void* sdf, const int32_t dims[3], float voxel_size,
                                   const float origin[3], int32_t dtype, const void* material,
                                   int32_t is_device_ptr, void* stream);

/* Makes the scene a union of analytic primitives (the paper's representation, Sec. 3.1)
 * instead of a voxel volume. The library groups the bounded primitives into clusters of
 * `cluster_size` by the Morton order of their centres, each with a bounding box; an SDF
 * query takes the unbounded primitives (planes, hollow balls), then visits only the
 * clusters whose box is no farther than the best distance so far (or contains the point,
 * once it is inside a primitive), and a sphere trace
 * starts each query from twice its last distance (the paper's culling, exact: the result
 * is the minimum over all primitives). cluster_size 0 puts all primitives in one cluster
 * (a plain loop, the paper's baseline).
 *  prims, n      -- host array of n >= 1 primitives (copied; the index is the position).
 *  lo, hi        -- world box that bounds every trace (rays leaving it are misses).
 *  unit          -- world length of one "voxel" for the voxel-unit parameters (eps, t_max,
 *                   normal bias, relocation clearances) and the normal's difference step.
 * Replaces any SDF; bumps the scene version (batches rebuild their graphs). */
SDFDDGI_API int sdfddgi_upload_primitives(sdfddgi_scene* s, const sdfddgi_primitive* prims, int32_t n,
                                          const float lo[3], const float hi[3], float unit, int32_t cluster_size);

/* Replaces the scene's lights (host array of n, 0..SDFDDGI_MAX_LIGHTS) and the
 * radiance of rays that leave the scene (sky_rgb, host, may be NULL for black). */
SDFDDGI_API int sdfddgi_set_lights(sdfddgi_scene* s, const sdfddgi_light* lights, int32_t n,
                                   const float sky_rgb[3]);

/* ---- probe volume (Sec. 3.2 probe grid) -------------------------------- */

/* Creates a probe volume over scene s (which must outlive it) with zeroed maps
 * and no history. The scene's SDF may be replaced later; the volume uses
 * whatever the scene holds at each update. */
SDFDDGI_API int sdfddgi_create_volume(const sdfddgi_volume_desc* desc, sdfddgi_scene* s, sdfddgi_volume** out);
SDFDDGI_API void sdfddgi_destroy_volume(sdfddgi_volume* v);

/* Number of probes of the volume. */
SDFDDGI_API int sdfddgi_volume_probe_count(const sdfddgi_volume* v, int64_t* n_probes);

/* The frame's ray rotation (row-major float 3x3) as update_probes derives it
 * when given no rotation: three uniforms from splitmix64 (Steele, Lea, Flood
 * 2014) started at seed*0x9E3779B97F4A7C15 + frame*0xBF58476D1CE4E5B9 +
 * volume_id*0x94D049BB133111EB, each (z >> 11) * 2^-53, mapped to a unit
 * quaternion by Shoemake's uniform random rotation (Graphics Gems III). */
SDFDDGI_API int sdfddgi_frame_rotation(uint32_t seed, uint32_t frame, uint32_t volume_id, float out[9]);

/* One probe update (Sec. 3.3, Eq. 3) on `stream`: for every active probe, R
 * rays d_i = Rot * sf(i, R) (spherical Fibonacci: z = 1-(2i+1)/R, azimuth
 * 2*pi*((i*2654435769) mod 2^32)/2^32) are sphere-traced through the SDF
 * from the probe; hits are shaded (emission + albedo/pi * sum of visible
 * lights' irradiance * cos + k * albedo * last frame's interpolated
 * irradiance); each interior octahedral texel of direction u takes
 * sum_i w_i v_i / sum_i w_i with w_i = max(0, u.d_i) (irradiance) or
 * max(0, u.d_i)^p (distance, distance^2; misses count as t_max), mixed as
 * h*old + (1-h)*new (h = 0 without history); then the borders are filled.
 *  frame     -- selects the rotation when `rotation` is NULL.
 *  rotation  -- NULL or host float[9] (row-major) rotation to use instead.
 *  states    -- NULL (every probe active at its grid position) or P states,
 *               host (states_on_device = 0) or device (1) memory.
 *  records   -- NULL or a device array of P*R records ([probe][ray]).
 * The maps of the previous update become the "previous" input (ping-pong). */
SDFDDGI_API int sdfddgi_update_probes(sdfddgi_volume* v, uint32_t frame, const float* rotation,
                                      const sdfddgi_probe_state* states, int32_t states_on_device,
                                      sdfddgi_ray_record* records, void* stream);

/* Stage timing (a profiling aid; the paper times its stages too, Table 1). With
 * n = SDFDDGI_STAGE_EVENTS caller-owned CUDA events (cudaEvent_t as void*), every later
 * update_probes records them on its stream: [0] at the start, [1] after the per-frame
 * texel weights, [2] after the primary traces, [3] after hit preparation, [4] after the
 * shadow traces, [5] after the gather (Eq. 3) and border fixup. n = 0 stops recording.
 * The events must outlive their use; the caller reads them with cudaEventElapsedTime.
 * While stage events are set, updates run serially (one slab, see sdfddgi_set_slabs). */
SDFDDGI_API int sdfddgi_set_stage_events(sdfddgi_volume* v, void* const* events, int32_t n);

/* Slab branches (a scheduling choice; the results are the same bit for bit). An update can
 * run its probes as `slabs` z-slabs of the probe grid (slab c: z-layers c*nz/slabs up to
 * (c+1)*nz/slabs), each slab's traces, shading, gather and fixup a chain of its own: slab 0,
 * 2 on the caller's stream, slab 1, 3 on a second stream owned by the volume, forked from
 * and joined back into the caller's stream (so the update stays one stream-ordered unit,
 * also under graph capture). The pools of a stage end with a few long rays that keep few
 * lanes busy; the other slab's kernels fill the SMs meanwhile. The ray directions are
 * computed once, before the fork; the texel weights, which only the gathers read, on a
 * stream of their own beside the traces. Each slab has its own pool counters and part of the
 * shadow-task list; the multi-bounce lookup still reads the whole volume's last maps.
 *  slabs -- 0: automatic (2 when P*R >= 2^19 rays, else 1), 1: serial, up to
 *           SDFDDGI_MAX_SLABS (at most nz slabs are used).
 * Returns SDFDDGI_ERR_INVALID_ARG outside [0, SDFDDGI_MAX_SLABS]. */
SDFDDGI_API int sdfddgi_set_slabs(sdfddgi_volume* v, int32_t slabs);
/* The number of slabs the next update_probes of v runs as (1 while stage events are set). */
SDFDDGI_API int sdfddgi_volume_slabs(const sdfddgi_volume* v, int32_t* slabs);

/* Probe relocation (Sec. 3.2, the procedure UpdateProbePos): the paper moves a probe
 * that lies too near a surface (SDF below threshold1) by gradient descent on the SDF,
 * and rejects its history when it then lies farther than threshold2 from last frame's
 * position. The paper does not specify the descent. This library takes Gauss-Newton
 * steps toward the level set sdf = clearance:
 *     p <- p + (c - sdf(p)) g / |g|^2,
 * where g is the gradient of the trilinear SDF by central differences at +-h/2. After
 * each step every coordinate is clamped to within max_offset * spacing of the grid
 * position. The steps stop at sdf >= c, at g = 0, or after max_iterations. A probe
 * ends ACTIVE iff its final SDF exceeds min_clearance, and gets REJECT_HISTORY iff
 * |p - last| > reject_distance. */
typedef struct {
    float clearance;         /* threshold1, voxels; <= 0: no probe moves */
    float reject_distance;   /* threshold2, world units; <= 0: history is never rejected */
    float max_offset;        /* per-axis limit of the move, fraction of the probe spacing, [0, 0.5] */
    float min_clearance;     /* voxels, >= 0 */
    int32_t max_iterations;  /* 0..64 */
} sdfddgi_relocation;

/* Writes the P probe states of v's grid to `out` (device). `last`: NULL (last frame's
 * positions = the grid positions) or P device states of the last frame; out may equal
 * last. The states feed sdfddgi_update_probes (states_on_device = 1). */
SDFDDGI_API int sdfddgi_relocate_probes(const sdfddgi_volume* v, const sdfddgi_relocation* r,
                                        const sdfddgi_probe_state* last, sdfddgi_probe_state* out, void* stream);

/* Interpolated normalised irradiance (Sec. 3.4 probe interpolation, without the
 * per-pixel SDF visibility test) at n world points with unit normals: trilinear
 * over the 8 probes of the grid cell containing the point (clamped to the grid),
 * each weighted by its trilinear weight times "has history", each contributing
 * the bilinear value of its irradiance map at the normal's octahedral
 * coordinates; weights renormalised, 0 where all are 0.
 * points, normals: device float[n][3]; out_rgb: device float[n][3]; n >= 0. */
SDFDDGI_API int sdfddgi_sample_irradiance(const sdfddgi_volume* v, const float* points, const float* normals,
                                          int64_t n, float* out_rgb, void* stream);

/* The paper's per-pixel interpolation with probe visibility (Sec. 3.4): as
 * sdfddgi_sample_irradiance, with each probe's weight also multiplied by its visibility
 * from the point, and no cosine or other extra weight. The paper tests visibility with
 * an SDF shadow trace and cites SDF soft shadows; the rule here: march from
 * x + normal_bias * n toward the probe by sphere tracing (the volume's eps and
 * max_steps); vis = min over the march (t > 0) of softness * sdf / t, 0 on a hit, clamped
 * to [0, 1]. The paper's screen-space parts (checkerboard depth, pixel selection, 4x4
 * de-duplication) need a frame buffer and are not part of this call.
 *  softness -- > 0; large values approach the binary test.
 *  states   -- NULL (probes at their grid positions) or P device states (positions used).
 *  points, normals, out_rgb -- device float[n][3]. */
SDFDDGI_API int sdfddgi_sample_irradiance_visible(const sdfddgi_volume* v, const float* points, const float* normals,
                                                  int64_t n, float softness, const sdfddgi_probe_state* states,
                                                  float* out_rgb, void* stream);

/* Irradiance from a cascade of probe volumes (Sec. 3.5: nested volumes of falling density,
 * blended across each volume's border with mean value coordinates instead of trilinear
 * weights, and no visibility test in the farthest one). volumes[0..n-1] run from the finest
 * to the coarsest (1 <= n <= 8; a host array of handles). For each point: k = the first
 * volume whose probe box (grid origin to origin + (dims - 1) * spacing, closed) holds it,
 * else n - 1; E = w E_k + (1 - w) E_{k+1}, w = 1 for k = n - 1. E_i is
 * sdfddgi_sample_irradiance's rule on volume i when softness = 0 or i = n - 1, else
 * sdfddgi_sample_irradiance_visible's rule (Sec. 3.4) with this softness, volume i's scene
 * and states[i]. The weight w is the sum of the mean value coordinates of the 8 corners of
 * volume k's probe box shrunk by one spacing (the inner box) over the closed shell between
 * the two boxes: 1 on and inside the inner box, 0 on the probe box's faces, smooth in
 * between; w = 1 everywhere when an axis of volume k has fewer than 4 probes (no inner box
 * of positive volume).
 *  points, normals, out_rgb -- device float[n_pts][3];
 *  softness -- 0 (no visibility test) or > 0 (finite);
 *  states -- NULL or a host array of n pointers, each NULL (probes at their grid positions)
 *            or that volume's P device probe states (positions used; only with softness > 0);
 *  out_level -- NULL or device int32[n_pts]: k;  out_weight -- NULL or device float[n_pts]: w.
 * Errors: INVALID_ARG for a NULL handle or array, n outside [1, 8], n_pts outside [0, 2^38]
 * or a negative or non-finite softness; STATE when softness > 0 and the scene of a volume
 * but the last holds no SDF; CUDA when the launch fails. Reads the volumes' current maps on
 * `stream`. */
SDFDDGI_API int sdfddgi_sample_irradiance_cascade(const sdfddgi_volume* const* volumes, int32_t n,
                                                  const float* points, const float* normals, int64_t n_pts,
                                                  float softness, const sdfddgi_probe_state* const* states,
                                                  float* out_rgb, int32_t* out_level, float* out_weight,
                                                  void* stream);

/* Device pointers to the current (latest) maps: irradiance [P][8][8][4] float,
 * depth [P][16][16][2] float, valid [P] uint8 (1 = probe has history). They stay
 * valid until the next update_probes / write_state / destroy. Any may be NULL. */
SDFDDGI_API int sdfddgi_get_maps(const sdfddgi_volume* v, const float** irr, const float** depth,
                                 const uint8_t** valid);

/* Checkpoint: copy the current maps out (read) or in (write). Arrays as in
 * get_maps; host (on_device = 0) or device (1) memory. write_state makes the
 * written maps the history of the next update. Host copies are synchronous. */
SDFDDGI_API int sdfddgi_read_state(const sdfddgi_volume* v, float* irr, float* depth, uint8_t* valid,
                                   int32_t on_device, void* stream);

/* Asynchronous read of the current maps, for a pipeline that reads frame f's maps while
 * frame f+1 updates: the copies run on a stream owned by the volume, ordered after
 * everything enqueued on `stream` so far (the update that wrote the maps), and return at
 * once. The maps are double-buffered: frame f+1 only reads the buffer being copied, and the
 * library makes the first later call that overwrites it (update_probes two frames on,
 * write_state, reset, a batch update or autotune) wait for the copy, on that call's stream.
 *  irr, depth, valid -- as for read_state (any may be NULL), host or device memory; host
 *                       memory must be page-locked for the copy to overlap device work.
 *  stream            -- the stream the volume's updates are enqueued on.
 *  done_event        -- NULL or a caller's cudaEvent_t (as void*), recorded after the
 *                       copies: synchronize on it before using the arrays.
 * Errors: INVALID_ARG for a NULL volume; CUDA when a copy or event call fails. */
SDFDDGI_API int sdfddgi_read_state_async(sdfddgi_volume* v, float* irr, float* depth, uint8_t* valid, void* stream,
                                         void* done_event);
SDFDDGI_API int sdfddgi_write_state(sdfddgi_volume* v, const float* irr, const float* depth,
                                    const uint8_t* valid, int32_t on_device, void* stream);

/* Device-side failures recorded by this volume's updates since the last call, in *flags
 * (may be NULL): bit 0 -- the shadow-task list overflowed and shadow rays were dropped (the
 * library sizes the list so that this cannot happen); bit 1 -- a bounded wait of the
 * tensor-core gather gave up: that update's maps are not valid, and later updates skip
 * the tensor-core gather (leaving their maps invalid too) until this call clears the bit;
 * bit 2 -- only in the bounds-checked build of the library (compiled with SDFDDGI_CHECKED,
 * libsdfddgi_checked.so): an update's kernel met an index outside its buffer (an SDF or
 * material sample, the multi-bounce map lookup, a per-ray array reached through a task) and
 * used element 0 instead; the maps are not valid.
 * Waits for the device, clears the bits, returns SDFDDGI_ERR_TIMEOUT if bit 1 was set, else
 * SDFDDGI_ERR_BOUNDS if bit 2 was set. */
SDFDDGI_API int sdfddgi_volume_status(sdfddgi_volume* v, uint32_t* flags);

/* Clears every map and the history (as at creation). */
SDFDDGI_API int sdfddgi_reset(sdfddgi_volume* v, void* stream);

/* Validation: how far the current irradiance maps are from a known value, reduced on the
 * device in FP64 (the library's only FP64 device arithmetic; no update step uses it). Eq. 3
 * (Sec. 3.3) is self-normalised, so a scene in which every ray brings radiance L (the white
 * furnace: a sky of L and no geometry, or surfaces of emission L and albedo 0) gives L on
 * every interior texel, and a closed room of emission Le and albedo rho lit only through the
 * multi-bounce term (k = 1, hysteresis h) gives s_n = S + (Le - S) r^n after update n (frame
 * 0 first), with S = Le / (1 - rho) and r = h + (1 - h) rho, for any ray set and rotation.
 *  states  -- NULL (every probe) or DEVICE memory, P entries as for update_probes: only the
 *             interior texels (6 x 6) of probes with SDFDDGI_PROBE_ACTIVE are counted. A host
 *             pointer is rejected (INVALID_ARG).
 *  ref_rgb -- host, the expected value per channel, finite and > 0.
 *  out     -- host, 11 doubles: [0] texels counted; [1..3] their mean per channel;
 *             [4..6] max |E - ref| / ref per channel; [7..9] root mean square of
 *             (E - ref) / ref per channel; [10] texels with a non-finite channel (left out of
 *             [0..9]). Zeroed first; the sums are formed in a fixed order, so equal maps give
 *             equal results.
 * Enqueued on `stream` after the work already there (the update that wrote the maps);
 * allocates its partial sums with cudaMallocAsync on that stream and synchronises it.
 * Errors: INVALID_ARG for a NULL volume/ref_rgb/out, a reference <= 0 or not finite, host
 * states; CUDA when a device call fails. */
SDFDDGI_API int sdfddgi_irradiance_deviation(const sdfddgi_volume* v, const sdfddgi_probe_state* states,
                                             const float ref_rgb[3], double out[11], void* stream);

/* ---- several volumes in one launch ------------------------------------- */

/* Sec. 3.5 (cascade volume) covers a large scene with several probe volumes of
 * different density -- dense near the camera, sparse far away -- all updated every
 * frame. A batch updates up to 8 volumes of one scene together: each frame is one
 * CUDA graph launch, in one of two forms (sdfddgi_batch_set_form):
 *  branches -- one branch of stage kernels per volume, so the volumes' stages overlap on
 *              the GPU;
 *  merged   -- one launch per stage covering every volume: the persistent trace kernels
 *              take (volume, task) work items from one pool over all the volumes' rays,
 *              the other stages lay the volumes' thread blocks one after another.
 * Each volume computes exactly what sdfddgi_update_probes would compute for it with the
 * same launch shapes (schedule), in either form; the results do not depend on the
 * schedule beyond the rounding order of the gather.
 *  volumes -- n distinct volumes of the same scene (not owned; they must outlive the
 *             batch and must not be updated by other calls while the batch is in use).
 *  states  -- NULL, or n pointers each NULL (grid positions) or P_i DEVICE states that
 *             the batch reads at every update (the caller may rewrite their contents
 *             between updates, not the pointers).
 *  n       -- 1..8.
 * Errors: SDFDDGI_ERR_INVALID_ARG (NULL, n out of range, a repeated volume, volumes of
 * different scenes), SDFDDGI_ERR_OOM / SDFDDGI_ERR_CUDA (stream, event or buffer). */
SDFDDGI_API int sdfddgi_create_batch(sdfddgi_volume* const* volumes, const sdfddgi_probe_state* const* states,
                                     int32_t n, sdfddgi_batch** out);
SDFDDGI_API void sdfddgi_destroy_batch(sdfddgi_batch* b);

/* One frame of every volume in the batch, enqueued on `stream` (any stream; NULL is the
 * legacy default stream). rotation: NULL (each volume's own sdfddgi_frame_rotation of
 * `frame`) or host float[9*n], volume i's row-major rotation at [9*i]. The graph is built
 * on first use and rebuilt after the scene changes (upload_sdf / set_lights) or a schedule
 * changes. Successive calls for one batch must be ordered on the GPU (the same stream,
 * or streams the caller orders), and not made from two host threads at once. */
SDFDDGI_API int sdfddgi_update_batch(sdfddgi_batch* b, uint32_t frame, const float* rotation, void* stream);

/* Chooses each volume's schedule by timing `repeats` real updates (plus one warm-up) of
 * each candidate on `stream`: trace-pool batch (16, 32, 64 tasks per warp claim, or, for
 * more than 64 rays per probe, a warp per probe: all of a probe's rays per claim), resident
 * CTAs per SM of the trace kernels (4 or the occupancy limit), gather (tensor cores when
 * rays_per_probe is a multiple of 16, or SIMT), the traces' SDF-index arithmetic (a
 * 32-bit row or 64-bit; the same addresses), and for plain voxel primary traces one or two
 * trace steps between a warp's votes (the same results). The trials write only each volume's
 * spare ping-pong buffer, so the maps and history are unchanged. Then, when the volumes
 * allow the merged form, it times `repeats` whole frames in each form and keeps the faster
 * one for SDFDDGI_BATCH_FORM_AUTO (sdfddgi_batch_form reports both times). Synchronises
 * `stream`. repeats: 1..64. */
SDFDDGI_API int sdfddgi_batch_autotune(sdfddgi_batch* b, int32_t repeats, void* stream);

/* Volume i's schedule: out[0] pool batch (tasks per warp claim; 0 = the default), out[1] CTAs
 * per SM (0 = occupancy limit),
 * out[2] gather (0 automatic, 1 tensor cores, 2 SIMT), out[3] the traces' SDF-index
 * arithmetic (0 automatic: the 32-bit row; 1 a 32-bit row, 2 64-bit; the
 * same addresses, a speed choice), out[4] trace steps between a warp's votes in the primary
 * pool of a plain voxel trace (0 automatic: 2; 1 or 2; the same results); tuned_ms
 * (nullable) receives the autotuner's mean update time of that schedule (0 before tuning). */
SDFDDGI_API int sdfddgi_batch_schedule(const sdfddgi_batch* b, int32_t i, int32_t out[5], float* tuned_ms);

/* The form of a batch's frames. AUTO (the default): the autotuner's choice (it times whole
 * frames in both forms after choosing the volumes' schedules), branches before tuning.
 * MERGED needs volumes that share the hit threshold, the step budget, the relaxation of
 * their traces, the depth exponent and the gather precision, a voxel SDF, and the
 * tensor-core gather for every volume (rays per probe a multiple of 16); its pools span every
 * volume and take the default launch shapes (not the volumes' tuned schedules), and a bounds
 * failure in a merged trace is reported by the first volume's status. */
#define SDFDDGI_BATCH_FORM_AUTO 0
#define SDFDDGI_BATCH_FORM_BRANCHES 1
#define SDFDDGI_BATCH_FORM_MERGED 2
/* Errors: SDFDDGI_ERR_INVALID_ARG (NULL, form out of range, MERGED for volumes that do not
 * allow it -- sdfddgi_last_error says why). */
SDFDDGI_API int sdfddgi_batch_set_form(sdfddgi_batch* b, int32_t form);
/* The form the next frame runs in (BRANCHES or MERGED), and (ms, nullable) the autotuner's
 * mean frame times of the two forms (0 where not timed). */
SDFDDGI_API int sdfddgi_batch_form(const sdfddgi_batch* b, int32_t* form, float ms[2]);

/* ---- the learned form: a denoiser of low-ray-count updates -------------- */

/* The paper has no learned part. A 32-ray update is noisy, and this network corrects it
 * toward the converged irradiance. It reads a probe's octahedral maps and those of its 6
 * grid neighbours. Input: 35 channels on the 8x8 bordered grid of the irradiance map.
 * The first 21 are the irradiance rgb of the probe and of its -x, +x, -y, +y, -z, +z
 * neighbours. The other 14 are their depth moments (mean / s, mean square / s^2), each
 * averaged over 2x2 texels of the 16x16 depth map, with s = depth_scale. A neighbour
 * outside its grid, or one with valid = 0, is replaced by the probe itself.
 * Network: three 3x3 convolutions 35 -> 64 -> 48 -> 3 over the 6x6 interior, with the
 * octahedral border fixup (the mirror rule of the maps' borders, Sec. 3.3) as padding
 * and ReLU between them. Output: irradiance = max(0, own interior irradiance +
 * residual), then the border fixup. The alpha channel and inactive probes pass through.
 * Loss: mean squared error over the interior rgb of active probes. Training: Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).
 * Parameters: SDFDDGI_DENOISER_PARAMS floats, in order w1 [9][35][64], b1 [64],
 * w2 [9][64][48], b2 [48], w3 [9][48][3], b3 [3], weight [tap][in][out] with tap =
 * (dy+1)*3 + (dx+1) reading the input at (row+dy, column+dx). */
enum { SDFDDGI_DENOISER_PARAMS = 49219 };

/* Arithmetic of a denoiser call.
 *  TENSOR     -- inference only: bf16 weights and layer inputs on the tensor cores, fp32
 *                accumulation (the deployed form).
 *  SIMT_BF16  -- the same rounding (weights and each layer's input to bf16) with fp32
 *                CUDA-core arithmetic; the training mode.
 *  SIMT_FP32  -- fp32 throughout (for gradient checks). */
enum { SDFDDGI_DENOISE_TENSOR = 0, SDFDDGI_DENOISE_SIMT_BF16 = 1, SDFDDGI_DENOISE_SIMT_FP32 = 2 };

/* A batch of probe grids and their maps, all in DEVICE memory, as the update leaves them.
 * P = n_grids * dims[0]*dims[1]*dims[2] probes; grid g holds probes [g*Pg, (g+1)*Pg), x
 * fastest, and a probe's neighbours are looked up within its own grid. */
typedef struct {
    int32_t dims[3];
    int32_t n_grids;
    const float* irr;                   /* [P][8][8][4] */
    const float* depth;                 /* [P][16][16][2] */
    const uint8_t* valid;               /* [P] 1 = the probe has history */
    const sdfddgi_probe_state* states;  /* [P] or NULL (all active); flags bit 0 = active */
} sdfddgi_probe_maps;

/* params: host float[SDFDDGI_DENOISER_PARAMS] (copied); depth_scale > 0 (world units;
 * e.g. the probe spacing). The Adam state starts at zero. */
SDFDDGI_API int sdfddgi_create_denoiser(const float* params, float depth_scale, sdfddgi_denoiser** out);
SDFDDGI_API void sdfddgi_destroy_denoiser(sdfddgi_denoiser* d);

/* Copies the parameters out to `read` and/or in from `write` (host arrays, either NULL).
 * Writing resets the Adam state. Synchronous. */
SDFDDGI_API int sdfddgi_denoiser_params(sdfddgi_denoiser* d, float* read, const float* write);

/* out_irr: device [P][8][8][4], the corrected maps (must not alias maps->irr). mode: one
 * of SDFDDGI_DENOISE_*. The work space grows on demand (device allocation). */
SDFDDGI_API int sdfddgi_denoise(sdfddgi_denoiser* d, const sdfddgi_probe_maps* maps, float* out_irr, int32_t mode,
                                void* stream);

/* Corrects volume v's current irradiance maps in place (its grid as one grid; states as
 * for sdfddgi_update_probes with states_on_device = 1, or NULL). */
SDFDDGI_API int sdfddgi_denoise_volume(sdfddgi_denoiser* d, sdfddgi_volume* v, const sdfddgi_probe_state* states,
                                       int32_t mode, void* stream);

/* Failures of the tensor-core inference since the last call, as sdfddgi_volume_status:
 * bit 1 -- a bounded wait gave up (those outputs are not valid, and later TENSOR calls do
 * no work until this call clears the bit). Waits for the device; SDFDDGI_ERR_TIMEOUT if set. */
SDFDDGI_API int sdfddgi_denoiser_status(sdfddgi_denoiser* d, uint32_t* flags);

/* Forward and backward pass: the loss against target_irr (device [P][8][8][4], interior rgb
 * of active probes) into *loss and its gradient in the parameters into grad (both
 * device: float[1] and float[SDFDDGI_DENOISER_PARAMS], overwritten). mode: SIMT_BF16 or
 * SIMT_FP32 (the gradient is straight-through for the bf16 rounding). */
SDFDDGI_API int sdfddgi_denoiser_gradients(sdfddgi_denoiser* d, const sdfddgi_probe_maps* maps,
                                           const float* target_irr, int32_t mode, float* grad, float* loss,
                                           void* stream);

/* One Adam step with the device gradient grad and learning rate lr. */
SDFDDGI_API int sdfddgi_denoiser_adam(sdfddgi_denoiser* d, const float* grad, float lr, void* stream);

/* gradients + adam with the denoiser's own gradient buffer; loss: device float[1] or NULL. */
SDFDDGI_API int sdfddgi_denoiser_train_step(sdfddgi_denoiser* d, const sdfddgi_probe_maps* maps,
                                            const float* target_irr, int32_t mode, float lr, float* loss,
                                            void* stream);

/* ---- the update without device allocation ------------------------------ */

/* The paper has no counterpart to this entry point; it exists for callers that may not
 * allocate device memory while they run -- an engine that reserves all GPU memory at
 * start-up and sub-allocates its own pools, a plug-in inside another framework's memory
 * manager, or a real-time loop where a cudaMalloc could stall the frame. It runs the same
 * kernels as sdfddgi_update_probes (including the tensor-core gather when R is a multiple
 * of 16) with the stages one after another on `stream`, never as slab branches; the maps
 * equal those of sdfddgi_update_probes bit for bit. It takes every input and output from
 * the caller and allocates nothing: no cudaMalloc, no cudaFree, no allocating library call.
 * The update's scratch (a copy of the SDF in the kernels' layout, per-ray buffers, the
 * shadow-task list, texel weights and their tensor-core image, counters) lives in one
 * fixed 32 MiB array in device memory that every GPU loading this library holds until
 * the process exits. An update needs, each part rounded up to 256 bytes: 16 bytes (8 at
 * binary16) per voxel of the SDF grown by one voxel on every side, (nx+2)(ny+2)(nz+2) with
 * nz+2 rounded up to even, 68 + 20*max(n_lights,1) bytes per
 * probe ray (P*R), 944*R + 928 bytes of texel weights and 32768*ceil(R/16) bytes of their
 * tensor-core image -- e.g. a 64^3 float32 SDF with 512 probes x 64 rays and 1 light
 * takes about 7.3 MiB. An update that does not fit in 32 MiB is rejected with
 * SDFDDGI_ERR_INVALID_ARG before any device work, and sdfddgi_last_error() states the
 * bytes needed and available.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) and makes the kernels' one-time set-up (occupancy and
 *    shared-memory limits); make that first call before capturing any stream.
 *  - Every call on a device shares the one array and leaves its contents behind (the
 *    parts that must start at zero are cleared by each call): calls whose work overlaps
 *    on the GPU (different streams, or different host threads) race; serialise them.
 * Arguments:
 *  desc                        -- the probe volume, as for sdfddgi_create_volume; of the
 *                                 flags only SDFDDGI_FLAG_BLEND_BF16 and the two RELAXED
 *                                 flags are accepted (others: SDFDDGI_ERR_INVALID_ARG).
 *  sdf, dims, voxel_size, origin, dtype, material
 *                              -- the scene, as for sdfddgi_upload_sdf, in DEVICE memory.
 *  lights, n_lights, sky_rgb   -- as for sdfddgi_set_lights (host memory; sky may be NULL).
 *  frame, rotation             -- as for sdfddgi_update_probes (rotation: host, nullable,
 *                                 finite).
 *  states                      -- NULL (grid positions, all active) or P device states.
 *  prev_irr/prev_depth/prev_valid -- the previous maps (device; zeros for no history).
 *  cur_irr/cur_depth/cur_valid -- receive the new maps (device). A cur_* range that shares
 *                                 a byte with a prev_* range or with another cur_* range is
 *                                 rejected with SDFDDGI_ERR_INVALID_ARG.
 *  records                     -- NULL or P*R device records, as for sdfddgi_update_probes.
 * The library cannot see the sizes of the caller's buffers: each must hold what the layouts
 * of sdfddgi_get_maps give for P = prod(desc->dims) probes (and P*R records), and the SDF
 * and material prod(dims) voxels; a smaller buffer is read or written out of bounds.
 * Work is enqueued on `stream`. */
SDFDDGI_API int sdfddgi_update_probes_noalloc(
    const sdfddgi_volume_desc* desc, const void* sdf, const int32_t dims[3], float voxel_size,
    const float origin[3], int32_t dtype, const void* material, const sdfddgi_light* lights, int32_t n_lights,
    const float sky_rgb[3], uint32_t frame, const float* rotation, const sdfddgi_probe_state* states,
    const float* prev_irr, const float* prev_depth, const uint8_t* prev_valid, float* cur_irr, float* cur_depth,
    uint8_t* cur_valid, sdfddgi_ray_record* records, void* stream);

/* ---- Measurement: the L2 read bandwidth, the second ceiling (beside the HBM copy rate) of
 * the gathers in the traces and the hit preparation (the measurement row of the scope,
 * "GB/s as a fraction of HBM and of the measured L2 peak").
 *  buf   -- device buffer of `bytes` bytes (16-byte aligned, a multiple of 16), small enough
 *           to stay in L2 (e.g. 32 MiB of the 126 MB); its contents are only read.
 *  reps  -- sweeps over the buffer in the timed launch, 1..1000 (one untimed sweep first).
 *  gbs   -- receives bytes * reps / time in GB/s: every SM's threads read the buffer with
 *           16-byte loads that bypass L1, timed with CUDA events on `stream`.
 * Synchronises `stream`. */
SDFDDGI_API int sdfddgi_l2_read_bandwidth(const void* buf, size_t bytes, int32_t reps, float* gbs, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SDFDDGI_H */
