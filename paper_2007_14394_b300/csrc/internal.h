// internal.h -- structures shared by the library's host code and its kernels.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sdfddgi.h"

namespace sdfddgi {

constexpr int kIrrN = SDFDDGI_IRR_INTERIOR;      // 6
constexpr int kIrrT = SDFDDGI_IRR_SIDE;          // 8
constexpr int kDepN = SDFDDGI_DEPTH_INTERIOR;    // 14
constexpr int kDepT = SDFDDGI_DEPTH_SIDE;        // 16
constexpr int kIrrTexels = kIrrN * kIrrN;        // 36 interior irradiance texels
constexpr int kDepTexels = kDepN * kDepN;        // 196 interior depth texels

enum Event : uint8_t { kLeftVolume = 0, kHit = 1, kPastLimit = 2, kExhausted = 3, kNoRay = 255 };

// One analytic primitive as the kernels read it (64 bytes): type and parameters as in
// sdfddgi_primitive, the caller's index (material ties go to the lowest), material.
struct PrimDev {
    int type;
    int index;
    float p[7];
    float albedo[3];
    float emission[3];
    float pad;
};

// A cluster of primitives: its box (inflated so that float rounding never culls a primitive
// that attains the minimum) and its run [first, first + count) of the primitive array.
struct ClusterDev {
    float lo[3];
    int first;
    float hi[3];
    int count;
};

constexpr int kAnalytic = 2;  // VolumeView::dtype of a scene made of primitives

// The scene's SDF as the kernels read it: a voxel volume (float or binary16, with its
// material volume) or, with dtype kAnalytic, a union of analytic primitives in clusters.
struct VolumeView {
    const void* quads;        // xy-quads of the same values (float4 or 4 x __half), in z-pairs with a
                              // one-voxel apron on every side: quad_index of the padded coordinates
    const uint4* material;    // 8 x binary16 per voxel (albedo rgb, -, emission rgb, -), or null
    int nx, ny, nz;
    int dtype;                // SDFDDGI_F32 / SDFDDGI_F16 / kAnalytic
    float h, inv_h;           // voxel size (analytic: the unit of voxel parameters)
    float lo[3];              // world box of the volume (bounds every trace)
    float hi[3];
    size_t n_quads;           // quads in the store (bounds of the checked build)
    uint32_t* fail;           // null, or the launch's failure word (the checked build reports there)
    int qx, qy;               // padded x and y extents of the quad store (nx + 2, ny + 2)
    float gmax[3];            // n - 1/2 per axis: the box in voxel coordinates is [-1/2, n - 1/2]
    const PrimDev* prims;     // analytic: unbounded primitives first, then each cluster's run
    const ClusterDev* clusters;
    int n_unbounded;
    int n_clusters;
};

// Launch shapes of one update; zero fields select the defaults.
struct Schedule {
    int pool_batch;      // trace tasks a warp claims per atomic, e.g. 16, 32, 64, or R (a warp per probe);
                         // 0: 64 primary, 128 shadow
    int blocks_per_sm;   // resident CTAs per SM of the persistent trace kernels (default: occupancy limit)
    int gather;          // 0 automatic (tensor cores when R % 16 == 0), 1 tensor cores, 2 SIMT
    int slabs;           // z-slabs of probes run as concurrent branches: 0 automatic, 1 (serial) .. kMaxSlabs
    int index;           // the traces' quad-index arithmetic: 0 automatic (the 32-bit row form),
                         // 1 a 32-bit z-pair row, 2 all in 64 bits (the same addresses either way)
    int refill;          // idle lanes of a trace warp before it hands out new tasks: 0 default, 1..32
    int steps;           // trace steps between a warp's votes in the primary pool of a plain voxel
                         // trace: 0 automatic (2), 1 or 2 (the same results either way)
};

constexpr int kMaxSlabs = SDFDDGI_MAX_SLABS;

struct LightDev {
    int type;
    float v[3];
    float rgb[3];
    float range;
};

struct UpdateParams {
    VolumeView vol;
    LightDev lights[SDFDDGI_MAX_LIGHTS];
    int n_lights;
    float sky[3];
    int gdims[3];
    float gorigin[3];
    float gspacing[3];
    int P;                    // probe count (of this launch: the volume, or one slab of it)
    int p_begin;              // the volume's index of probe 0 of this launch (a slab's first probe)
    int R;                    // rays per probe
    int max_steps;
    int depth_exp;
    float eps_w;              // hit threshold, world units
    float tmax_w;             // trace limit, world units
    float hyst;
    float k_bounce;
    float bias_w;             // shadow-ray offset, world units
    float rot[9];             // row-major frame rotation
    const sdfddgi_probe_state* states;  // device; null = grid positions, all active
    const float4* prev_irr;   // [P][8][8]
    const float2* prev_depth; // [P][16][16]
    const uint8_t* prev_valid;
    const float4* look_irr;   // the whole volume's previous irradiance and validity (multi-bounce
    const uint8_t* look_valid;// lookups reach any probe); null: prev_irr / prev_valid
    float4* cur_irr;
    float2* cur_depth;
    uint8_t* cur_valid;
    sdfddgi_ray_record* records;  // null or [P][R]
    // per-ray scratch of the staged update, index k = probe * R + ray
    float* ray_t;             // hit distance (t_max for misses)
    uint32_t* ray_es;         // event | steps << 8
    float4* ray_n;            // (records only) a hit with shadow tasks: its material owner (bits of x)
    float4* ray_alb;          // per finalize-list entry: albedo rgb, gated-light mask (bits of w)
    float4* ray_base;         // per finalize-list entry: emission + k * albedo * last-frame irradiance, first task (bits of w)
    uint32_t* ray_lit;        // per finalize-list entry: visible-light mask
    uint32_t* ray_ssteps;     // per finalize-list entry: shadow steps (kept only when records are asked for)
    float4* tasks;            // shadow tasks: origin xyz, bits of (finalize-list entry << 5 | light)
    float* task_scale;        // [task_capacity] each task's light factor at its hit (light_scale)
    uint32_t task_capacity;
    uint32_t* fin_list;       // [P*R] the hits with shadow tasks, for the finalize stage
    uint32_t* counters;       // kCounterWords words: pools and counts (zeroed by each launch), then at
                              // kFailWord the failure bits, sticky: 1 task overflow, 2 a tensor-core wait gave up
    float* weights;           // [R][kTexels] texel weights of the frame's ray set, [kTexels] column sums,
                              // then room for [R] float4 ray directions (weights_bytes(R) in all)
    float4* dirs;             // [R] the frame's ray directions (same for every probe), set by launch_update
    float4* ray_val;          // [P*R] radiance rgb + clamped distance per ray, set by launch_update
    void* wimage;             // null, or wimage_bytes(R): the weights as the tensor-core gather's operand
    int blend_bf16;           // 1: the tensor-core gather multiplies bf16 x bf16 (the precision form)
    int test_stall;           // 1: the tensor-core gather leaves chunk 0's weight copy out (failure tests)
    float omega_primary;      // relaxation factor of the primary traces (1: plain sphere tracing)
    float omega_shadow;       // relaxation factor of the shadow traces
    const float* rot_dev;     // null, or the frame rotation in device memory (read instead of rot)
    Schedule sched;           // launch shapes (chosen by the autotuner for batches)
};

constexpr int kTexels = kIrrTexels + kDepTexels;  // 232 gather rows: irradiance texels first

// Words of UpdateParams::counters: 0 primary pool, 1 shadow-task count, 2 shadow pool, 3 the
// finalize list's length;
// words 0..kFailWord-1 are zeroed by every launch.
constexpr int kPrimaryPool = 0, kTaskCount = 1, kShadowPool = 2, kFinCount = 3;
constexpr int kFailWord = 7;
// Bits of the failure word: 1 the shadow-task list overflowed, 2 a tensor-core wait gave up,
// 4 (checked build) an index lay outside its buffer.
constexpr uint32_t kFailTasks = 1u, kFailWait = 2u, kFailBounds = 4u;
// The bounds-checked build (compiled with SDFDDGI_CHECKED): the update's data-dependent
// accesses -- SDF and material samples, the multi-bounce map lookup, per-ray arrays reached
// through task payloads -- check their index and, outside the buffer, set kFailBounds and use
// element 0 instead, so that a bad index is reported rather than read or written.
#ifdef SDFDDGI_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif
constexpr int kCounterWords = 8;
// The slabs of one update keep their counters 256 bytes apart, so that concurrent slab
// branches' atomics do not meet in one L2 line.
constexpr int kSlabCounterStride = 64;

struct SampleParams {
    int gdims[3];
    float gorigin[3];
    float gspacing[3];
    const float4* irr;
    const uint8_t* valid;
    const float* points;
    const float* normals;
    float* out;
    int64_t n;
};

// The per-point probe visibility test of sample_irradiance_visible.
struct VisParams {
    VolumeView vol;
    float softness;
    float eps_w;       // hit threshold, world units
    float bias_w;      // start offset along the normal, world units
    int max_steps;
    const sdfddgi_probe_state* states;  // null: probes at their grid positions
};

// The streams and events with which one update forks its slab branches off `stream` and joins
// them again (owned by the volume): slab c > 0 runs on side[c - 1].
struct SlabLanes {
    cudaStream_t side[SDFDDGI_MAX_SLABS - 1];
    cudaEvent_t fork;
    cudaEvent_t join[SDFDDGI_MAX_SLABS - 1];
    cudaEvent_t weights_ready;  // the texel weights and their image, made on slab 1's stream
};

// stage_events: null, or SDFDDGI_STAGE_EVENTS events recorded on `stream` at the stage boundaries
// (the update then runs serially); lanes: null (serial), or the streams for slab branches.
cudaError_t launch_update(const UpdateParams& p, cudaStream_t stream, cudaEvent_t const* stage_events = nullptr,
                          const SlabLanes* lanes = nullptr);
// The number of slab branches launch_update runs p as (1 = serial).
int slab_count(const UpdateParams& p, bool have_lanes, bool stage_events);
// The parameters launch_update actually runs: plain traces unless relaxation was asked for,
// the multi-bounce lookup maps, the directions and value slots inside the scratch, the
// failure word.
UpdateParams prepared_params(const UpdateParams& p);

// Several volumes of one scene updated with one launch per stage, each launch covering every
// volume (the batched form's merged schedule). Per stage, the volumes' parts follow one
// another: volume v owns tasks ray_begin[v] .. ray_begin[v + 1] - 1 of the merged primary
// pool (its P*R rays, padded to a multiple of the pool batch, so that a claimed batch lies
// within one volume), CTAs prep_begin[v] .. of the hit preparation, gather_begin[v] .. of the
// gather, and blocks dir_begin[v] .. (one per ray) of the texel weights and their image. The
// shadow pool is laid out the same way from the task counts on the device. The merged pools'
// counters are volume 0's pool words, which the launch zeroes with every volume's counters.
constexpr int kMaxMerged = 8;
struct MergedParams {
    int n;
    uint32_t primary_batch, shadow_batch;  // tasks per claim of the two merged pools
    uint32_t ray_begin[kMaxMerged + 1];
    uint32_t prep_begin[kMaxMerged + 1];
    uint32_t prep_rays[kMaxMerged];  // rays per hit-preparation CTA of each volume
    uint32_t gather_begin[kMaxMerged + 1];
    uint32_t dir_begin[kMaxMerged + 1];
    UpdateParams p[kMaxMerged];  // prepared_params of each volume
};
// Whether n volumes (their launch parameters) can run as one launch per stage: one scene, the
// same hit threshold, step budget, relaxation, depth exponent and gather precision, the
// tensor-core gather for every volume, and at most kMaxMerged of them. The message says why not.
bool merged_supported(const UpdateParams* p, int n, const char** why);
// Builds m from the volumes' parameters (prepared here) and enqueues the frame on `stream`:
// the counters, the texel weights and their image, then one launch per stage.
cudaError_t launch_merged(const UpdateParams* p, int n, MergedParams* m, cudaStream_t stream);
// The merged tensor-core gather (with pack: first the volumes' weight images).
cudaError_t launch_gather_tc_merged(const MergedParams& m, cudaStream_t stream, bool pack);
cudaError_t launch_sample(const SampleParams& p, cudaStream_t stream);
cudaError_t launch_sample_visible(const SampleParams& p, const VisParams& v, cudaStream_t stream);
// Position of quad (x, y, z) in an xy-quad store of padded extents qx, qy: z-pairs,
// [z/2][y][x][z%2]. Padded coordinates: voxel (i, j, k) is quad (i + 1, j + 1, k + 1).
__host__ __device__ __forceinline__ size_t quad_index(size_t x, size_t y, size_t z, size_t qx, size_t qy) {
    return (((z >> 1) * qy + y) * qx + x) * 2 + (z & 1);
}
// Bytes of the xy-quad copy of an SDF of `dims` voxels: a one-voxel apron on every side,
// nz + 2 rounded up to even.
size_t quad_bytes(int dtype, const int dims[3]);
// The view's derived constants of the voxel-space traces (qx, qy, gmax), from nx, ny, nz.
// Padded x extent of the quad store.
inline int padded_qx(int nx) { return nx + 2; }
inline void set_trace_constants(VolumeView* v) {
    v->qx = padded_qx(v->nx);
    v->qy = v->ny + 2;
    v->n_quads = (size_t)v->qx * v->qy * (((size_t)v->nz + 3) / 2 * 2);
    v->gmax[0] = (float)v->nx - 0.5f;
    v->gmax[1] = (float)v->ny - 0.5f;
    v->gmax[2] = (float)v->nz - 0.5f;
}
inline size_t weights_bytes(int R) { return ((size_t)(R + 1) * kTexels + (size_t)R * 4) * sizeof(float); }
int report_error(int code, const char* msg);  // sets the text of sdfddgi_last_error(), returns code
// the gather of Eq. 3 on the tensor cores (R a multiple of 16 and a weight image present)
bool gather_tc_supported(const UpdateParams& p);
size_t wimage_bytes(int R);
constexpr int kGatherTcProbes = 19;  // probes per CTA of the tensor-core gather
// The tensor-core gather; with pack, first the frame's weight image (otherwise already packed
// by launch_pack_weights on a stream this one waits for).
cudaError_t launch_gather_tc(const UpdateParams& p, cudaStream_t stream, bool pack = true);
cudaError_t launch_pack_weights(const UpdateParams& p, cudaStream_t stream);
cudaError_t prepare_gather_tc();  // dynamic shared-memory limits of the tensor-core gathers
// one-time per-device set-up of the update's kernels (occupancy, shared-memory limits); the
// first update makes it otherwise, but it must not happen inside a stream capture
struct DeviceSetup;
cudaError_t prepare_update_kernels(const DeviceSetup** out = nullptr);
cudaError_t build_quads(const void* sdf, void* quads, int dtype, const int dims[3], cudaStream_t stream);

}  // namespace sdfddgi
