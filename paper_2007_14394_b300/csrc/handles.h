// handles.h -- the library's opaque handles (scene, volume) and the helper that turns a
// volume into the parameters of one update; shared by the C ABI and the batched update.
#pragma once

#include "internal.h"

struct sdfddgi_scene {
    uint64_t version = 0;  // bumped by every upload_sdf / set_lights (captured graphs depend on it)
    int device = 0;
    void* sdf = nullptr;
    size_t sdf_bytes = 0;
    void* quads = nullptr;  // xy-quad copy of the SDF read by the trace kernels
    size_t quads_bytes = 0;
    void* material = nullptr;
    size_t material_bytes = 0;
    int dims[3] = {0, 0, 0};
    int dtype = SDFDDGI_F32;
    float h = 0.f;
    float origin[3] = {0.f, 0.f, 0.f};
    bool has_sdf = false;
    bool has_material = false;
    // a scene of analytic primitives (dtype kAnalytic) instead of a voxel volume
    sdfddgi::PrimDev* prims = nullptr;  // unbounded primitives first, then each cluster's run
    sdfddgi::ClusterDev* clusters = nullptr;
    int n_prims = 0, n_unbounded = 0, n_clusters = 0;
    sdfddgi::LightDev lights[SDFDDGI_MAX_LIGHTS] = {};
    int n_lights = 0;
    float sky[3] = {0.f, 0.f, 0.f};
};

struct sdfddgi_volume {
    sdfddgi_volume_desc desc{};
    sdfddgi_scene* scene = nullptr;
    int64_t P = 0;
    float4* irr[2] = {nullptr, nullptr};
    float2* depth[2] = {nullptr, nullptr};
    uint8_t* valid[2] = {nullptr, nullptr};
    sdfddgi_probe_state* states = nullptr;  // staging for host-side probe states
    int cur = 0;
    // per-ray scratch of the staged update (P * R entries each) and the shadow-task list
    float* ray_t = nullptr;
    uint32_t* ray_es = nullptr;
    float4* ray_n = nullptr;
    float4* ray_alb = nullptr;
    float4* ray_base = nullptr;
    uint32_t* ray_lit = nullptr;
    uint32_t* ray_ssteps = nullptr;
    uint32_t* counters = nullptr;  // kMaxSlabs slabs' kCounterWords words, kSlabCounterStride apart
    float4* tasks = nullptr;
    float* task_scale = nullptr;  // one light factor per task slot
    size_t task_capacity = 0;
    uint32_t* fin_list = nullptr;  // P * R: the hits the finalize stage completes
    float* weights = nullptr;  // texel weights of the frame's ray set and their column sums
    void* wimage = nullptr;    // the weights as the tensor-core gather's operand image
    cudaEvent_t stage_events[SDFDDGI_STAGE_EVENTS] = {};  // caller's, recorded at stage boundaries
    bool has_stage_events = false;
    int slabs = 0;                    // slab branches per update (0 automatic)
    sdfddgi::SlabLanes lanes = {};    // the second stream and fork/join events of slab branches
    // asynchronous reads of the maps (read_state_async): they run on `copy`; read_done[b] is
    // recorded after a read of buffer b, and pending_read[b] tells that work which writes
    // buffer b must wait for it
    cudaStream_t copy = nullptr;
    cudaEvent_t read_order = nullptr;
    cudaEvent_t read_done[2] = {nullptr, nullptr};
    bool pending_read[2] = {false, false};
};

namespace sdfddgi {
// The scene's SDF as the kernels read it (voxel volume or primitives).
void scene_view(const sdfddgi_scene* s, VolumeView* v);
// Everything of one update of v that follows from the scene and the volume at the current
// ping-pong parity (rotation, probe states, records and schedule are left zero); ensures the
// shadow-task capacity. Returns an sdfddgi_status.
int volume_params(sdfddgi_volume* v, UpdateParams* p);
// Makes `stream` wait for a pending asynchronous read of map buffer `buf` before work that
// writes the buffer (a no-op when none is pending).
cudaError_t order_map_write(sdfddgi_volume* v, int buf, cudaStream_t stream);
}  // namespace sdfddgi
