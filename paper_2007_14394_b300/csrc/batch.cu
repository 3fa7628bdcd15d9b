// batch.cu -- several probe volumes (e.g. the nested cascades of the paper's Sec. 3.5)
// updated together, each frame one CUDA graph launch from the host, in one of two forms:
//  branches -- one branch of stage kernels per volume, so that the volumes' stages overlap
//              on the GPU (a small volume's pool tails fill with the large volumes' work);
//  merged   -- one launch per stage covering every volume: the persistent trace kernels
//              take (volume, task) work items from one pool over all the volumes' rays, and
//              the other stages lay the volumes' CTAs one after another (MergedParams).
// The graph is captured once per ping-pong parity, form and scene version and replayed; the
// frame's rotations reach it through a small device buffer written before each replay.
//
// The autotuner picks each volume's launch shapes (trace-pool batch, resident CTAs per
// SM of the trace kernels, tensor-core or SIMT gather, index arithmetic) by timing real
// updates of that volume, then the faster form by timing whole frames; the trials write
// only the volumes' spare ping-pong buffers.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "handles.h"

using namespace sdfddgi;

namespace {

constexpr int kMaxBatch = 8;
constexpr int kGraphCache = 4;

struct CachedGraph {
    uint64_t key = 0;
    uint64_t version = 0;
    cudaGraphExec_t exec = nullptr;
};

int bfail(int code, const char* msg) { return report_error(code, msg); }

}  // namespace

struct sdfddgi_batch {
    int n = 0;
    sdfddgi_volume* vols[kMaxBatch] = {};
    const sdfddgi_probe_state* states[kMaxBatch] = {};  // device, or null (grid positions)
    Schedule sched[kMaxBatch] = {};
    float tuned_ms[kMaxBatch] = {};
    cudaStream_t side[kMaxBatch] = {};
    cudaStream_t capture = nullptr;  // graphs are captured here (capture needs a non-legacy stream)
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kMaxBatch] = {};
    float* rot_dev = nullptr;  // [n][9]
    CachedGraph cache[kGraphCache];
    int next_slot = 0;
    int form_asked = SDFDDGI_BATCH_FORM_AUTO;  // SDFDDGI_BATCH_FORM_*
    int form_tuned = 0;                        // the autotuner's choice (0 before tuning)
    float form_ms[2] = {0.f, 0.f};             // the autotuner's frame times: branches, merged
    MergedParams merged;                       // the merged launches' parameters (host copy)
};

namespace {

void drop_graphs(sdfddgi_batch* b) {
    for (auto& c : b->cache) {
        if (c.exec) cudaGraphExecDestroy(c.exec);
        c = CachedGraph();
    }
}

// The launch parameters of volume i's next frame (reads the current maps, writes the other).
int batch_params(sdfddgi_batch* b, int i, UpdateParams* p) {
    int rc = volume_params(b->vols[i], p);
    if (rc) return rc;
    p->rot_dev = b->rot_dev + 9 * i;
    p->states = b->states[i];
    p->sched = b->sched[i];
    return SDFDDGI_OK;
}

// Whether the volumes can run merged (and, when not, why).
bool merged_ok(sdfddgi_batch* b, const char** why) {
    UpdateParams p[kMaxBatch];
    for (int i = 0; i < b->n; ++i)
        if (batch_params(b, i, &p[i])) {
            if (why) *why = "a volume's parameters could not be prepared";
            return false;
        }
    return merged_supported(p, b->n, why);
}

// The form a frame runs in: the caller's, else the autotuner's, else branches.
int frame_form(const sdfddgi_batch* b) {
    if (b->form_asked != SDFDDGI_BATCH_FORM_AUTO) return b->form_asked;
    return b->form_tuned ? b->form_tuned : SDFDDGI_BATCH_FORM_BRANCHES;
}

// Records every volume's stages with one launch per stage on the capturing stream.
int record_frame_merged(sdfddgi_batch* b, cudaStream_t st) {
    UpdateParams p[kMaxBatch];
    for (int i = 0; i < b->n; ++i) {
        int rc = batch_params(b, i, &p[i]);
        if (rc) return rc;
    }
    const char* why = nullptr;
    if (!merged_supported(p, b->n, &why)) return bfail(SDFDDGI_ERR_INVALID_ARG, why);
    cudaError_t e = launch_merged(p, b->n, &b->merged, st);
    if (e != cudaSuccess) return bfail(SDFDDGI_ERR_CUDA, cudaGetErrorString(e));
    return SDFDDGI_OK;
}

// Records the stages of every volume, one forked stream each, on the capturing stream.
int record_frame(sdfddgi_batch* b, cudaStream_t st) {
    if (frame_form(b) == SDFDDGI_BATCH_FORM_MERGED) return record_frame_merged(b, st);
    cudaError_t e = cudaEventRecord(b->fork, st);
    for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
        UpdateParams p;
        int rc = batch_params(b, i, &p);
        if (rc) return rc;
        e = cudaStreamWaitEvent(b->side[i], b->fork, 0);
        if (e == cudaSuccess) e = launch_update(p, b->side[i]);
        if (e == cudaSuccess) e = cudaEventRecord(b->join[i], b->side[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->join[i], 0);
    }
    if (e != cudaSuccess) return bfail(SDFDDGI_ERR_CUDA, cudaGetErrorString(e));
    return SDFDDGI_OK;
}

uint64_t parity_key(const sdfddgi_batch* b) {
    uint64_t k = 0;
    for (int i = 0; i < b->n; ++i) k |= (uint64_t)(b->vols[i]->cur & 1) << i;
    return k | (uint64_t)frame_form(b) << 32;
}

// Every volume's frame rotations for `frame` into rot (host, [n][9]).
void frame_rotations(const sdfddgi_batch* b, uint32_t frame, float* rot) {
    for (int i = 0; i < b->n; ++i) {
        const sdfddgi_volume_desc& d = b->vols[i]->desc;
        sdfddgi_frame_rotation(d.seed, frame, d.volume_id, rot + 9 * i);
    }
}

}  // namespace

extern "C" {

SDFDDGI_API int sdfddgi_create_batch(sdfddgi_volume* const* volumes, const sdfddgi_probe_state* const* states,
                                     int32_t n, sdfddgi_batch** out) {
    if (out) *out = nullptr;
    if (!out || !volumes) return bfail(SDFDDGI_ERR_INVALID_ARG, "create_batch: NULL argument");
    if (n < 1 || n > kMaxBatch) return bfail(SDFDDGI_ERR_INVALID_ARG, "create_batch: n must be in [1, 8]");
    for (int i = 0; i < n; ++i) {
        if (!volumes[i]) return bfail(SDFDDGI_ERR_INVALID_ARG, "create_batch: a volume is NULL");
        if (volumes[i]->scene != volumes[0]->scene)
            return bfail(SDFDDGI_ERR_INVALID_ARG, "create_batch: the volumes must share one scene");
        for (int j = 0; j < i; ++j)
            if (volumes[j] == volumes[i]) return bfail(SDFDDGI_ERR_INVALID_ARG, "create_batch: a volume appears twice");
    }
    sdfddgi_batch* b = new (std::nothrow) sdfddgi_batch();
    if (!b) return bfail(SDFDDGI_ERR_OOM, "create_batch: host allocation failed");
    b->n = n;
    cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        b->vols[i] = volumes[i];
        b->states[i] = states ? states[i] : nullptr;
        e = cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->rot_dev, sizeof(float) * 9 * n);
    if (e == cudaSuccess) {  // frame 0's rotations until the first update writes its own
        float rot[kMaxBatch * 9];
        frame_rotations(b, 0, rot);
        e = cudaMemcpy(b->rot_dev, rot, sizeof(float) * 9 * n, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        sdfddgi_destroy_batch(b);
        return bfail(e == cudaErrorMemoryAllocation ? SDFDDGI_ERR_OOM : SDFDDGI_ERR_CUDA, cudaGetErrorString(e));
    }
    *out = b;
    return SDFDDGI_OK;
}

SDFDDGI_API void sdfddgi_destroy_batch(sdfddgi_batch* b) {
    if (!b) return;
    drop_graphs(b);
    for (int i = 0; i < kMaxBatch; ++i) {
        if (b->side[i]) cudaStreamDestroy(b->side[i]);
        if (b->join[i]) cudaEventDestroy(b->join[i]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->capture) cudaStreamDestroy(b->capture);
    cudaFree(b->rot_dev);
    delete b;
}

SDFDDGI_API int sdfddgi_update_batch(sdfddgi_batch* b, uint32_t frame, const float* rotations, void* stream) {
    if (!b) return bfail(SDFDDGI_ERR_INVALID_ARG, "update_batch: batch is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float rot[kMaxBatch * 9];
    if (rotations) {
        for (int k = 0; k < 9 * b->n; ++k) {
            if (!std::isfinite(rotations[k])) return bfail(SDFDDGI_ERR_INVALID_ARG, "update_batch: rotation not finite");
            rot[k] = rotations[k];
        }
    } else {
        frame_rotations(b, frame, rot);
    }
    // everything the captured work reads from the host side must be current
    UpdateParams probe;
    for (int i = 0; i < b->n; ++i) {
        int rc = volume_params(b->vols[i], &probe);  // also sizes the shadow-task lists
        if (rc) return rc;
    }
    const uint64_t key = parity_key(b), version = b->vols[0]->scene->version;
    cudaGraphExec_t exec = nullptr;
    for (auto& c : b->cache)
        if (c.exec && c.key == key && c.version == version) exec = c.exec;
    cudaError_t e;
    if (!exec) {
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return bfail(SDFDDGI_ERR_CUDA, cudaGetErrorString(e));
        int rc = record_frame(b, b->capture);
        e = cudaStreamEndCapture(b->capture, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return bfail(SDFDDGI_ERR_CUDA, cudaGetErrorString(e));
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return bfail(SDFDDGI_ERR_CUDA, cudaGetErrorString(e));
        CachedGraph& slot = b->cache[b->next_slot];
        b->next_slot = (b->next_slot + 1) % kGraphCache;
        if (slot.exec) cudaGraphExecDestroy(slot.exec);
        slot.key = key;
        slot.version = version;
        slot.exec = exec;
    }
    e = cudaMemcpyAsync(b->rot_dev, rot, sizeof(float) * 9 * b->n, cudaMemcpyHostToDevice, st);
    for (int i = 0; i < b->n && e == cudaSuccess; ++i) e = order_map_write(b->vols[i], b->vols[i]->cur ^ 1, st);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
    if (e != cudaSuccess) return bfail(SDFDDGI_ERR_CUDA, cudaGetErrorString(e));
    for (int i = 0; i < b->n; ++i) b->vols[i]->cur ^= 1;
    return SDFDDGI_OK;
}

SDFDDGI_API int sdfddgi_batch_autotune(sdfddgi_batch* b, int32_t repeats, void* stream) {
    if (!b || repeats < 1 || repeats > 64) return bfail(SDFDDGI_ERR_INVALID_ARG, "batch_autotune: invalid arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return bfail(SDFDDGI_ERR_CUDA, "batch_autotune: cudaEventCreate failed");
    int rc = SDFDDGI_OK;
    for (int i = 0; i < b->n && rc == SDFDDGI_OK; ++i) {
        sdfddgi_volume* v = b->vols[i];
        // every trial reads the current maps and writes the other buffer, which the next
        // real update overwrites: the volume's state is untouched
        if (order_map_write(v, v->cur ^ 1, st) != cudaSuccess) {
            rc = bfail(SDFDDGI_ERR_CUDA, "batch_autotune: cudaStreamWaitEvent failed");
            break;
        }
        UpdateParams probe;
        rc = volume_params(v, &probe);
        if (rc) break;
        const bool tc_ok = gather_tc_supported(probe);
        std::vector<Schedule> cand;
        // trace tasks per warp claim: 16, 32 or 64 rays, or a warp per probe (all R rays of one
        // probe per claim, where R is larger)
        const int R = probe.R;
        std::vector<int> batches = {16, 32, 64};
        if (R > 64) batches.push_back(R);
        // one or two trace steps between a warp's votes in the primary pool (plain voxel traces)
        const bool steps_choice = probe.vol.dtype != kAnalytic && !(probe.omega_primary > 1.f);
        for (int pb : batches)
            for (int bps : {0, 4})
                for (int g : {1, 2})
                    for (int ix : {1, 2})  // the traces' quad-index arithmetic (same addresses)
                        for (int stp : {2, 1}) {
                            if (g == 1 && !tc_ok) continue;
                            if (stp == 1 && !steps_choice) continue;
                            Schedule c = {};
                            c.pool_batch = pb;
                            c.blocks_per_sm = bps;
                            c.gather = g;
                            c.index = ix;
                            c.steps = stp;
                            cand.push_back(c);
                        }
        float best = 1e30f;
        Schedule best_s = {};
        for (const Schedule& sc : cand) {
            float total = 0.f;
            for (int r = 0; r <= repeats && rc == SDFDDGI_OK; ++r) {  // the first run warms up
                UpdateParams p;
                rc = volume_params(v, &p);
                if (rc) break;
                sdfddgi_frame_rotation(v->desc.seed, (uint32_t)r, v->desc.volume_id, p.rot);
                p.states = b->states[i];
                p.sched = sc;
                cudaEventRecord(e0, st);
                cudaError_t e = launch_update(p, st);
                cudaEventRecord(e1, st);
                if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                    rc = bfail(SDFDDGI_ERR_CUDA, "batch_autotune: trial update failed");
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (r > 0) total += ms;
            }
            if (rc) break;
            if (total / repeats < best) {
                best = total / repeats;
                best_s = sc;
            }
        }
        if (rc == SDFDDGI_OK) {
            b->sched[i] = best_s;
            b->tuned_ms[i] = best;
        }
    }
    // then the form: whole frames in each form the volumes allow, launched directly on `stream`
    // (each writes the volumes' spare buffers, as the trials above)
    if (rc == SDFDDGI_OK) {
        b->form_ms[0] = b->form_ms[1] = 0.f;
        const bool can_merge = merged_ok(b, nullptr);
        const int saved = b->form_asked;
        for (int f = SDFDDGI_BATCH_FORM_BRANCHES; f <= SDFDDGI_BATCH_FORM_MERGED && rc == SDFDDGI_OK; ++f) {
            if (f == SDFDDGI_BATCH_FORM_MERGED && !can_merge) break;
            b->form_asked = f;
            float total = 0.f;
            for (int r = 0; r <= repeats && rc == SDFDDGI_OK; ++r) {  // the first frame warms up
                float rot[kMaxBatch * 9];
                frame_rotations(b, (uint32_t)r, rot);
                cudaError_t e = cudaMemcpyAsync(b->rot_dev, rot, sizeof(float) * 9 * b->n, cudaMemcpyHostToDevice, st);
                for (int i = 0; i < b->n && e == cudaSuccess; ++i) e = order_map_write(b->vols[i], b->vols[i]->cur ^ 1, st);
                if (e == cudaSuccess) e = cudaEventRecord(e0, st);
                if (e != cudaSuccess) {
                    rc = bfail(SDFDDGI_ERR_CUDA, "batch_autotune: frame trial failed");
                    break;
                }
                rc = record_frame(b, st);
                if (rc) break;
                if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                    rc = bfail(SDFDDGI_ERR_CUDA, "batch_autotune: frame trial failed");
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (r > 0) total += ms;
            }
            b->form_ms[f - 1] = total / repeats;
        }
        b->form_asked = saved;
        if (rc == SDFDDGI_OK)
            b->form_tuned = can_merge && b->form_ms[1] < b->form_ms[0] ? SDFDDGI_BATCH_FORM_MERGED
                                                                       : SDFDDGI_BATCH_FORM_BRANCHES;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    drop_graphs(b);
    return rc;
}

SDFDDGI_API int sdfddgi_batch_set_form(sdfddgi_batch* b, int32_t form) {
    if (!b || form < SDFDDGI_BATCH_FORM_AUTO || form > SDFDDGI_BATCH_FORM_MERGED)
        return bfail(SDFDDGI_ERR_INVALID_ARG, "batch_set_form: invalid arguments");
    if (form == SDFDDGI_BATCH_FORM_MERGED) {
        const char* why = nullptr;
        if (!merged_ok(b, &why)) return bfail(SDFDDGI_ERR_INVALID_ARG, why ? why : "batch_set_form: not mergeable");
    }
    b->form_asked = form;  // the graph cache is keyed by the form
    return SDFDDGI_OK;
}

SDFDDGI_API int sdfddgi_batch_form(const sdfddgi_batch* b, int32_t* form, float ms[2]) {
    if (!b || !form) return bfail(SDFDDGI_ERR_INVALID_ARG, "batch_form: NULL argument");
    *form = frame_form(b);
    if (ms) {
        ms[0] = b->form_ms[0];
        ms[1] = b->form_ms[1];
    }
    return SDFDDGI_OK;
}

SDFDDGI_API int sdfddgi_batch_schedule(const sdfddgi_batch* b, int32_t i, int32_t out[5], float* tuned_ms) {
    if (!b || !out || i < 0 || i >= b->n) return bfail(SDFDDGI_ERR_INVALID_ARG, "batch_schedule: invalid arguments");
    out[0] = b->sched[i].pool_batch;
    out[1] = b->sched[i].blocks_per_sm;
    out[2] = b->sched[i].gather;
    out[3] = b->sched[i].index;
    out[4] = b->sched[i].steps;
    if (tuned_ms) *tuned_ms = b->tuned_ms[i];
    return SDFDDGI_OK;
}

}  // extern "C"
