// primitives.cu -- the scene as a union of analytic SDF primitives grouped into clusters
// (Sec. 3.1, "SDF Cluster"). The host groups the bounded primitives (spheres, boxes,
// capsules) by the Morton order of their centres into clusters of a fixed size, each with
// a bounding box; the unbounded ones (half-spaces, hollow balls) are kept apart and taken
// by every query. The kernels' query (device.cuh, analytic_sdf) then skips every cluster
// whose box lies farther than the best distance found so far.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "handles.h"

using namespace sdfddgi;

namespace {

bool bounded(int type) {
    return type == SDFDDGI_PRIM_SPHERE || type == SDFDDGI_PRIM_BOX || type == SDFDDGI_PRIM_CAPSULE;
}

int n_params(int type) {
    switch (type) {
        case SDFDDGI_PRIM_SPHERE: return 4;
        case SDFDDGI_PRIM_BOX: return 6;
        case SDFDDGI_PRIM_CAPSULE: return 7;
        case SDFDDGI_PRIM_PLANE_Y: return 1;
        case SDFDDGI_PRIM_INV_SPHERE: return 4;
        default: return -1;
    }
}

// Axis-aligned bounds of a bounded primitive.
void prim_box(const sdfddgi_primitive& q, float lo[3], float hi[3]) {
    const float* p = q.params;
    for (int a = 0; a < 3; ++a) {
        switch (q.type) {
            case SDFDDGI_PRIM_SPHERE:
                lo[a] = p[a] - p[3];
                hi[a] = p[a] + p[3];
                break;
            case SDFDDGI_PRIM_BOX:
                lo[a] = p[a] - p[3 + a];
                hi[a] = p[a] + p[3 + a];
                break;
            default:  // capsule
                lo[a] = std::min(p[a], p[3 + a]) - p[6];
                hi[a] = std::max(p[a], p[3 + a]) + p[6];
                break;
        }
    }
}

uint32_t spread10(uint32_t x) {  // 10 bits to every third bit
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

PrimDev to_dev(const sdfddgi_primitive& q, int index) {
    PrimDev d{};
    d.type = q.type;
    d.index = index;
    for (int k = 0; k < 7; ++k) d.p[k] = q.params[k];
    for (int k = 0; k < 3; ++k) {
        d.albedo[k] = q.albedo[k];
        d.emission[k] = q.emission[k];
    }
    return d;
}

}  // namespace

extern "C" SDFDDGI_API int sdfddgi_upload_primitives(sdfddgi_scene* s, const sdfddgi_primitive* prims, int32_t n,
                                                     const float lo[3], const float hi[3], float unit,
                                                     int32_t cluster_size) {
    if (!s || !prims || !lo || !hi) return report_error(SDFDDGI_ERR_INVALID_ARG, "upload_primitives: NULL argument");
    if (n < 1 || n > (1 << 20)) return report_error(SDFDDGI_ERR_INVALID_ARG, "upload_primitives: n outside [1, 2^20]");
    if (cluster_size < 0 || cluster_size > 4096)
        return report_error(SDFDDGI_ERR_INVALID_ARG, "upload_primitives: cluster_size outside [0, 4096]");
    if (!(unit > 0.f) || !std::isfinite(unit))
        return report_error(SDFDDGI_ERR_INVALID_ARG, "upload_primitives: unit must be positive and finite");
    int dims[3];
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(lo[a]) || !std::isfinite(hi[a]) || !(hi[a] > lo[a]))
            return report_error(SDFDDGI_ERR_INVALID_ARG, "upload_primitives: the box needs lo < hi, finite");
        const double cells = std::ceil((double)(hi[a] - lo[a]) / unit);
        if (cells < 2 || cells > 1e6) return report_error(SDFDDGI_ERR_INVALID_ARG, "upload_primitives: box / unit out of range");
        dims[a] = (int)cells;
    }
    std::vector<int> order, free_list;
    std::vector<uint32_t> key(n, 0);
    for (int k = 0; k < n; ++k) {
        const sdfddgi_primitive& q = prims[k];
        const int np = n_params(q.type);
        if (np < 0) return report_error(SDFDDGI_ERR_INVALID_ARG, "upload_primitives: unknown primitive type");
        for (int j = 0; j < np; ++j)
            if (!std::isfinite(q.params[j]))
                return report_error(SDFDDGI_ERR_INVALID_ARG, "upload_primitives: a parameter is not finite");
        for (int j = 0; j < 3; ++j)
            if (!std::isfinite(q.albedo[j]) || !std::isfinite(q.emission[j]) || q.albedo[j] < 0.f || q.emission[j] < 0.f)
                return report_error(SDFDDGI_ERR_INVALID_ARG, "upload_primitives: a material is negative or not finite");
        if ((q.type == SDFDDGI_PRIM_SPHERE || q.type == SDFDDGI_PRIM_INV_SPHERE) && q.params[3] < 0.f)
            return report_error(SDFDDGI_ERR_INVALID_ARG, "upload_primitives: negative radius");
        if (q.type == SDFDDGI_PRIM_CAPSULE && q.params[6] < 0.f)
            return report_error(SDFDDGI_ERR_INVALID_ARG, "upload_primitives: negative radius");
        if (q.type == SDFDDGI_PRIM_BOX && (q.params[3] < 0.f || q.params[4] < 0.f || q.params[5] < 0.f))
            return report_error(SDFDDGI_ERR_INVALID_ARG, "upload_primitives: negative half-extent");
        if (!bounded(q.type)) {
            free_list.push_back(k);
            continue;
        }
        float bl[3], bh[3];
        prim_box(q, bl, bh);
        uint32_t code = 0;
        for (int a = 0; a < 3; ++a) {
            const double c = (0.5 * ((double)bl[a] + bh[a]) - lo[a]) / ((double)hi[a] - lo[a]);
            const uint32_t q10 = (uint32_t)std::min(1023.0, std::max(0.0, std::floor(c * 1024.0)));
            code |= spread10(q10) << a;
        }
        key[k] = code;
        order.push_back(k);
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return key[a] < key[b]; });
    const int size = cluster_size > 0 ? cluster_size : std::max<int>(1, (int)order.size());
    std::vector<PrimDev> dev;
    std::vector<ClusterDev> cl;
    for (int k : free_list) dev.push_back(to_dev(prims[k], k));
    for (size_t start = 0; start < order.size(); start += size) {
        ClusterDev c{};
        c.first = (int)dev.size();
        c.count = (int)std::min<size_t>(size, order.size() - start);
        for (int a = 0; a < 3; ++a) {
            c.lo[a] = INFINITY;
            c.hi[a] = -INFINITY;
        }
        for (int j = 0; j < c.count; ++j) {
            const int k = order[start + j];
            float bl[3], bh[3];
            prim_box(prims[k], bl, bh);
            for (int a = 0; a < 3; ++a) {
                c.lo[a] = std::min(c.lo[a], bl[a]);
                c.hi[a] = std::max(c.hi[a], bh[a]);
            }
            dev.push_back(to_dev(prims[k], k));
        }
        // inflate by far more than the float rounding of the box distance and of the
        // primitives' distances, so that culling never drops the nearest primitive
        for (int a = 0; a < 3; ++a) {
            const float pad = 1e-3f * unit + 1e-5f * std::max(std::fabs(c.lo[a]), std::fabs(c.hi[a]));
            c.lo[a] -= pad;
            c.hi[a] += pad;
        }
        cl.push_back(c);
    }
    PrimDev* d_prims = nullptr;
    ClusterDev* d_cl = nullptr;
    cudaError_t e = cudaMalloc(&d_prims, sizeof(PrimDev) * dev.size());
    if (e == cudaSuccess && !cl.empty()) e = cudaMalloc(&d_cl, sizeof(ClusterDev) * cl.size());
    if (e == cudaSuccess) e = cudaMemcpy(d_prims, dev.data(), sizeof(PrimDev) * dev.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !cl.empty())
        e = cudaMemcpy(d_cl, cl.data(), sizeof(ClusterDev) * cl.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d_prims);
        cudaFree(d_cl);
        return report_error(e == cudaErrorMemoryAllocation ? SDFDDGI_ERR_OOM : SDFDDGI_ERR_CUDA, cudaGetErrorString(e));
    }
    cudaFree(s->prims);
    cudaFree(s->clusters);
    s->prims = d_prims;
    s->clusters = d_cl;
    s->n_prims = n;
    s->n_unbounded = (int)free_list.size();
    s->n_clusters = (int)cl.size();
    for (int a = 0; a < 3; ++a) {
        s->dims[a] = dims[a];
        s->origin[a] = lo[a];
    }
    s->h = unit;
    s->dtype = kAnalytic;
    s->has_sdf = true;
    s->has_material = false;
    s->version++;
    return SDFDDGI_OK;
}
