// denoiser.cu -- the learned form: a small convolutional network that corrects a low-ray-
// count probe update toward the converged irradiance (not in the paper; the network and
// its input are defined in sdfddgi.h). Training and the CUDA-core inference run here:
//   features   thread per (probe, texel): the 35 input channels from the probe's and its 6
//              neighbours' maps (irradiance rgb, 2 x 2-averaged depth moments);
//   conv_fwd   CTA per probe: the layer input (64 texels x Cin) staged in shared memory, a
//              thread per (interior texel, output channel), then ReLU and the octahedral
//              border fixup of the output (the next layer's padding). The last layer adds
//              the residual to the probe's irradiance and, when training, forms the loss
//              and its gradient;
//   bwd_data   CTA per probe: the gradient in a layer's input, folded from the border
//              texels back onto the interior texels they copy, times the ReLU mask;
//   bwd_weight thread per weight and chunk of probes, accumulated with atomics;
//   adam       thread per parameter.
// The tensor-core inference is in denoiser_tc.cu.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>

#include "denoiser.h"
#include "handles.h"

using namespace sdfddgi;
using namespace sdfddgi::dn;

namespace {

__device__ __forceinline__ float rnd(float x, bool r) { return r ? __bfloat162float(__float2bfloat16_rn(x)) : x; }

// ---------------------------------------------------------------- features
__global__ void features_kernel(MapsView m, float inv_s, bool round, float* __restrict__ X0) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)m.P * kTex) return;
    const int p = (int)(i >> 6), t = (int)(i & 63);
    int src[7];
    neighbour_sources(m, p, src);
    float* out = X0 + i * kCin;
    for (int k = 0; k < 7; ++k) {
        const float4 v = m.irr[(size_t)src[k] * kTex + t];
        out[3 * k + 0] = rnd(v.x, round);
        out[3 * k + 1] = rnd(v.y, round);
        out[3 * k + 2] = rnd(v.z, round);
    }
    const int r = t >> 3, c = t & 7;
    for (int k = 0; k < 7; ++k) {
        const float2* d = m.depth + (size_t)src[k] * 256 + (2 * r) * 16 + 2 * c;
        const float2 a = d[0], b = d[1], e = d[16], f = d[17];
        const float mu = ((a.x + b.x) + (e.x + f.x)) * 0.25f;
        const float mu2 = ((a.y + b.y) + (e.y + f.y)) * 0.25f;
        out[21 + 2 * k] = rnd(mu * inv_s, round);
        out[22 + 2 * k] = rnd(mu2 * inv_s * inv_s, round);
    }
}

__global__ void count_active_kernel(MapsView m, int* n_active) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = p < m.P && probe_active(m, p);
    const unsigned ballot = __ballot_sync(0xffffffffu, act);
    if ((threadIdx.x & 31) == 0 && ballot) atomicAdd(n_active, __popc(ballot));
}

// ---------------------------------------------------------------- forward
struct LastArgs {
    MapsView m;
    const float4* target;  // null: inference
    float* pre;            // [P][36][3] own irradiance + residual (before the output ReLU)
    float* dZ;             // [P][36][3] loss gradient in the residual (training)
    float* loss;
    const int* n_active;
    float4* out;           // null, or the corrected maps
};

// One CTA per probe. in: [P][64][CIN] bordered layer input; out (hidden layers): [P][64][COUT].
template <int CIN, int COUT, bool LAST>
__global__ void __launch_bounds__(256) conv_fwd_kernel(const float* __restrict__ in, const float* __restrict__ w,
                                                       const float* __restrict__ b, float* __restrict__ out,
                                                       bool round, LastArgs la) {
    extern __shared__ float sm[];
    float* fin = sm;                      // [64][CIN]
    float* fo = sm + kTex * CIN;          // [36][COUT]
    const int p = blockIdx.x;
    const float* src = in + (size_t)p * kTex * CIN;
    for (int i = threadIdx.x; i < kTex * CIN; i += blockDim.x) fin[i] = src[i];
    __syncthreads();
    float part = 0.f;
    bool act = true;
    float nn = 1.f;
    if constexpr (LAST) {
        act = probe_active(la.m, p);
        nn = (float)max(*la.n_active, 1) * (float)(kInt * 3);
    }
    for (int o = threadIdx.x; o < kInt * COUT; o += blockDim.x) {
        const int q = o / COUT, co = o - q * COUT;
        const int t = interior_texel(q);
        float acc = b[co];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float* f = fin + (t + tap_offset(k)) * CIN;
            const float* wk = w + (size_t)k * CIN * COUT + co;
#pragma unroll 5
            for (int ci = 0; ci < CIN; ++ci) acc = fmaf(f[ci], wk[ci * COUT], acc);
        }
        if constexpr (!LAST) {
            fo[o] = rnd(fmaxf(acc, 0.f), round);
        } else {
            const float4 x = la.m.irr[(size_t)p * kTex + t];
            const float base = co == 0 ? x.x : (co == 1 ? x.y : x.z);
            const float pr = base + acc;
            const size_t k3 = (size_t)p * kInt * 3 + o;
            la.pre[k3] = pr;
            fo[o] = fmaxf(pr, 0.f);
            if (la.target) {
                const float4 tg = la.target[(size_t)p * kTex + t];
                const float tv = co == 0 ? tg.x : (co == 1 ? tg.y : tg.z);
                const float d = act ? fmaxf(pr, 0.f) - tv : 0.f;
                part = fmaf(d, d, part);
                la.dZ[k3] = pr > 0.f ? 2.f * d / nn : 0.f;
            }
        }
    }
    __syncthreads();
    if constexpr (!LAST) {
        float* dst = out + (size_t)p * kTex * COUT;
        for (int i = threadIdx.x; i < kTex * COUT; i += blockDim.x) {
            const int t = i / COUT, c = i - t * COUT;
            dst[i] = fo[interior_index(border_source(t)) * COUT + c];
        }
    } else {
        if (la.target) {
            __shared__ float red[8];
            for (int off = 16; off; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
            __syncthreads();
            if (threadIdx.x == 0) {
                float s = 0.f;
                for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
                if (s != 0.f) atomicAdd(la.loss, s / nn);
            }
        }
        if (la.out) {
            for (int t = threadIdx.x; t < kTex; t += blockDim.x) {
                const float4 x = la.m.irr[(size_t)p * kTex + t];
                float4 y = x;
                if (act) {
                    const int q = interior_index(border_source(t));
                    y = make_float4(fo[q * 3 + 0], fo[q * 3 + 1], fo[q * 3 + 2], x.w);
                }
                la.out[(size_t)p * kTex + t] = y;
            }
        }
    }
}

// ---------------------------------------------------------------- backward
// dZprev[p][q][ci] = mask(q, ci) * sum over the texels t that show interior texel q (q
// itself and the border texels copying it) of sum_k sum_co W[k][ci][co] dZ[t - tap k][co].
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) bwd_data_kernel(const float* __restrict__ dZ, const float* __restrict__ wt,
                                                       const float* __restrict__ fin, float* __restrict__ dZprev) {
    __shared__ float dz[kInt * COUT];
    __shared__ int8_t shows[kInt][4];  // texels showing each interior texel, -1 terminated
    const int p = blockIdx.x;
    for (int i = threadIdx.x; i < kInt * COUT; i += blockDim.x) dz[i] = dZ[(size_t)p * kInt * COUT + i];
    if (threadIdx.x < kInt) {
        const int q = threadIdx.x, tq = interior_texel(q);
        int n = 0;
        for (int t = 0; t < kTex; ++t)
            if (border_source(t) == tq) shows[q][n++] = (int8_t)t;
        for (; n < 4; ++n) shows[q][n] = -1;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < kInt * CIN; o += blockDim.x) {
        const int q = o / CIN, ci = o - q * CIN;
        const int tq = interior_texel(q);
        float acc = 0.f;
        for (int j = 0; j < 4 && shows[q][j] >= 0; ++j) {
            const int t = shows[q][j], r = t >> 3, c = t & 7;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const int r0 = r - (k / 3 - 1), c0 = c - (k % 3 - 1);
                if (r0 < 1 || r0 > kN || c0 < 1 || c0 > kN) continue;
                const float* g = dz + ((r0 - 1) * kN + (c0 - 1)) * COUT;
                const float* wk = wt + (size_t)k * COUT * CIN + ci;
                for (int co = 0; co < COUT; ++co) acc = fmaf(g[co], wk[co * CIN], acc);
            }
        }
        const bool live = fin[((size_t)p * kTex + tq) * CIN + ci] > 0.f;
        dZprev[(size_t)p * kInt * CIN + o] = live ? acc : 0.f;
    }
}

// gw[k][ci][co] += sum over a chunk of probes and the 36 interior texels q of
// fin[p][q + tap k][ci] * dZ[p][q][co]; gb[co] += the sum of dZ over the chunk.
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) bwd_weight_kernel(const float* __restrict__ fin, const float* __restrict__ dZ,
                                                         int P, int chunk, float* __restrict__ gw,
                                                         float* __restrict__ gb) {
    const int wi = blockIdx.x * blockDim.x + threadIdx.x;
    const int p0 = blockIdx.y * chunk, p1 = min(P, p0 + chunk);
    constexpr int kW = 9 * CIN * COUT;
    if (wi < kW) {
        const int k = wi / (CIN * COUT), ci = (wi / COUT) % CIN, co = wi % COUT;
        const int off = tap_offset(k);
        float acc = 0.f;
        for (int p = p0; p < p1; ++p) {
            const float* f = fin + (size_t)p * kTex * CIN + ci;
            const float* g = dZ + (size_t)p * kInt * COUT + co;
#pragma unroll 6
            for (int q = 0; q < kInt; ++q) acc = fmaf(f[(interior_texel(q) + off) * CIN], g[q * COUT], acc);
        }
        atomicAdd(gw + wi, acc);
    } else if (wi < kW + COUT) {
        const int co = wi - kW;
        float acc = 0.f;
        for (int p = p0; p < p1; ++p)
            for (int q = 0; q < kInt; ++q) acc += dZ[((size_t)p * kInt + q) * COUT + co];
        atomicAdd(gb + co, acc);
    }
}

// ---------------------------------------------------------------- parameters
__global__ void adam_kernel(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, float lr, float bc1, float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    const float gi = g[i];
    const float mi = kBeta1 * m[i] + (1.f - kBeta1) * gi;
    const float vi = kBeta2 * v[i] + (1.f - kBeta2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + kEps);
}

// The weights as the kernels read them: rounded to bf16 or not, biases unrounded, and
// each layer's weights also transposed to [tap][out][in] for the backward pass.
__global__ void prepare_weights_kernel(const float* __restrict__ theta, bool round, float* __restrict__ use,
                                       float* __restrict__ wt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    const bool is_bias = (i >= kOffB1 && i < kOffW2) || (i >= kOffB2 && i < kOffW3) || i >= kOffB3;
    const float x = is_bias ? theta[i] : rnd(theta[i], round);
    use[i] = x;
    if (is_bias) return;
    int off, cin, cout;
    if (i < kOffB1) off = kOffW1, cin = kCin, cout = kC1;
    else if (i < kOffB2) off = kOffW2, cin = kC1, cout = kC2;
    else off = kOffW3, cin = kC2, cout = kCout;
    const int j = i - off, k = j / (cin * cout), ci = (j / cout) % cin, co = j % cout;
    wt[off + ((size_t)k * cout + co) * cin + ci] = x;
}

int dfail(int code, const char* msg) { return report_error(code, msg); }

}  // namespace

// ---------------------------------------------------------------- handle
struct sdfddgi_denoiser {
    float depth_scale = 1.f;
    float* theta = nullptr;  // [kParams] master parameters
    float* m = nullptr;      // Adam moments
    float* v = nullptr;
    float* grad = nullptr;
    float* use = nullptr;    // weights as read by the kernels (see prepare_weights_kernel)
    float* wt = nullptr;     // transposed weights
    int prepared = -1;       // mode the use/wt copies were made for (-1: stale)
    int step = 0;
    // work space for P probes
    int64_t ws_P = 0;
    float* X0 = nullptr;
    float* F1 = nullptr;
    float* F2 = nullptr;
    float* pre = nullptr;
    float* dZ3 = nullptr;
    float* dZ2 = nullptr;
    float* dZ1 = nullptr;
    float4* out = nullptr;   // denoise_volume's result before it is copied back
    int* n_active = nullptr;
    float* loss = nullptr;
    sdfddgi::dn::TcState tc;
};

namespace {

void free_ws(sdfddgi_denoiser* d) {
    for (void* p : {(void*)d->X0, (void*)d->F1, (void*)d->F2, (void*)d->pre, (void*)d->dZ3, (void*)d->dZ2,
                    (void*)d->dZ1, (void*)d->out})
        cudaFree(p);
    d->X0 = d->F1 = d->F2 = d->pre = d->dZ3 = d->dZ2 = d->dZ1 = nullptr;
    d->out = nullptr;
    d->ws_P = 0;
}

int ensure_ws(sdfddgi_denoiser* d, int64_t P) {
    if (P <= d->ws_P) return SDFDDGI_OK;
    cudaDeviceSynchronize();  // earlier work may still read the old buffers
    free_ws(d);
    const size_t n = (size_t)P;
    cudaError_t e = cudaMalloc(&d->X0, n * kTex * kCin * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&d->F1, n * kTex * kC1 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&d->F2, n * kTex * kC2 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&d->pre, n * kInt * 3 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&d->dZ3, n * kInt * 3 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&d->dZ2, n * kInt * kC2 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&d->dZ1, n * kInt * kC1 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&d->out, n * kTex * sizeof(float4));
    if (e != cudaSuccess) {
        free_ws(d);
        return dfail(SDFDDGI_ERR_OOM, "denoiser: work space allocation failed");
    }
    d->ws_P = P;
    return SDFDDGI_OK;
}

int check_maps(const sdfddgi_probe_maps* m, MapsView* v) {
    if (!m || !m->irr || !m->depth || !m->valid) return dfail(SDFDDGI_ERR_INVALID_ARG, "denoiser: NULL maps");
    int64_t pg = 1;
    for (int a = 0; a < 3; ++a) {
        if (m->dims[a] < 1 || m->dims[a] > 4096) return dfail(SDFDDGI_ERR_INVALID_ARG, "denoiser: dims out of range");
        pg *= m->dims[a];
    }
    if (m->n_grids < 1 || pg * m->n_grids > ((int64_t)1 << 24))
        return dfail(SDFDDGI_ERR_INVALID_ARG, "denoiser: n_grids out of range (at most 2^24 probes)");
    for (int a = 0; a < 3; ++a) v->dims[a] = m->dims[a];
    v->per_grid = (int)pg;
    v->P = (int)(pg * m->n_grids);
    v->irr = reinterpret_cast<const float4*>(m->irr);
    v->depth = reinterpret_cast<const float2*>(m->depth);
    v->valid = m->valid;
    v->states = m->states;
    return SDFDDGI_OK;
}

cudaError_t prepare(sdfddgi_denoiser* d, int mode, cudaStream_t st) {
    if (d->prepared == mode) return cudaSuccess;
    prepare_weights_kernel<<<(kParams + 255) / 256, 256, 0, st>>>(d->theta, mode != SDFDDGI_DENOISE_SIMT_FP32,
                                                                  d->use, d->wt);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && mode == SDFDDGI_DENOISE_TENSOR) e = tc_prepare(d->tc, d->use, st);
    if (e == cudaSuccess) d->prepared = mode;
    return e;
}

template <int CIN, int COUT, bool LAST>
cudaError_t launch_fwd(const float* in, const float* w, const float* b, float* out, bool round, const LastArgs& la,
                       int P, cudaStream_t st) {
    const size_t smem = (size_t)(kTex * CIN + kInt * COUT) * sizeof(float);
    static_assert((kTex * CIN + kInt * COUT) * sizeof(float) <= 48 * 1024, "static shared-memory limit");
    conv_fwd_kernel<CIN, COUT, LAST><<<P, 256, smem, st>>>(in, w, b, out, round, la);
    return cudaGetLastError();
}

// features and the three layers; target non-null: also the loss and dZ3
cudaError_t forward_simt(sdfddgi_denoiser* d, const MapsView& m, bool round, const float4* target, float4* out,
                         float* loss, cudaStream_t st) {
    const int P = m.P;
    cudaError_t e = cudaMemsetAsync(d->n_active, 0, sizeof(int), st);
    if (e == cudaSuccess && loss) e = cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (e != cudaSuccess) return e;
    count_active_kernel<<<(P + 255) / 256, 256, 0, st>>>(m, d->n_active);
    features_kernel<<<(unsigned)(((int64_t)P * kTex + 255) / 256), 256, 0, st>>>(m, 1.f / d->depth_scale, round,
                                                                               d->X0);
    LastArgs none{};
    const float* u = d->use;
    if ((e = launch_fwd<kCin, kC1, false>(d->X0, u + kOffW1, u + kOffB1, d->F1, round, none, P, st)) != cudaSuccess)
        return e;
    if ((e = launch_fwd<kC1, kC2, false>(d->F1, u + kOffW2, u + kOffB2, d->F2, round, none, P, st)) != cudaSuccess)
        return e;
    LastArgs la{m, target, d->pre, d->dZ3, loss, d->n_active, out};
    return launch_fwd<kC2, kCout, true>(d->F2, u + kOffW3, u + kOffB3, nullptr, round, la, P, st);
}

cudaError_t backward_simt(sdfddgi_denoiser* d, int P, float* grad, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(grad, 0, kParams * sizeof(float), st);
    if (e != cudaSuccess) return e;
    const int chunk = 32;
    const unsigned nch = (unsigned)((P + chunk - 1) / chunk);
    const float* wt = d->wt;
    bwd_weight_kernel<kC2, kCout><<<dim3((9 * kC2 * kCout + kCout + 255) / 256, nch), 256, 0, st>>>(
        d->F2, d->dZ3, P, chunk, grad + kOffW3, grad + kOffB3);
    bwd_data_kernel<kC2, kCout><<<P, 256, 0, st>>>(d->dZ3, wt + kOffW3, d->F2, d->dZ2);
    bwd_weight_kernel<kC1, kC2><<<dim3((9 * kC1 * kC2 + kC2 + 255) / 256, nch), 256, 0, st>>>(
        d->F1, d->dZ2, P, chunk, grad + kOffW2, grad + kOffB2);
    bwd_data_kernel<kC1, kC2><<<P, 256, 0, st>>>(d->dZ2, wt + kOffW2, d->F1, d->dZ1);
    bwd_weight_kernel<kCin, kC1><<<dim3((9 * kCin * kC1 + kC1 + 255) / 256, nch), 256, 0, st>>>(
        d->X0, d->dZ1, P, chunk, grad + kOffW1, grad + kOffB1);
    return cudaGetLastError();
}

int run_denoise(sdfddgi_denoiser* d, const MapsView& m, float4* out, int mode, cudaStream_t st) {
    int rc = ensure_ws(d, m.P);
    if (rc) return rc;
    cudaError_t e = prepare(d, mode, st);
    if (e == cudaSuccess) {
        if (mode == SDFDDGI_DENOISE_TENSOR)
            e = tc_forward(d->tc, m, d->depth_scale, d->use, d->X0, out, st);  // X0 holds P * 64 * 140 bytes
        else
            e = forward_simt(d, m, mode == SDFDDGI_DENOISE_SIMT_BF16, nullptr, out, nullptr, st);
    }
    if (e != cudaSuccess) return dfail(SDFDDGI_ERR_CUDA, cudaGetErrorString(e));
    return SDFDDGI_OK;
}

int run_gradients(sdfddgi_denoiser* d, const sdfddgi_probe_maps* maps, const float* target, int mode, float* grad,
                  float* loss, cudaStream_t st) {
    MapsView m{};
    int rc = check_maps(maps, &m);
    if (rc) return rc;
    if (!target || !grad || !loss) return dfail(SDFDDGI_ERR_INVALID_ARG, "denoiser_gradients: NULL argument");
    if (mode != SDFDDGI_DENOISE_SIMT_BF16 && mode != SDFDDGI_DENOISE_SIMT_FP32)
        return dfail(SDFDDGI_ERR_INVALID_ARG, "denoiser_gradients: mode must be SIMT_BF16 or SIMT_FP32");
    if ((rc = ensure_ws(d, m.P))) return rc;
    cudaError_t e = prepare(d, mode, st);
    if (e == cudaSuccess)
        e = forward_simt(d, m, mode == SDFDDGI_DENOISE_SIMT_BF16, reinterpret_cast<const float4*>(target), nullptr,
                         loss, st);
    if (e == cudaSuccess) e = backward_simt(d, m.P, grad, st);
    if (e != cudaSuccess) return dfail(SDFDDGI_ERR_CUDA, cudaGetErrorString(e));
    return SDFDDGI_OK;
}

}  // namespace

extern "C" {

SDFDDGI_API int sdfddgi_create_denoiser(const float* params, float depth_scale, sdfddgi_denoiser** out) {
    if (out) *out = nullptr;
    if (!out || !params) return dfail(SDFDDGI_ERR_INVALID_ARG, "create_denoiser: NULL argument");
    if (!(depth_scale > 0.f) || !std::isfinite(depth_scale))
        return dfail(SDFDDGI_ERR_INVALID_ARG, "create_denoiser: depth_scale must be positive and finite");
    for (int i = 0; i < kParams; ++i)
        if (!std::isfinite(params[i])) return dfail(SDFDDGI_ERR_INVALID_ARG, "create_denoiser: a parameter is not finite");
    sdfddgi_denoiser* d = new (std::nothrow) sdfddgi_denoiser();
    if (!d) return dfail(SDFDDGI_ERR_OOM, "create_denoiser: host allocation failed");
    d->depth_scale = depth_scale;
    const size_t bytes = kParams * sizeof(float);
    cudaError_t e = cudaMalloc(&d->theta, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&d->m, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&d->v, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&d->grad, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&d->use, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&d->wt, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&d->n_active, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&d->loss, sizeof(float));
    if (e == cudaSuccess) e = tc_create(d->tc);
    if (e == cudaSuccess) e = cudaMemcpy(d->theta, params, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(d->m, 0, bytes);
    if (e == cudaSuccess) e = cudaMemset(d->v, 0, bytes);
    if (e != cudaSuccess) {
        sdfddgi_destroy_denoiser(d);
        return dfail(e == cudaErrorMemoryAllocation ? SDFDDGI_ERR_OOM : SDFDDGI_ERR_CUDA, cudaGetErrorString(e));
    }
    *out = d;
    return SDFDDGI_OK;
}

SDFDDGI_API void sdfddgi_destroy_denoiser(sdfddgi_denoiser* d) {
    if (!d) return;
    cudaDeviceSynchronize();
    free_ws(d);
    tc_destroy(d->tc);
    for (void* p : {(void*)d->theta, (void*)d->m, (void*)d->v, (void*)d->grad, (void*)d->use, (void*)d->wt,
                    (void*)d->n_active, (void*)d->loss})
        cudaFree(p);
    delete d;
}

SDFDDGI_API int sdfddgi_denoiser_params(sdfddgi_denoiser* d, float* read, const float* write) {
    if (!d) return dfail(SDFDDGI_ERR_INVALID_ARG, "denoiser_params: denoiser is NULL");
    const size_t bytes = kParams * sizeof(float);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && read) e = cudaMemcpy(read, d->theta, bytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && write) {
        for (int i = 0; i < kParams; ++i)
            if (!std::isfinite(write[i])) return dfail(SDFDDGI_ERR_INVALID_ARG, "denoiser_params: a parameter is not finite");
        e = cudaMemcpy(d->theta, write, bytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(d->m, 0, bytes);
        if (e == cudaSuccess) e = cudaMemset(d->v, 0, bytes);
        d->step = 0;
        d->prepared = -1;
    }
    if (e != cudaSuccess) return dfail(SDFDDGI_ERR_CUDA, cudaGetErrorString(e));
    return SDFDDGI_OK;
}

SDFDDGI_API int sdfddgi_denoise(sdfddgi_denoiser* d, const sdfddgi_probe_maps* maps, float* out_irr, int32_t mode,
                                void* stream) {
    if (!d || !out_irr) return dfail(SDFDDGI_ERR_INVALID_ARG, "denoise: NULL argument");
    if (mode < SDFDDGI_DENOISE_TENSOR || mode > SDFDDGI_DENOISE_SIMT_FP32)
        return dfail(SDFDDGI_ERR_INVALID_ARG, "denoise: unknown mode");
    MapsView m{};
    int rc = check_maps(maps, &m);
    if (rc) return rc;
    if (out_irr == maps->irr) return dfail(SDFDDGI_ERR_INVALID_ARG, "denoise: out_irr must not alias maps->irr");
    return run_denoise(d, m, reinterpret_cast<float4*>(out_irr), mode, static_cast<cudaStream_t>(stream));
}

SDFDDGI_API int sdfddgi_denoise_volume(sdfddgi_denoiser* d, sdfddgi_volume* v, const sdfddgi_probe_state* states,
                                       int32_t mode, void* stream) {
    if (!d || !v) return dfail(SDFDDGI_ERR_INVALID_ARG, "denoise_volume: NULL argument");
    if (mode < SDFDDGI_DENOISE_TENSOR || mode > SDFDDGI_DENOISE_SIMT_FP32)
        return dfail(SDFDDGI_ERR_INVALID_ARG, "denoise_volume: unknown mode");
    sdfddgi_probe_maps maps{};
    for (int a = 0; a < 3; ++a) maps.dims[a] = v->desc.dims[a];
    maps.n_grids = 1;
    maps.irr = reinterpret_cast<const float*>(v->irr[v->cur]);
    maps.depth = reinterpret_cast<const float*>(v->depth[v->cur]);
    maps.valid = v->valid[v->cur];
    maps.states = states;
    MapsView m{};
    int rc = check_maps(&maps, &m);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((rc = ensure_ws(d, m.P))) return rc;
    // the tensor-core path reads its neighbours from the feature texels it makes first, so it
    // writes the volume's map in place; the CUDA-core path writes a copy
    if (mode == SDFDDGI_DENOISE_TENSOR) return run_denoise(d, m, reinterpret_cast<float4*>(v->irr[v->cur]), mode, st);
    if ((rc = run_denoise(d, m, d->out, mode, st))) return rc;
    cudaError_t e = cudaMemcpyAsync(v->irr[v->cur], d->out, (size_t)m.P * kTex * sizeof(float4),
                                    cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return dfail(SDFDDGI_ERR_CUDA, cudaGetErrorString(e));
    return SDFDDGI_OK;
}

SDFDDGI_API int sdfddgi_denoiser_status(sdfddgi_denoiser* d, uint32_t* flags) {
    if (flags) *flags = 0;
    if (!d) return dfail(SDFDDGI_ERR_INVALID_ARG, "denoiser_status: denoiser is NULL");
    uint32_t f = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&f, d->tc.status, sizeof f, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(d->tc.status, 0, sizeof f);
    if (e != cudaSuccess) return dfail(SDFDDGI_ERR_CUDA, cudaGetErrorString(e));
    if (flags) *flags = f;
    if (f & 2u) return dfail(SDFDDGI_ERR_TIMEOUT, "denoiser_status: a bounded wait of the tensor-core kernel gave up");
    return SDFDDGI_OK;
}

SDFDDGI_API int sdfddgi_denoiser_gradients(sdfddgi_denoiser* d, const sdfddgi_probe_maps* maps,
                                           const float* target_irr, int32_t mode, float* grad, float* loss,
                                           void* stream) {
    if (!d) return dfail(SDFDDGI_ERR_INVALID_ARG, "denoiser_gradients: denoiser is NULL");
    return run_gradients(d, maps, target_irr, mode, grad, loss, static_cast<cudaStream_t>(stream));
}

SDFDDGI_API int sdfddgi_denoiser_adam(sdfddgi_denoiser* d, const float* grad, float lr, void* stream) {
    if (!d || !grad) return dfail(SDFDDGI_ERR_INVALID_ARG, "denoiser_adam: NULL argument");
    if (!(lr >= 0.f) || !std::isfinite(lr)) return dfail(SDFDDGI_ERR_INVALID_ARG, "denoiser_adam: lr must be >= 0");
    d->step += 1;
    const float bc1 = (float)(1.0 - std::pow((double)kBeta1, d->step));
    const float bc2 = (float)(1.0 - std::pow((double)kBeta2, d->step));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    adam_kernel<<<(kParams + 255) / 256, 256, 0, st>>>(d->theta, d->m, d->v, grad, lr, bc1, bc2);
    d->prepared = -1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return dfail(SDFDDGI_ERR_CUDA, cudaGetErrorString(e));
    return SDFDDGI_OK;
}

SDFDDGI_API int sdfddgi_denoiser_train_step(sdfddgi_denoiser* d, const sdfddgi_probe_maps* maps,
                                            const float* target_irr, int32_t mode, float lr, float* loss,
                                            void* stream) {
    if (!d) return dfail(SDFDDGI_ERR_INVALID_ARG, "denoiser_train_step: denoiser is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = run_gradients(d, maps, target_irr, mode, d->grad, loss ? loss : d->loss, st);
    if (rc) return rc;
    return sdfddgi_denoiser_adam(d, d->grad, lr, stream);
}

}  // extern "C"
