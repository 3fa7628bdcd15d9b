// denoiser_tc.cu -- inference of the probe denoiser on the tensor cores (tcgen05, bf16 x
// bf16 -> fp32), one persistent CTA per SM.
//
// A 3 x 3 convolution over the 8 x 8 bordered texel grid is 9 shifted matrix products:
//   D[row][co] += sum_ci A[row + tap_k][ci] * W[k][ci][co],   tap_k = dy * 8 + dx,
// with one row per texel. A tile is 128 rows = the 64 texels of 2 probes. The layer input
// lives in shared memory as a K-major image without swizzle: 8 channels of one texel per
// 16-byte row, rows consecutive, so a shifted operand is the same image read from a start
// address 16 * tap_k bytes further on (10 guard rows at both ends absorb the shift). Rows of
// border texels (and rows a shift carries into the neighbouring probe) produce values that
// are discarded: the epilogue keeps the 36 interior rows of each probe and rebuilds the
// border with the octahedral fixup, which is the next layer's padding.
//   weights   all three layers as bf16 B-operand images (121.5 KiB), loaded once per CTA by
//             the bulk-copy engine and kept in shared memory;
//   layer 1   K = 35 channels padded to 48, N = 64;  layer 2 K = 64, N = 48;
//   layer 3   K = 48, N = 16 (3 used); accumulators in tensor-memory columns 0, 64, 112.
// Per tile: features (the group gathers the 7 probes' map texels) -> MMA 1 -> epilogue
// (bias, ReLU, bf16, border) -> MMA 2 -> epilogue -> MMA 3 -> residual + output maps.
// The CTA's three warp groups (4 warps each, one thread per row of a tile) run independent
// tile streams with their own activation images, tensor-memory columns and mbarrier, so
// that one group's MMAs overlap the others' feature gathers and epilogues (three streams
// fill the shared memory: 121.5 KiB of weights + 3 x 32.4 KiB of activation images). The group's
// first thread issues its MMAs; completion is an mbarrier armed by tcgen05.commit.
// Every wait is bounded; on timeout the kernel records bit 1 of the status word, releases
// its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "denoiser.h"
#include "tcgen05.cuh"

namespace sdfddgi {
namespace dn {
namespace {

using namespace sdfddgi::tc;

constexpr int kRows = 128;                      // texel rows per tile: 2 probes x 64
constexpr int kProbesPerTile = kRows / kTex;
constexpr int kGuard = 10;                      // guard rows at each end (shifts reach +-9)
constexpr int kBufRows = kRows + 2 * kGuard;    // 148
constexpr int kK1 = 48, kK2 = 64, kK3 = 48;     // input channels, padded to multiples of 16
constexpr int kN1 = 64, kN2 = 48, kN3 = 16;     // accumulator columns (layer 3: 3 used)
constexpr int kCol1 = 0, kCol2 = 64, kCol3 = 112;   // within a warp group's 128 columns
constexpr int kGroups = 3;                          // warp groups, each with its own tile stream
constexpr int kGroupThreads = 128;
constexpr int kGroupCols = 128;
constexpr int kTmemCols = 512;                      // 3 x 128 used; allocations are powers of 2
constexpr int kThreads = kGroups * kGroupThreads;
// B images: per layer, per tap, [K / 8][N][8 channels] bf16 (K-major, no swizzle)
constexpr int kImg1 = 9 * kK1 * kN1 * 2, kImg2 = 9 * kK2 * kN2 * 2, kImg3 = 9 * kK3 * kN3 * 2;
constexpr int kImgBytes = kImg1 + kImg2 + kImg3;  // 124,416
// A images: [K / 8][kBufRows][8 channels] bf16
constexpr int kActA = kBufRows * kK1 * 2;       // 48 channels: the features, then layer 2's output
constexpr int kActB = kBufRows * kK2 * 2;       // 64 channels: layer 1's output
constexpr int kSmemBytes = kImgBytes + kGroups * (kActA + kActB);
static_assert(kImgBytes % 16 == 0 && kActA % 16 == 0 && kActB % 16 == 0, "16-byte alignment of the images");
static_assert(kK1 >= kCin && kK3 == kC2 && kK2 == kC1 && kN1 == kC1 && kN2 == kC2 && kN3 >= kCout, "layer shapes");

// instruction descriptor: D fp32, A and B bf16, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc(int n) { return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24); }

// byte offset of (row, channel) in an A image / of (n, k) in one tap of a B image
__host__ __device__ constexpr uint32_t a_off(int row, int c) { return (uint32_t)((c >> 3) * kBufRows * 16 + row * 16 + (c & 7) * 2); }
__host__ __device__ constexpr uint32_t b_off(int n, int k, int N) { return (uint32_t)((k >> 3) * N * 16 + n * 16 + (k & 7) * 2); }

__device__ __forceinline__ uint32_t pack2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// The weights (already rounded to bf16 values in `use`) as the B images.
__global__ void build_images_kernel(const float* __restrict__ use, __nv_bfloat16* __restrict__ img) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // one image element
    int e = i, base = 0, K, N, cin, cout, woff;
    if (e < kImg1 / 2) {
        K = kK1, N = kN1, cin = kCin, cout = kC1, woff = kOffW1;
    } else if ((e -= kImg1 / 2) < kImg2 / 2) {
        K = kK2, N = kN2, cin = kC1, cout = kC2, woff = kOffW2, base = kImg1 / 2;
    } else if ((e -= kImg2 / 2) < kImg3 / 2) {
        K = kK3, N = kN3, cin = kC2, cout = kCout, woff = kOffW3, base = (kImg1 + kImg2) / 2;
    } else {
        return;
    }
    const int tap = e / (K * N), r = e % (K * N), n = r / K, k = r % K;
    const float w = (k < cin && n < cout) ? use[woff + (tap * cin + k) * cout + n] : 0.f;
    img[base + tap * K * N + b_off(n, k, N) / 2] = __float2bfloat16_rn(w);
}

struct TcArgs {
    MapsView m;
    float inv_s;
    const __nv_bfloat16* img;
    const float* use;       // biases at kOffB1, kOffB2, kOffB3
    float4* out;
    uint32_t* status;       // bit 1: a bounded wait gave up (sticky)
    int n_tiles;
};

// Issues the 9 taps x (K / 16) MMAs of one layer and arms `bar` with their completion.
__device__ __forceinline__ void issue_layer(uint32_t a_img, uint32_t b_img, int K, int N, uint32_t d_tmem,
                                            uint64_t* bar) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t id = idesc(N);
    for (int k = 0; k < 9; ++k) {
        const int shift = tap_offset(k);
        for (int s = 0; s < K / 16; ++s) {
            const uint32_t a = a_img + (uint32_t)(2 * s) * kBufRows * 16 + (uint32_t)(kGuard + shift) * 16;
            const uint32_t b = b_img + (uint32_t)(k * K * N * 2) + (uint32_t)(2 * s) * N * 16;
            mma_bf16(d_tmem, make_desc(a, kBufRows * 16, 128), make_desc(b, N * 16, 128), id, (k | s) ? 1u : 0u);
        }
    }
    mma_commit(bar);
}

// Copies into every border row of both probes of a tile, for channel groups [g0, g1), the
// 16-byte rows of the interior texels they mirror.
__device__ __forceinline__ void fix_borders(unsigned char* act, int g0, int g1, int gtid) {
    constexpr int kBorder = kTex - kInt;  // 28
    const int n = kProbesPerTile * kBorder * (g1 - g0);
    for (int e = gtid; e < n; e += kGroupThreads) {
        const int g = g0 + e / (kProbesPerTile * kBorder), r = e % (kProbesPerTile * kBorder);
        const int pl = r / kBorder, b = r % kBorder;
        // the b-th border texel in row-major order
        const int t = b < 8 ? b : (b >= 20 ? 56 + (b - 20) : 8 * (1 + (b - 8) / 2) + ((b - 8) & 1) * 7);
        const int row = kGuard + pl * kTex + t, src = kGuard + pl * kTex + border_source(t);
        *reinterpret_cast<uint4*>(act + a_off(row, g * 8)) = *reinterpret_cast<const uint4*>(act + a_off(src, g * 8));
    }
}

__device__ __forceinline__ bool interior_row(int row) {
    const int t = row & 63, r = t >> 3, c = t & 7;
    return r >= 1 && r <= kN && c >= 1 && c <= kN;
}

// barrier of one warp group (128 threads); ids 1 and 2 (0 is __syncthreads)
__device__ __forceinline__ void group_sync(int g) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kGroupThreads) : "memory");
}

// the same barrier, returning the OR of v over the group (one decision for all its threads)
__device__ __forceinline__ bool group_sync_or(int g, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(1 + g), "r"(kGroupThreads)
        : "memory");
    return r != 0;
}

// Epilogue of a hidden layer for this thread's row: bias, ReLU, bf16, into channels
// [0, n) of the next layer's A image (interior rows only).
template <int NCOLS>
__device__ __forceinline__ void hidden_epilogue(uint32_t taddr, const float* bias, int row, unsigned char* act,
                                                bool write) {
    float v[NCOLS];
    __syncwarp();
#pragma unroll
    for (int c = 0; c < NCOLS; c += 16) tmem_ld16(taddr + c, v + c);
    if (!write || !interior_row(row)) return;
#pragma unroll
    for (int g = 0; g < NCOLS / 8; ++g) {
        float x[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = fmaxf(v[8 * g + j] + bias[8 * g + j], 0.f);
        *reinterpret_cast<uint4*>(act + a_off(kGuard + row, 8 * g)) =
            make_uint4(pack2(x[0], x[1]), pack2(x[2], x[3]), pack2(x[4], x[5]), pack2(x[6], x[7]));
    }
}

__global__ void __launch_bounds__(kThreads, 1) denoise_tc_kernel(const __grid_constant__ TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* s_img = smem;
    __shared__ float s_y[kGroups][kRows * 3];       // layer 3 outputs of each group's tile
    __shared__ __align__(8) uint64_t bar_w, bar_mma[kGroups];
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    __shared__ float s_bias[kC1 + kC2 + kCout];
    __shared__ uint32_t s_active[kGroups][kProbesPerTile];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int grp = tid / kGroupThreads, gtid = tid % kGroupThreads;  // warp group and its thread

    if (tid == 0) s_fail = (int)(*reinterpret_cast<const volatile uint32_t*>(a.status) & 2u);
    __syncthreads();
    if (s_fail) return;
    if (warp == 0) tmem_alloc(&s_tmem, kTmemCols);
    if (tid == 0) {
        mbar_init(&bar_w, 1);
        for (int g = 0; g < kGroups; ++g) mbar_init(&bar_mma[g], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = tid; i < kC1; i += kThreads) s_bias[i] = a.use[kOffB1 + i];
    for (int i = tid; i < kC2; i += kThreads) s_bias[kC1 + i] = a.use[kOffB2 + i];
    if (tid < kCout) s_bias[kC1 + kC2 + tid] = a.use[kOffB3 + tid];
    // zero the activation images once (guard rows and padding channels stay zero)
    for (int i = tid; i < kGroups * (kActA + kActB) / 16; i += kThreads)
        reinterpret_cast<uint4*>(smem + kImgBytes)[i] = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) bulk_copy_g2s(s_img, a.img, kImgBytes, &bar_w);  // all weights, once per CTA
    if (!mbar_wait(&bar_w, 0, a.status)) s_fail = 1;
    __syncthreads();

    // ---- from here on the three warp groups run independent tile streams
    unsigned char* s_actA = smem + kImgBytes + grp * (kActA + kActB);  // 48 channels: features, layer 2 out
    unsigned char* s_actB = s_actA + kActA;                             // 64 channels: layer 1 out
    const uint32_t imgA = smem_u32(s_actA), imgB = smem_u32(s_actB), img0 = smem_u32(s_img);
    const uint32_t tmem = s_tmem + (uint32_t)(grp * kGroupCols);
    uint64_t* bar = &bar_mma[grp];
    const int quarter = warp & 3, row = quarter * 32 + lane;  // this thread's tensor-memory lane
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    const bool leader = gtid == 0;
    bool fail = s_fail != 0;
    uint32_t phase = 0;
    auto wait_mma = [&]() {
        if (!mbar_wait(bar, phase & 1, a.status)) fail = true;
        ++phase;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    };

    for (int tile = blockIdx.x * kGroups + grp; tile < a.n_tiles; tile += gridDim.x * kGroups) {
        const int p0 = tile * kProbesPerTile;
        // ---- features of the tile's 128 texels, bf16 into image A
        if (gtid < kProbesPerTile) s_active[grp][gtid] = (p0 + gtid < a.m.P) && probe_active(a.m, p0 + gtid);
        {
            const int pl = gtid / kTex, t = gtid % kTex, p = p0 + pl;
            float f[kK1];
#pragma unroll
            for (int c = 0; c < kK1; ++c) f[c] = 0.f;
            if (p < a.m.P) {
                int src[7];
                neighbour_sources(a.m, p, src);
                const int r = t >> 3, c = t & 7;
#pragma unroll
                for (int k = 0; k < 7; ++k) {
                    const float4 v = a.m.irr[(size_t)src[k] * kTex + t];
                    f[3 * k] = v.x, f[3 * k + 1] = v.y, f[3 * k + 2] = v.z;
                    const float2* d = a.m.depth + (size_t)src[k] * 256 + (2 * r) * 16 + 2 * c;
                    const float2 d0 = d[0], d1 = d[1], d2 = d[16], d3 = d[17];
                    const float mu = ((d0.x + d1.x) + (d2.x + d3.x)) * 0.25f;
                    const float mu2 = ((d0.y + d1.y) + (d2.y + d3.y)) * 0.25f;
                    f[21 + 2 * k] = mu * a.inv_s;
                    f[22 + 2 * k] = mu2 * a.inv_s * a.inv_s;
                }
            }
#pragma unroll
            for (int g = 0; g < kK1 / 8; ++g) {
                const uint4 v = make_uint4(pack2(f[8 * g], f[8 * g + 1]), pack2(f[8 * g + 2], f[8 * g + 3]),
                                           pack2(f[8 * g + 4], f[8 * g + 5]), pack2(f[8 * g + 6], f[8 * g + 7]));
                *reinterpret_cast<uint4*>(s_actA + a_off(kGuard + gtid, 8 * g)) = v;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
        group_sync(grp);
        if (leader) issue_layer(imgA, img0, kK1, kN1, tmem + kCol1, bar);

        // ---- layer 1 epilogue into image B (64 channels), then its borders
        wait_mma();
        hidden_epilogue<kN1>(lane_base + kCol1, s_bias, row, s_actB, !fail);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        fail = group_sync_or(grp, fail);
        if (fail) break;
        fix_borders(s_actB, 0, kC1 / 8, gtid);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        group_sync(grp);
        if (leader) issue_layer(imgB, img0 + kImg1, kK2, kN2, tmem + kCol2, bar);

        // ---- layer 2 epilogue into image A (the features are no longer read)
        wait_mma();
        hidden_epilogue<kN2>(lane_base + kCol2, s_bias + kC1, row, s_actA, !fail);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        fail = group_sync_or(grp, fail);
        if (fail) break;
        fix_borders(s_actA, 0, kC2 / 8, gtid);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        group_sync(grp);
        if (leader) issue_layer(imgA, img0 + kImg1 + kImg2, kK3, kN3, tmem + kCol3, bar);

        // ---- layer 3: residual on the probe's own irradiance, output maps
        wait_mma();
        {
            float v[16];
            __syncwarp();
            tmem_ld16(lane_base + kCol3, v);
            const int pl = row / kTex, t = row % kTex, p = p0 + pl;
            if (interior_row(row) && p < a.m.P && !fail) {
                const float4 x = a.m.irr[(size_t)p * kTex + t];
                s_y[grp][row * 3 + 0] = fmaxf(x.x + (v[0] + s_bias[kC1 + kC2 + 0]), 0.f);
                s_y[grp][row * 3 + 1] = fmaxf(x.y + (v[1] + s_bias[kC1 + kC2 + 1]), 0.f);
                s_y[grp][row * 3 + 2] = fmaxf(x.z + (v[2] + s_bias[kC1 + kC2 + 2]), 0.f);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        fail = group_sync_or(grp, fail);
        if (fail) break;
        {
            const int pl = gtid / kTex, t = gtid % kTex, p = p0 + pl;
            if (p < a.m.P) {
                const float4 x = a.m.irr[(size_t)p * kTex + t];
                float4 y = x;
                if (s_active[grp][pl]) {
                    const int sr = pl * kTex + border_source(t);
                    y = make_float4(s_y[grp][sr * 3 + 0], s_y[grp][sr * 3 + 1], s_y[grp][sr * 3 + 2], x.w);
                }
                a.out[(size_t)p * kTex + t] = y;
            }
        }
        group_sync(grp);  // s_y and s_active are rewritten by the group's next tile
    }
    if (fail) s_fail = 1;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) tmem_dealloc(s_tmem, kTmemCols);
    if (s_fail && tid == 0) atomicOr(a.status, 2u);
}

}  // namespace

cudaError_t tc_create(TcState& s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMalloc(&s.wimg, kImgBytes);
    if (e == cudaSuccess) e = cudaMalloc(&s.status, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(s.status, 0, sizeof(uint32_t));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(denoise_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    s.wimg_bytes = kImgBytes;
    return e;
}

void tc_destroy(TcState& s) {
    cudaFree(s.wimg);
    cudaFree(s.status);
    s.wimg = nullptr;
    s.status = nullptr;
}

cudaError_t tc_prepare(TcState& s, const float* use, cudaStream_t st) {
    const int n = kImgBytes / 2;
    build_images_kernel<<<(n + 255) / 256, 256, 0, st>>>(use, static_cast<__nv_bfloat16*>(s.wimg));
    return cudaGetLastError();
}

cudaError_t tc_forward(TcState& s, const MapsView& m, float depth_scale, const float* use, float4* out,
                       cudaStream_t st) {
    TcArgs a;
    a.m = m;
    a.inv_s = 1.f / depth_scale;
    a.img = static_cast<const __nv_bfloat16*>(s.wimg);
    a.use = use;
    a.out = out;
    a.status = s.status;
    a.n_tiles = (m.P + kProbesPerTile - 1) / kProbesPerTile;
    const int grid = std::min((a.n_tiles + kGroups - 1) / kGroups, std::max(1, s.sms));
    denoise_tc_kernel<<<grid, kThreads, kSmemBytes, st>>>(a);
    return cudaGetLastError();
}

}  // namespace dn
}  // namespace sdfddgi
