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
// are discarded: the epilogue keeps the 36 interior rows of each probe and writes each also
// into the border rows that mirror it (the octahedral fixup), the next layer's padding.
// Every MMA reads its whole 4 KiB A tile from shared memory, which bounds these narrow
// products; layer 3 (3 outputs) therefore keeps the three horizontal taps apart in N and
// sums them across neighbouring rows in its epilogue (9 MMAs instead of 27), and layer 1
// puts its last 3 input channels of all three horizontal taps into one K step (21 MMAs
// instead of 27).
//   weights   all three layers as bf16 B-operand images (100.5 KiB), loaded once per CTA by
//             the bulk-copy engine and kept in shared memory;
//   layer 1   K = 35 channels padded to 48, N = 64;  layer 2 K = 64, N = 48, 9 taps;
//   layer 3   K = 48, N = 16 (3 dx x 3 outputs), 3 taps (dy);
//   accumulators in tensor-memory columns 0, 64, 112 of the group's 128.
// The inputs are first reduced, per probe and texel, to one 16-byte feature texel (bf16
// irradiance rgb and the two scaled depth moments of the texel's 2 x 2 depth block), so a
// tile row gathers its 7 probes' features with 7 vector loads.
// Per tile: features -> MMA 1 -> epilogue (bias, ReLU, bf16, borders) -> MMA 2 -> epilogue ->
// MMA 3 -> residual + output maps. The CTA's four warp groups (4 warps each, one thread per
// row of a tile) run independent tile streams, each with one activation image (a layer's
// output overwrites its input once the layer's MMAs are done), its tensor-memory columns
// and its mbarrier, so that one group's MMAs overlap the others' epilogues. A group loads
// the next tile's feature texels, validity bytes, residual texel and probe flags into
// registers while the current tile's layers run. The group's first thread issues its MMAs;
// completion is an mbarrier armed by tcgen05.commit.
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
constexpr int kN1 = 64, kN2 = 48, kN3 = 16;     // accumulator columns (layer 3: 3 dx x 3 outputs)
constexpr int kCol1 = 0, kCol2 = 64, kCol3 = 112;   // within a warp group's 128 columns
constexpr int kGroups = 4;                          // warp groups, each with its own tile stream
constexpr int kGroupThreads = 128;
constexpr int kGroupCols = 128;
constexpr int kTmemCols = 512;                      // 4 x 128; allocations are powers of 2
constexpr int kThreads = kGroups * kGroupThreads;
// B images: per layer, per tap, [K / 8][N][8 channels] bf16 (K-major, no swizzle)
// layer 3 keeps the horizontal taps apart in N: column (dx + 1) * 3 + co of the image of
// vertical tap dy holds W3[dy][dx][.][co], so its B images are 3 (dy) of N = 16 (9 used)
// layer 1: its first 32 input channels per tap (9 x [32][64]), then its channels 32-34 with
// the three dx side by side in K per vertical tap (3 x [16][64]; see store_features)
constexpr int kImg1a = 9 * 32 * kN1 * 2, kImg1 = kImg1a + 3 * 16 * kN1 * 2;
constexpr int kImg2 = 9 * kK2 * kN2 * 2, kImg3 = 3 * kK3 * kN3 * 2;
constexpr int kImgBytes = kImg1 + kImg2 + kImg3;  // 102,912
// A images: [K / 8][kBufRows][8 channels] bf16
// A image of a group, 64 channels: the features (48), layer 1's output (64), layer 2's (48)
constexpr int kAct = kBufRows * kK2 * 2;
constexpr int kSmemBytes = kImgBytes + kGroups * kAct;
static_assert(kImgBytes % 16 == 0 && kAct % 16 == 0, "16-byte alignment of the images");
static_assert(kK2 >= kK1 && kK2 >= kK3 && kK2 >= kN1 && kK2 >= kN2, "one image holds every layer's input");
static_assert(kK1 >= kCin && kK3 == kC2 && kK2 == kC1 && kN1 == kC1 && kN2 == kC2 && kN3 >= 3 * kCout, "layer shapes");

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
    if (base == 0) {  // layer 1 (K = 48 of which 35 used, N = 64)
        float w = 0.f;
        int off;
        if (e < kImg1a / 2) {  // tap, channel k < 32
            const int tap = e / (32 * N), n = e % (32 * N) / 32, k = e % 32;
            w = use[woff + (tap * cin + k) * cout + n];
            off = tap * 32 * N + b_off(n, k, N) / 2;
        } else {               // vertical tap dy + 1 = slot, K row j: channel 32 + j % 3 of dx = j / 3 - 1
            const int f = e - kImg1a / 2, slot = f / (16 * N), n = f % (16 * N) / 16, j = f % 16;
            if (j < 9) w = use[woff + ((slot * 3 + j / 3) * cin + 32 + j % 3) * cout + n];
            off = kImg1a / 2 + slot * 16 * N + b_off(n, j, N) / 2;
        }
        img[off] = __float2bfloat16_rn(w);
        return;
    }
    const int slot = e / (K * N), r = e % (K * N), n = r / K, k = r % K;
    float w = 0.f;
    if (base == (kImg1 + kImg2) / 2) {  // layer 3: slot = dy + 1, n = (dx + 1) * 3 + co
        if (k < cin && n < 3 * kCout) w = use[woff + ((slot * 3 + n / kCout) * cin + k) * cout + n % kCout];
    } else if (k < cin && n < cout) {   // layer 2: slot = tap
        w = use[woff + (slot * cin + k) * cout + n];
    }
    img[base + slot * K * N + b_off(n, k, N) / 2] = __float2bfloat16_rn(w);
}

// The feature texel of (probe, texel t): bf16 {r, g | b, mu / s | mu2 / s^2, 0 | 0, 0}, with
// mu, mu2 the means of the t's 2 x 2 block of depth moments and s the depth scale; the
// values and their rounding are those of the features the CUDA-core path computes.
__global__ void feature_texels_kernel(MapsView m, float inv_s, uint4* __restrict__ feat) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)m.P * kTex) return;
    const int p = (int)(i >> 6), t = (int)(i & 63), r = t >> 3, c = t & 7;
    const float4 v = m.irr[i];
    const float2* d = m.depth + (size_t)p * 256 + (2 * r) * 16 + 2 * c;
    const float2 d0 = d[0], d1 = d[1], d2 = d[16], d3 = d[17];
    const float mu = ((d0.x + d1.x) + (d2.x + d3.x)) * 0.25f;
    const float mu2 = ((d0.y + d1.y) + (d2.y + d3.y)) * 0.25f;
    feat[i] = make_uint4(pack2(v.x, v.y), pack2(v.z, mu * inv_s), pack2(mu2 * inv_s * inv_s, 0.f), 0u);
}

struct TcArgs {
    MapsView m;
    const uint4* feat;      // [P][64] feature texels
    const __nv_bfloat16* img;
    const float* use;       // biases at kOffB1, kOffB2, kOffB3
    float4* out;            // may be m.irr: each texel is read and written by one thread
    uint32_t* status;       // bit 1: a bounded wait gave up (sticky)
    int n_tiles;
};

// What one thread of a group needs of a tile before its layers run: the feature texels of
// its row's probe and 6 neighbour candidates, the candidates' validity, its own irradiance
// texel (the residual's base) and its probe's flags. Loaded a tile ahead.
struct Pending {
    uint2 f[7];     // words 0, 1 of the feature texels: (r, g), (b, mu)
    uint32_t h[7];  // word 2: (mu2, 0)
    uint32_t ok[6];
    float4 x;
    uint32_t act;
};

__device__ __forceinline__ void load_pending(const TcArgs& a, int tile, int gtid, Pending& q) {
    const int p = tile * kProbesPerTile + gtid / kTex, t = gtid % kTex;
    if (p >= a.m.P) {
#pragma unroll
        for (int k = 0; k < 7; ++k) q.f[k] = make_uint2(0u, 0u), q.h[k] = 0u;
#pragma unroll
        for (int k = 0; k < 6; ++k) q.ok[k] = 0u;
        q.x = make_float4(0.f, 0.f, 0.f, 0.f);
        q.act = 0u;
        return;
    }
    // the -x, +x, -y, +y, -z, +z neighbours within the probe's grid; one outside the grid is
    // the probe itself, and so is one without history (chosen where the texels are used)
    const int nx = a.m.dims[0], ny = a.m.dims[1], nz = a.m.dims[2];
    const int g0 = p - p % a.m.per_grid, l = p - g0;
    const int x = l % nx, y = (l / nx) % ny, z = l / (nx * ny);
    const int cand[6] = {x > 0 ? p - 1 : p, x + 1 < nx ? p + 1 : p, y > 0 ? p - nx : p,
                         y + 1 < ny ? p + nx : p, z > 0 ? p - nx * ny : p, z + 1 < nz ? p + nx * ny : p};
    const uint32_t* f = reinterpret_cast<const uint32_t*>(a.feat);  // word 3 of a texel is zero: not read
    q.f[0] = *reinterpret_cast<const uint2*>(f + ((size_t)p * kTex + t) * 4);
    q.h[0] = f[((size_t)p * kTex + t) * 4 + 2];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        q.ok[k] = a.m.valid[cand[k]];
        q.f[k + 1] = *reinterpret_cast<const uint2*>(f + ((size_t)cand[k] * kTex + t) * 4);
        q.h[k + 1] = f[((size_t)cand[k] * kTex + t) * 4 + 2];
    }
    q.x = a.m.irr[(size_t)p * kTex + t];
    q.act = probe_active(a.m, p) ? 1u : 0u;
}

// The row's input channels into the group's A image as bf16 pairs: channels 0-31 in the
// CUDA-core path's order -- irradiance rgb of the probe and its 6 neighbours (0-20), then
// their depth moment pairs (21-34) -- and in the padding after channels 32-34, copies of
// channels 32-34 of the next two rows (35-37, 38-40; from the neighbouring lanes, the same
// 8-texel row wherever a kept output reads them), zeros in 41-47. One K step of layer 1 on
// the image shifted for dx = -1 then covers channels 32-34 of all three horizontal taps.
// Called by all threads of the group (the shuffles).
__device__ __forceinline__ void store_features(const Pending& q, unsigned char* act, int row) {
    uint3 f[7];
    f[0] = make_uint3(q.f[0].x, q.f[0].y, q.h[0]);
#pragma unroll
    for (int k = 1; k < 7; ++k)
        f[k] = q.ok[k - 1] ? make_uint3(q.f[k].x, q.f[k].y, q.h[k]) : f[0];
    // bf16 halves: x = (r, g), y = (b, mu), z = (mu2, 0)
    const auto lo_lo = [](uint32_t u, uint32_t v) { return __byte_perm(u, v, 0x5410); };
    const auto hi_lo = [](uint32_t u, uint32_t v) { return __byte_perm(u, v, 0x5432); };
    const auto lo_hi = [](uint32_t u, uint32_t v) { return __byte_perm(u, v, 0x7610); };
    uint32_t w[24];
#pragma unroll
    for (int j = 0; j < 3; ++j) {  // neighbours 2j, 2j + 1: channels 6j .. 6j + 5
        w[3 * j] = f[2 * j].x;
        w[3 * j + 1] = lo_lo(f[2 * j].y, f[2 * j + 1].x);
        w[3 * j + 2] = hi_lo(f[2 * j + 1].x, f[2 * j + 1].y);
    }
    w[9] = f[6].x;                       // channels 18, 19
    w[10] = lo_hi(f[6].y, f[0].y);       // 20 (b of neighbour 6), 21 (mu of the probe)
#pragma unroll
    for (int k = 0; k < 6; ++k) w[11 + k] = lo_hi(f[k].z, f[k + 1].y);  // mu2 of k, mu of k + 1
    // channels 32, 33 = w[16] and 34 = the low half of f[6].z, of this row and the next two
    const uint32_t u1 = __shfl_down_sync(0xffffffffu, w[16], 1), u2 = __shfl_down_sync(0xffffffffu, w[16], 2);
    const uint32_t c0 = f[6].z, c1 = __shfl_down_sync(0xffffffffu, c0, 1), c2 = __shfl_down_sync(0xffffffffu, c0, 2);
    w[17] = __byte_perm(c0, u1, 0x5410);  // 34, 35 (= 32 of the next row)
    w[18] = __byte_perm(u1, c1, 0x5432);  // 36, 37
    w[19] = u2;                           // 38, 39
    w[20] = c2 & 0xffffu;                 // 40, 41 = 0
#pragma unroll
    for (int k = 21; k < 24; ++k) w[k] = 0u;
#pragma unroll
    for (int g = 0; g < kK1 / 8; ++g)
        *reinterpret_cast<uint4*>(act + a_off(kGuard + row, 8 * g)) =
            make_uint4(w[4 * g], w[4 * g + 1], w[4 * g + 2], w[4 * g + 3]);
}

// Issues the MMAs of one layer and arms `bar` with their completion: for every tap slot, the
// A image shifted by the slot's row offset times the slot's B image, K / 16 steps each.
// TAPS = 9: one slot per tap (shift dy * 8 + dx); TAPS = 3: one per dy (shift dy * 8),
// the B image carrying the three dx in N.
template <int TAPS>
__device__ __forceinline__ void issue_layer(uint32_t a_img, uint32_t b_img, int K, int N, uint32_t d_tmem,
                                            uint64_t* bar) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t id = idesc(N);
#pragma unroll
    for (int k = 0; k < TAPS; ++k) {
        const int shift = TAPS == 9 ? tap_offset(k) : (k - 1) * 8;
        for (int s = 0; s < K / 16; ++s) {
            const uint32_t a = a_img + (uint32_t)(2 * s) * kBufRows * 16 + (uint32_t)(kGuard + shift) * 16;
            const uint32_t b = b_img + (uint32_t)(k * K * N * 2) + (uint32_t)(2 * s) * N * 16;
            mma_bf16(d_tmem, make_desc(a, kBufRows * 16, 128), make_desc(b, N * 16, 128), id, (k | s) ? 1u : 0u);
        }
    }
    mma_commit(bar);
}

// Issues layer 1's MMAs (N = 64) and arms `bar` with their completion: per tap, channels
// 0-31 of the A image shifted by dy * 8 + dx (2 K steps); then per vertical tap, channels
// 32-47 of the image shifted by dy * 8 - 1, which hold channels 32-34 of the rows for
// dx = -1, 0, +1 side by side (1 K step). 21 MMAs instead of 27.
__device__ __forceinline__ void issue_first(uint32_t a_img, uint32_t b_img, uint32_t d_tmem, uint64_t* bar) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t id = idesc(kN1);
#pragma unroll
    for (int k = 0; k < 9; ++k)
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const uint32_t a = a_img + (uint32_t)(2 * s) * kBufRows * 16 + (uint32_t)(kGuard + tap_offset(k)) * 16;
            const uint32_t b = b_img + (uint32_t)(k * 32 * kN1 * 2) + (uint32_t)(2 * s) * kN1 * 16;
            mma_bf16(d_tmem, make_desc(a, kBufRows * 16, 128), make_desc(b, kN1 * 16, 128), id, (k | s) ? 1u : 0u);
        }
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
        const uint32_t a = a_img + 4u * kBufRows * 16 + (uint32_t)(kGuard + (dy - 1) * 8 - 1) * 16;
        const uint32_t b = b_img + (uint32_t)kImg1a + (uint32_t)(dy * 16 * kN1 * 2);
        mma_bf16(d_tmem, make_desc(a, kBufRows * 16, 128), make_desc(b, kN1 * 16, 128), id, 1u);
    }
    mma_commit(bar);
}

// The rows of a tile that copy row `row` under the octahedral border fixup (Sec. 3.3): up
// to 3 border texels of the same probe mirror an interior texel. Packed 8 bits per row.
__device__ __forceinline__ uint32_t border_copies(int row, int* n) {
    const int pl = row / kTex, t = row % kTex;
    uint32_t rows = 0;
    int c = 0;
    for (int b = 0; b < kTex; ++b)
        if (b != t && border_source(b) == t) rows |= (uint32_t)(pl * kTex + b) << (8 * c++);
    *n = c;
    return rows;
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

// 32 consecutive fp32 columns of this thread's tensor-memory lane; the wait names the
// registers, so that no use of them is scheduled ahead of it
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
        "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

// Epilogue of a hidden layer for this thread's row: bias, ReLU, bf16, into channels
// [0, NCOLS) of the group's A image, 32 columns at a time. Interior rows only, each also
// into the `nb` border rows that mirror it (packed in `brows`): the next layer's padding.
template <int NCOLS>
__device__ __forceinline__ void hidden_epilogue(uint32_t taddr, const float* bias, int row, unsigned char* act,
                                                bool write, uint32_t brows, int nb) {
    const bool w = write && interior_row(row);
    __syncwarp();
#pragma unroll
    for (int c0 = 0; c0 < NCOLS; c0 += 32) {
        constexpr int kChunk = 32;
        float v[kChunk];
        if (NCOLS - c0 >= 32)
            tmem_ld32(taddr + c0, v);
        else
            tmem_ld16(taddr + c0, v);
        const int n = NCOLS - c0 >= 32 ? 32 : 16;
#pragma unroll
        for (int g = 0; g < kChunk / 8; ++g) {
            if (8 * g >= n || !w) continue;
            float x[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) x[j] = fmaxf(v[8 * g + j] + bias[c0 + 8 * g + j], 0.f);
            const uint4 u = make_uint4(pack2(x[0], x[1]), pack2(x[2], x[3]), pack2(x[4], x[5]), pack2(x[6], x[7]));
            *reinterpret_cast<uint4*>(act + a_off(kGuard + row, c0 + 8 * g)) = u;
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (j < nb) *reinterpret_cast<uint4*>(act + a_off(kGuard + (int)((brows >> (8 * j)) & 255u), c0 + 8 * g)) = u;
        }
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
    for (int i = tid; i < kGroups * kAct / 16; i += kThreads)
        reinterpret_cast<uint4*>(smem + kImgBytes)[i] = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) bulk_copy_g2s(s_img, a.img, kImgBytes, &bar_w);  // all weights, once per CTA
    if (!mbar_wait(&bar_w, 0, a.status)) s_fail = 1;
    __syncthreads();

    // ---- from here on the four warp groups run independent tile streams
    unsigned char* s_act = smem + kImgBytes + grp * kAct;
    const uint32_t img = smem_u32(s_act), img0 = smem_u32(s_img);
    const uint32_t tmem = s_tmem + (uint32_t)(grp * kGroupCols);
    uint64_t* bar = &bar_mma[grp];
    const int quarter = warp & 3, row = quarter * 32 + lane;  // this thread's tensor-memory lane (= gtid)
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    const bool leader = gtid == 0;
    int nb;
    const uint32_t brows = border_copies(row, &nb);
    bool fail = s_fail != 0;
    uint32_t phase = 0;
    auto wait_mma = [&]() {
        if (!mbar_wait(bar, phase & 1, a.status)) fail = true;
        ++phase;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    };

    const int stride = gridDim.x * kGroups;
    int tile = blockIdx.x * kGroups + grp;
    Pending pend;
    if (tile < a.n_tiles) load_pending(a, tile, gtid, pend);
    for (; tile < a.n_tiles; tile += stride) {
        const int p = tile * kProbesPerTile + gtid / kTex, t = gtid % kTex;  // this thread's texel
        // ---- features of the tile's 128 texels, bf16 into the A image
        store_features(pend, s_act, gtid);
        const float4 x = pend.x;
        const bool active = pend.act != 0u;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
        group_sync(grp);
        if (leader) issue_first(img, img0, tmem + kCol1, bar);
        if (tile + stride < a.n_tiles) load_pending(a, tile + stride, gtid, pend);  // in flight meanwhile

        // ---- layer 1 epilogue into the A image (64 channels; MMA 1 is done reading it)
        wait_mma();
        hidden_epilogue<kN1>(lane_base + kCol1, s_bias, row, s_act, !fail, brows, nb);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        fail = group_sync_or(grp, fail);
        if (fail) break;
        if (leader) issue_layer<9>(img, img0 + kImg1, kK2, kN2, tmem + kCol2, bar);

        // ---- layer 2 epilogue into channels 0-47 of the A image
        wait_mma();
        hidden_epilogue<kN2>(lane_base + kCol2, s_bias + kC1, row, s_act, !fail, brows, nb);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        fail = group_sync_or(grp, fail);
        if (fail) break;
        if (leader) issue_layer<3>(img, img0 + kImg1 + kImg2, kK3, kN3, tmem + kCol3, bar);

        // ---- layer 3: the dx taps' partial sums of rows row - 1, row, row + 1 (neighbouring
        // lanes; a warp's first and last rows are border texels, whose values are not kept),
        // then the residual on the probe's own irradiance, output maps
        wait_mma();
        {
            float v[16];
            __syncwarp();
            tmem_ld16(lane_base + kCol3, v);
            float o[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float l = __shfl_up_sync(0xffffffffu, v[c], 1);
                const float r = __shfl_down_sync(0xffffffffu, v[6 + c], 1);
                o[c] = (l + v[3 + c]) + r;
            }
            if (interior_row(row) && p < a.m.P && !fail) {
                s_y[grp][row * 3 + 0] = fmaxf(x.x + (o[0] + s_bias[kC1 + kC2 + 0]), 0.f);
                s_y[grp][row * 3 + 1] = fmaxf(x.y + (o[1] + s_bias[kC1 + kC2 + 1]), 0.f);
                s_y[grp][row * 3 + 2] = fmaxf(x.z + (o[2] + s_bias[kC1 + kC2 + 2]), 0.f);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        fail = group_sync_or(grp, fail);
        if (fail) break;
        if (p < a.m.P) {
            float4 y = x;
            if (active) {
                const int sr = (gtid / kTex) * kTex + border_source(t);
                y = make_float4(s_y[grp][sr * 3 + 0], s_y[grp][sr * 3 + 1], s_y[grp][sr * 3 + 2], x.w);
            }
            a.out[(size_t)p * kTex + t] = y;
        }
        group_sync(grp);  // s_y and the A image are rewritten by the group's next tile
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

cudaError_t tc_forward(TcState& s, const MapsView& m, float depth_scale, const float* use, void* feat, float4* out,
                       cudaStream_t st) {
    const int64_t texels = (int64_t)m.P * kTex;
    feature_texels_kernel<<<(unsigned)((texels + 255) / 256), 256, 0, st>>>(m, 1.f / depth_scale,
                                                                          static_cast<uint4*>(feat));
    TcArgs a;
    a.m = m;
    a.feat = static_cast<const uint4*>(feat);
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
