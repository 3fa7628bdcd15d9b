// gather_tc.cu -- the gather of Eq. 3 on the 5th-generation tensor cores (tcgen05).
//
// For one frame the texel weights W[texel][ray] = max(0, u.d)^e are shared by every probe,
// so the gather of G probes is one dense contraction
//     D[texel][probe*5 + c] = sum_ray W[texel][ray] * V[ray][probe*5 + c],
// c = (radiance r, g, b, distance t, t^2), plus one column of ones shared by the G probes:
// every ray of a probe counts in its texels' weight sums, so that sum is the same for all
// probes, and numerator and denominator see the same rounding of W.
//   A = W, 256 texel rows (irradiance 0..35, depth 36..231, zero padding) as two M = 128
//       tiles, K-major, prepared once per frame by pack_weights_kernel as a shared-memory
//       image and brought in per 16-ray chunk with one bulk copy;
//   B = V for the CTA's 19 probes and the ones (N = 19 * 5 + 1 = 96), split by the CTA
//       from the rays' values;
//   D = two 128 x 96 fp32 accumulators in tensor memory.
// Precision (template parameter): fp32 operands split as hi + lo tf32 and multiplied as
// hi*hi + hi*lo + lo*hi (kind::tf32, fp32 accumulation; products carry about 21 significant
// bits), or the precision form: one bf16 x bf16 product (kind::f16, fp32 accumulation).
// The K loop is warp-specialized over a ring of shared-memory stages: one lane copies the
// weight images in, four warps build the B operands, one lane issues the MMAs, with mbarriers
// between them (weights in, B built, MMAs done) and no CTA-wide barrier. Every wait is
// bounded: on a timeout the kernel records an error bit that stops the other roles and CTAs,
// waits for its own copies and MMAs in flight, and releases its tensor memory.
#include <cuda_bf16.h>

#include <algorithm>

#include "device.cuh"
#include "tcgen05.cuh"

namespace sdfddgi {

namespace tc {

constexpr int kG = kGatherTcProbes;           // probes per CTA
constexpr int kCh = 5;                        // value channels per probe
constexpr int kN = kG * kCh + 1;              // 96 accumulator columns per tile: the probes', then the ones
constexpr int kOnes = kN - 1;                 // the weight-sum column
static_assert(kN % 16 == 0 && kN <= 256, "an MMA of M = 128 takes N a multiple of 16 up to 256");
constexpr int kChunk = 16;                    // rays per K chunk
constexpr int kThreads = 256;
constexpr int kTmemCols = 256;                // 2 x 96 used
constexpr int kStagesTf32 = 2;                // stages of the tf32 ring (88 KiB: two CTAs per SM)

// Operand format: 4-byte tf32 in hi + lo parts, or one 2-byte bf16 part. Operands are
// K-major without swizzle: 8 x 16-byte core matrices, adjacent along K 128 B apart,
// adjacent along rows kRowBytes * 8 apart; one MMA consumes 32 bytes of K.
template <bool BF16>
struct Fmt {
    static constexpr int kElem = BF16 ? 2 : 4;
    static constexpr int kParts = BF16 ? 1 : 2;
    static constexpr int kRowBytes = kChunk * kElem;           // one row of one chunk
    static constexpr int kSbo = kRowBytes * 8;                 // between 8-row groups
    static constexpr int kTilePart = 128 * kRowBytes;          // one M = 128 tile, one part
    static constexpr int kABytes = 2 * kParts * kTilePart;     // both tiles, all parts
    static constexpr int kBPart = kN * kRowBytes;
    static constexpr int kBBytes = kParts * kBPart;
    static constexpr int kKSteps = kRowBytes / 32;
    // D fp32; A, B tf32 (kind::tf32) or bf16 (kind::f16); K-major; N = kN; M = 128
    static constexpr uint32_t kIdesc = (1u << 4) | ((BF16 ? 1u : 2u) << 7) | ((BF16 ? 1u : 2u) << 10) |
                                       ((uint32_t)(kN >> 3) << 17) | ((128u >> 4) << 24);
    __host__ __device__ static constexpr uint32_t offset(int row, int k) {
        return (uint32_t)((row >> 3) * kSbo + ((k * kElem) >> 4) * 128 + (row & 7) * 16 + ((k * kElem) & 15));
    }
};

// Operand stages of the gather's ring (44 KiB each for tf32, 11 KiB for bf16).
template <bool BF16>
struct Stages {
    static constexpr int value = BF16 ? 4 : kStagesTf32;
};
// Threads that build the B operand: one 16-byte core-matrix row of every channel of one
// probe and part per chunk (the ones rows are written once per CTA).
template <bool BF16>
struct Producers {
    static constexpr int value = kG * (kChunk / (16 / Fmt<BF16>::kElem)) * Fmt<BF16>::kParts;
};

template <bool BF16>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    if constexpr (BF16) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(Fmt<true>::kIdesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(Fmt<false>::kIdesc), "r"(accumulate)
            : "memory");
    }
}

// one operand element (hi or lo part) at byte offset off of a part
template <bool BF16>
__device__ __forceinline__ void put(unsigned char* part, uint32_t off, float v) {
    if constexpr (BF16)
        *reinterpret_cast<__nv_bfloat16*>(part + off) = __float2bfloat16_rn(v);
    else
        *reinterpret_cast<float*>(part + off) = v;
}

}  // namespace tc

// The weight matrix as the A operand's shared-memory image: per 16-ray chunk, per tile,
// its parts (tf32: hi then lo; bf16: one), element (row, k) at Fmt::offset(row, k).
// Thread per (texel row, ray).
template <bool BF16>
__device__ __forceinline__ void pack_weights_body(const UpdateParams& P, int i) {  // ray i
    using F = tc::Fmt<BF16>;
    const int m = threadIdx.x;         // texel row 0..255
    const float w = m < kTexels ? P.weights[(size_t)i * kTexels + m] : 0.f;
    const int c = i / tc::kChunk, k = i % tc::kChunk, t = m >> 7, r = m & 127;
    unsigned char* base = reinterpret_cast<unsigned char*>(P.wimage) + (size_t)c * F::kABytes + t * F::kParts * F::kTilePart;
    if constexpr (BF16) {
        tc::put<true>(base, F::offset(r, k), w);
    } else {
        const float hi = tc::to_tf32(w), lo = tc::to_tf32(w - hi);
        tc::put<false>(base, F::offset(r, k), hi);
        tc::put<false>(base + F::kTilePart, F::offset(r, k), lo);
    }
}

template <bool BF16>
__global__ void __launch_bounds__(256) pack_weights_kernel(const __grid_constant__ UpdateParams P) {
    pack_weights_body<BF16>(P, blockIdx.x);  // one ray per block
}

// The CTA of probes block * kG .. + kG - 1 of one launch's probes.
template <bool BF16>
__device__ __forceinline__ void gather_tc_body(const UpdateParams& P, int block) {
    using namespace tc;
    using F = Fmt<BF16>;
    constexpr int kABytes = F::kABytes, kBBytes = F::kBBytes, kBPart = F::kBPart, kTilePart = F::kTilePart;
    constexpr int kStages = Stages<BF16>::value;
    extern __shared__ __align__(1024) unsigned char smem[];
    auto sA = [&](int s) { return smem + (size_t)s * kABytes; };
    auto sB = [&](int s) { return smem + (size_t)kStages * kABytes + (size_t)s * kBBytes; };
    __shared__ __align__(8) uint64_t bar_full_a[kStages], bar_full_b[kStages], bar_empty[kStages], bar_prev;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_fail;
    __shared__ float s_hyst[kG];
    __shared__ uint32_t s_flags[kG];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int p0 = block * kG;
    const int ng = min(kG, P.P - p0);
    const int n_chunks = P.R / kChunk;

    // a launch in which a CTA already gave up does no further work (decided once per CTA)
    if (tid == 0) s_fail = (int)(*reinterpret_cast<const volatile uint32_t*>(&P.counters[kFailWord]) & 2u);
    __syncthreads();
    if (s_fail) return;

    if (warp == 0) {  // tensor-memory allocation: one warp, then give up the permit
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&bar_full_a[s], 1);
            mbar_init(&bar_full_b[s], Producers<BF16>::value);
            mbar_init(&bar_empty[s], 1);
        }
        mbar_init(&bar_prev, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the ones rows of every stage's B operand (tf32: hi 1, lo 0), which no chunk rewrites
    if (tid < kStages * F::kParts * kChunk) {
        const int st = tid / (F::kParts * kChunk), part = tid / kChunk % F::kParts, k = tid % kChunk;
        tc::put<BF16>(sB(st) + part * kBPart, F::offset(kOnes, k), part ? 0.f : 1.f);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    // ---- K loop over 16-ray chunks through a ring of kStages operand stages, in three roles
    // and without a CTA-wide barrier:
    //  the copier (warp 5, lane 0) brings chunk c's weight image into stage c % kStages with one
    //    bulk copy as soon as the MMAs of chunk c - kStages are done (full_a counts the bytes);
    //  producers (the first kProducers threads, in warps 0..4) build chunk c's B operand from
    //    the rays' values at the same time (they too wait only for chunk c - kStages's MMAs),
    //    split as the format asks, and arrive on full_b; each loads its values of the next
    //    chunk into registers one chunk ahead;
    //  the issuer (warp 6, lane 0) issues chunk c's MMAs once both operands are in and commits
    //    them to empty[c % kStages], which frees the stage for both.
    // Copies thus run up to kStages - 1 chunks ahead of the MMAs.
    constexpr int kVec = 16 / F::kElem;                   // K values per 16-byte core-matrix row
    constexpr int kQuads = kChunk / kVec;                 // such rows per operand row and chunk
    constexpr int kProducers = kG * kQuads * F::kParts;   // one (probe, rows, part) each
    constexpr int kProducerWarps = (kProducers + 31) / 32;
    static_assert(kProducerWarps <= 5, "producers fit in warps 0..4");
    static_assert(kStages * F::kParts * kChunk <= kThreads, "one thread per ones element");
    const uint32_t* fail_word = &P.counters[kFailWord];
    auto give_up = [&]() {
        atomicOr(&P.counters[kFailWord], 2u);  // the other roles and CTAs stop waiting too
        s_fail = 1;
    };
    if (warp < kProducerWarps) {  // whole warps: the stage wait is one lane's, shared by shuffle
        const bool worker = tid < kProducers;
        const int g = tid % kG, kq = (tid / kG) % kQuads, part = tid / (kG * kQuads);
        const bool live = worker && g < ng;
        const float4* src =
            P.ray_val + checked((size_t)(p0 + (live ? g : 0)) * P.R + kq * kVec,
                                (size_t)P.P * P.R - P.R + kChunk - kVec + 1,  // the reads below stay inside
                                P.vol.fail);
        float4 nxt[kVec];  // the next chunk's values, loaded one chunk ahead
#pragma unroll
        for (int j = 0; j < kVec; ++j) nxt[j] = live ? src[j] : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int c = 0; c < n_chunks; ++c) {
            const int s = c % kStages;
            float4 cur[kVec];
#pragma unroll
            for (int j = 0; j < kVec; ++j) cur[j] = nxt[j];
            if (live && c + 1 < n_chunks) {
#pragma unroll
                for (int j = 0; j < kVec; ++j) nxt[j] = src[(size_t)(c + 1) * kChunk + j];
            }
            if (c >= kStages) {  // the stage is free once chunk c - kStages's MMAs are done (its
                                 // weights may still be arriving); one lane of the warp waits,
                                 // the others take its answer
                int ok = 1;
                if (lane == 0) ok = mbar_wait(&bar_empty[s], ((c / kStages) - 1) & 1, fail_word);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) give_up();
                    break;
                }
            }
            if (!worker) continue;
            unsigned char* dst = sB(s) + part * kBPart;
#pragma unroll
            for (int q = 0; q < kCh; ++q) {  // the channel is a compile-time index: no divergence
                float x[kVec];
#pragma unroll
                for (int j = 0; j < kVec; ++j) {
                    const float4 v = cur[j];
                    x[j] = q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : q == 3 ? v.w : v.w * v.w;
                }
                uint4 w;
                if constexpr (BF16) {
                    uint32_t h[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const __nv_bfloat162 b2 = __floats2bfloat162_rn(x[2 * j], x[2 * j + 1]);
                        h[j] = *reinterpret_cast<const uint32_t*>(&b2);
                    }
                    w = make_uint4(h[0], h[1], h[2], h[3]);
                } else {
                    uint32_t h[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float hi = to_tf32(x[j]);
                        h[j] = __float_as_uint(part ? to_tf32(x[j] - hi) : hi);
                    }
                    w = make_uint4(h[0], h[1], h[2], h[3]);
                }
                *reinterpret_cast<uint4*>(dst + F::offset(g * kCh + q, kq * kVec)) = w;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar_full_b[s])) : "memory");
        }
    } else if (warp == 5 && lane == 0) {
        int last[kStages];  // per stage, the last chunk whose weight copy was issued into it
        for (int s = 0; s < kStages; ++s) last[s] = -1;
        for (int c = 0; c < n_chunks && !s_fail; ++c) {
            const int s = c % kStages;
            if (c >= kStages && !mbar_wait(&bar_empty[s], ((c / kStages) - 1) & 1, fail_word)) {
                give_up();
                break;
            }
            if (c == 0 && P.test_stall) continue;  // failure tests: chunk 0's weights never arrive
            bulk_copy_g2s(sA(s), reinterpret_cast<const unsigned char*>(P.wimage) + (size_t)c * kABytes, kABytes,
                          &bar_full_a[s]);
            last[s] = c;
        }
        // no copy of this CTA may still be writing its shared memory when the stages are
        // reused or the CTA ends (bounded, and not cut short by the failure bit)
        const uint32_t no_abort = 0;
        for (int s = 0; s < kStages; ++s)
            if (last[s] >= 0) mbar_wait(&bar_full_a[s], (last[s] / kStages) & 1, &no_abort);
    } else if (warp == 7 && lane < kG) {
        // the probes' flags and history weights, which only the epilogue reads: fetched here,
        // beside the K loop, rather than ahead of it
        uint32_t flags = 0;
        if (lane < ng) flags = P.states ? P.states[p0 + lane].flags : (uint32_t)SDFDDGI_PROBE_ACTIVE;
        s_flags[lane] = flags;
        s_hyst[lane] = (lane < ng && P.prev_valid[p0 + lane] && !(flags & SDFDDGI_PROBE_REJECT_HISTORY)) ? P.hyst : 0.f;
    } else if (warp == 6 && lane == 0) {
        int committed = 0;  // chunks whose MMAs were committed
        for (int c = 0; c < n_chunks && !s_fail; ++c) {
            const int s = c % kStages;
            const uint32_t ph = (c / kStages) & 1;
            if (!mbar_wait(&bar_full_a[s], ph, fail_word) || !mbar_wait(&bar_full_b[s], ph, fail_word)) {
                give_up();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(sA(s)), b0 = smem_u32(sB(s));
#pragma unroll
            for (int t = 0; t < 2; ++t) {
#pragma unroll
                for (int ks = 0; ks < F::kKSteps; ++ks) {
                    const uint32_t ak = ks * 256, d = tmem + t * kN;  // 32 bytes of K per MMA
                    const uint32_t at = a0 + t * F::kParts * kTilePart + ak;
                    const uint64_t ahi = make_desc(at, 128, F::kSbo), bhi = make_desc(b0 + ak, 128, F::kSbo);
                    mma<BF16>(d, ahi, bhi, (c > 0 || ks > 0) ? 1u : 0u);
                    if constexpr (!BF16) {
                        const uint64_t alo = make_desc(at + kTilePart, 128, F::kSbo);
                        const uint64_t blo = make_desc(b0 + kBPart + ak, 128, F::kSbo);
                        mma<false>(d, ahi, blo, 1u);
                        mma<false>(d, alo, bhi, 1u);
                    }
                }
            }
            mma_commit(&bar_empty[s]);
            committed = c + 1;
        }
        // every committed MMA complete before the accumulators are read or released (bounded,
        // not cut short: a commit covers all earlier MMAs of this thread)
        if (committed > 0) {
            const uint32_t no_abort = 0;
            const int c = committed - 1;
            if (!mbar_wait(&bar_empty[c % kStages], (c / kStages) & 1, s_fail ? &no_abort : fail_word)) give_up();
        }
        if (committed < n_chunks && !s_fail) give_up();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // ---- epilogue. The CTA's probes are consecutive, so their previous maps are two contiguous
    // blocks; bulk copies bring them into the staging buffers (the free operand stages) while
    // the accumulators come out of tensor memory, and each texel is blended in place.
    float4* s_irr = reinterpret_cast<float4*>(smem);                       // [kG][64]   (stages reused)
    float2* s_dep = reinterpret_cast<float2*>(smem + kG * kIrrT * kIrrT * 16);  // [kG][256]
    const uint32_t prev_bytes = (uint32_t)ng * (kIrrT * kIrrT * 16 + kDepT * kDepT * 8);
    const bool prev_issued = !s_fail;  // thread 0 issues the copies exactly when this holds
    if (prev_issued && tid == 0) {
        bulk_expect(&bar_prev, prev_bytes);
        bulk_copy(s_irr, P.prev_irr + (size_t)p0 * (kIrrT * kIrrT), (uint32_t)ng * kIrrT * kIrrT * 16, &bar_prev);
        bulk_copy(s_dep, P.prev_depth + (size_t)p0 * (kDepT * kDepT), (uint32_t)ng * kDepT * kDepT * 8, &bar_prev);
    }
    if (!s_fail) {
        const int t = warp >> 2, row = (warp & 3) * 32 + lane, j = t * 128 + row;
        const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + t * kN;
        // Blends probe g's texel j from its five sums and the shared weight sum.
        auto blend = [&](int g, float wsum, float a0, float a1, float a2, float a3, float a4) {
            if (g >= ng) return;
            const bool live = (s_flags[g] & SDFDDGI_PROBE_ACTIVE) && wsum > 0.f;
            const float hyst = s_hyst[g], keep = 1.f - hyst, inv = live ? 1.f / wsum : 0.f;
            if (j < kIrrTexels) {
                const int k = (j / kIrrN + 1) * kIrrT + (j % kIrrN + 1);
                float4 out = s_irr[g * kIrrT * kIrrT + k];  // last frame's texel
                if (live) {
                    out.x = fmaf(hyst, out.x, keep * (a0 * inv));
                    out.y = fmaf(hyst, out.y, keep * (a1 * inv));
                    out.z = fmaf(hyst, out.z, keep * (a2 * inv));
                    out.w = 1.f;
                }
                s_irr[g * kIrrT * kIrrT + k] = out;
            } else {
                const int jj = j - kIrrTexels, k = (jj / kDepN + 1) * kDepT + (jj % kDepN + 1);
                float2 out = s_dep[g * kDepT * kDepT + k];  // last frame's texel
                if (live) {
                    out.x = fmaf(hyst, out.x, keep * (a3 * inv));
                    out.y = fmaf(hyst, out.y, keep * (a4 * inv));
                }
                s_dep[g * kDepT * kDepT + k] = out;
            }
        };
        static_assert(kG == 19 && kCh == 5, "the column ranges below");
        // columns 80..95 (probes 16..18 and the weight sum), then 0..47 (probes 0..8 and the
        // first three sums of probe 9), then 48..79 (the rest of probe 9, probes 10..15);
        // tcgen05.ld is warp-collective, so every lane loads
        float hi[16], lo[48], mid[32];
        __syncwarp();
        tmem_ld16(lane_addr + 80, hi);
        tmem_ld16(lane_addr, lo);
        tmem_ld16(lane_addr + 16, lo + 16);
        tmem_ld16(lane_addr + 32, lo + 32);
        if (!mbar_wait(&bar_prev, 0, &P.counters[kFailWord])) s_fail = 1;
        const float wsum = hi[kOnes - 80];
        const bool mine = j < kTexels && !s_fail;
        if (mine) {
#pragma unroll
            for (int g = 0; g < 9; ++g) {
                const float* a = lo + g * kCh;
                blend(g, wsum, a[0], a[1], a[2], a[3], a[4]);
            }
        }
        __syncwarp();
        tmem_ld16(lane_addr + 48, mid);
        tmem_ld16(lane_addr + 64, mid + 16);
        if (mine) {
            blend(9, wsum, lo[45], lo[46], lo[47], mid[0], mid[1]);
#pragma unroll
            for (int g = 10; g < 16; ++g) {
                const float* a = mid + (g * kCh - 48);
                blend(g, wsum, a[0], a[1], a[2], a[3], a[4]);
            }
#pragma unroll
            for (int g = 16; g < 19; ++g) {
                const float* a = hi + (g * kCh - 80);
                blend(g, wsum, a[0], a[1], a[2], a[3], a[4]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    if (s_fail) {
        if (tid == 0) {
            // the copies of last frame's maps may still be in flight (bounded, not cut short)
            const uint32_t no_abort = 0;
            if (prev_issued) mbar_wait(&bar_prev, 0, &no_abort);
            atomicOr(&P.counters[kFailWord], 2u);  // reported by the host as a timeout
        }
        return;
    }

    // ---- contiguous stores of the staged maps. An active probe's border texel takes the
    // interior texel it mirrors (every border texel's source is an interior one, so no border
    // pass over shared memory is needed); an inactive probe's staged map is its old map.
    static_assert(kIrrT == 8 && kDepT == 16, "the index arithmetic below");
    float4* cur_i = P.cur_irr + (size_t)p0 * (kIrrT * kIrrT);
    for (int e = tid; e < ng * kIrrT * kIrrT; e += kThreads) {
        const int g = e >> 6;
        int y = (e >> 3) & 7, x = e & 7;
        if ((y == 0 || y == kIrrT - 1 || x == 0 || x == kIrrT - 1) && (s_flags[g] & SDFDDGI_PROBE_ACTIVE)) {
            const int2 sc = border_source(y, x, kIrrN);
            y = sc.x;
            x = sc.y;
        }
        cur_i[e] = s_irr[(g << 6) + y * kIrrT + x];
    }
    // depth: two texels of one row per 16-byte store
    float4* cur_d4 = reinterpret_cast<float4*>(P.cur_depth + (size_t)p0 * (kDepT * kDepT));
    for (int e = tid; e < ng * kDepT * kDepT / 2; e += kThreads) {
        const int g = e >> 7, y = (e >> 3) & 15, x = (e & 7) * 2;
        const float2* m = s_dep + (g << 8);
        float2 a, b;
        if ((y == 0 || y == kDepT - 1 || x == 0 || x + 1 == kDepT - 1) && (s_flags[g] & SDFDDGI_PROBE_ACTIVE)) {
            const int2 sa = border_source(y, x, kDepN), sb = border_source(y, x + 1, kDepN);
            a = m[sa.x * kDepT + sa.y];
            b = m[sb.x * kDepT + sb.y];
        } else {
            a = m[y * kDepT + x];
            b = m[y * kDepT + x + 1];
        }
        cur_d4[e] = make_float4(a.x, a.y, b.x, b.y);
    }
    if (tid < ng) P.cur_valid[p0 + tid] = (s_flags[tid] & SDFDDGI_PROBE_ACTIVE) ? 1 : P.prev_valid[p0 + tid];
}

template <bool BF16>
__global__ void __launch_bounds__(tc::kThreads, 2) gather_tc_kernel(const __grid_constant__ UpdateParams P) {
    gather_tc_body<BF16>(P, blockIdx.x);
}

// The merged launches of the batched form: one block per ray of every volume for the weight
// images, and each volume's gather CTAs after the earlier volumes'.
__device__ __forceinline__ int merged_part_tc(const uint32_t* begin, int n, uint32_t x) {
    int v = 0;
#pragma unroll
    for (int i = 1; i < kMaxMerged; ++i) v += (i < n && x >= begin[i]) ? 1 : 0;
    return v;
}

template <bool BF16>
__global__ void __launch_bounds__(256) pack_weights_merged_kernel(const __grid_constant__ MergedParams M) {
    const int v = merged_part_tc(M.dir_begin, M.n, blockIdx.x);
    pack_weights_body<BF16>(M.p[v], (int)(blockIdx.x - M.dir_begin[v]));
}

template <bool BF16>
__global__ void __launch_bounds__(tc::kThreads, 2) gather_tc_merged_kernel(const __grid_constant__ MergedParams M) {
    const int v = merged_part_tc(M.gather_begin, M.n, blockIdx.x);
    gather_tc_body<BF16>(M.p[v], (int)(blockIdx.x - M.gather_begin[v]));
}

bool gather_tc_supported(const UpdateParams& p) { return p.R % tc::kChunk == 0 && p.wimage != nullptr; }

size_t wimage_bytes(int R) { return (size_t)((R + tc::kChunk - 1) / tc::kChunk) * tc::Fmt<false>::kABytes; }

// dynamic shared memory of the gather: the two operand stages, reused by the epilogue's map
// staging (kG probes x 3 KiB)
template <bool BF16>
static size_t tc_smem() {
    using F = tc::Fmt<BF16>;
    const size_t epilogue = (size_t)tc::kG * (kIrrT * kIrrT * sizeof(float4) + kDepT * kDepT * sizeof(float2));
    return std::max<size_t>((size_t)tc::Stages<BF16>::value * (F::kABytes + F::kBBytes), epilogue);
}

cudaError_t prepare_gather_tc() {
    cudaError_t e = cudaFuncSetAttribute(gather_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tc_smem<false>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gather_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tc_smem<true>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gather_tc_merged_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tc_smem<false>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gather_tc_merged_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tc_smem<true>());
    return e;
}

template <bool BF16>
static cudaError_t launch_tc(const UpdateParams& p, cudaStream_t stream, bool pack, bool gather) {
    if (pack) pack_weights_kernel<BF16><<<p.R, 256, 0, stream>>>(p);
    if (gather) gather_tc_kernel<BF16><<<(p.P + tc::kG - 1) / tc::kG, tc::kThreads, tc_smem<BF16>(), stream>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_gather_tc(const UpdateParams& p, cudaStream_t stream, bool pack) {
    return p.blend_bf16 ? launch_tc<true>(p, stream, pack, true) : launch_tc<false>(p, stream, pack, true);
}

cudaError_t launch_pack_weights(const UpdateParams& p, cudaStream_t stream) {
    return p.blend_bf16 ? launch_tc<true>(p, stream, true, false) : launch_tc<false>(p, stream, true, false);
}

template <bool BF16>
static cudaError_t launch_tc_merged(const MergedParams& m, cudaStream_t stream, bool pack) {
    if (pack) pack_weights_merged_kernel<BF16><<<m.dir_begin[m.n], 256, 0, stream>>>(m);
    gather_tc_merged_kernel<BF16><<<m.gather_begin[m.n], tc::kThreads, tc_smem<BF16>(), stream>>>(m);
    return cudaGetLastError();
}

cudaError_t launch_gather_tc_merged(const MergedParams& m, cudaStream_t stream, bool pack) {
    return m.p[0].blend_bf16 ? launch_tc_merged<true>(m, stream, pack) : launch_tc_merged<false>(m, stream, pack);
}

}  // namespace sdfddgi
