// denoiser.h -- layout and index helpers of the probe denoiser shared by its CUDA-core
// (denoiser.cu) and tensor-core (denoiser_tc.cu) kernels.
#pragma once

#include "internal.h"

namespace sdfddgi {
namespace dn {

constexpr int kCin = 35, kC1 = 64, kC2 = 48, kCout = 3;  // channels of the input and the three layers
constexpr int kN = 6;                                    // interior texels per side
constexpr int kTex = 64;                                 // texels of the 8 x 8 bordered grid
constexpr int kInt = kN * kN;                            // interior texels
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + 9 * kCin * kC1;
constexpr int kOffW2 = kOffB1 + kC1, kOffB2 = kOffW2 + 9 * kC1 * kC2;
constexpr int kOffW3 = kOffB2 + kC2, kOffB3 = kOffW3 + 9 * kC2 * kCout;
constexpr int kParams = kOffB3 + kCout;
static_assert(kParams == SDFDDGI_DENOISER_PARAMS, "parameter layout");
constexpr float kBeta1 = 0.9f, kBeta2 = 0.999f, kEps = 1e-8f;

struct MapsView {
    int dims[3];
    int per_grid;  // probes per grid
    int P;         // probes in all
    const float4* irr;
    const float2* depth;
    const uint8_t* valid;
    const sdfddgi_probe_state* states;
};

__device__ __forceinline__ bool probe_active(const MapsView& m, int p) {
    return !m.states || (m.states[p].flags & 1u);
}

// The probe itself, then its -x, +x, -y, +y, -z, +z neighbours within its grid; a
// neighbour outside the grid or without history is replaced by the probe.
__device__ __forceinline__ void neighbour_sources(const MapsView& m, int p, int src[7]) {
    const int nx = m.dims[0], ny = m.dims[1], nz = m.dims[2];
    const int g0 = p - p % m.per_grid, l = p - g0;
    const int x = l % nx, y = (l / nx) % ny, z = l / (nx * ny);
    src[0] = p;
    const int c[6][3] = {{x - 1, y, z}, {x + 1, y, z}, {x, y - 1, z}, {x, y + 1, z}, {x, y, z - 1}, {x, y, z + 1}};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const bool in = c[k][0] >= 0 && c[k][0] < nx && c[k][1] >= 0 && c[k][1] < ny && c[k][2] >= 0 && c[k][2] < nz;
        const int q = in ? g0 + (c[k][2] * ny + c[k][1]) * nx + c[k][0] : p;
        src[k + 1] = (in && m.valid[q]) ? q : p;
    }
}

// texel (r, c) of the bordered grid is r * 8 + c; interior texel q = (r - 1) * 6 + (c - 1)
__host__ __device__ constexpr int interior_texel(int q) { return (1 + q / kN) * 8 + 1 + q % kN; }
__host__ __device__ constexpr int interior_index(int t) { return ((t >> 3) - 1) * kN + (t & 7) - 1; }
// tap k = (dy + 1) * 3 + (dx + 1) reads texel t + dy * 8 + dx
__host__ __device__ constexpr int tap_offset(int k) { return (k / 3 - 1) * 8 + (k % 3 - 1); }

// The texel a border texel copies under the octahedral border fixup (Sec. 3.3; interior
// n = 6): top/bottom rows mirror across the vertical axis, left/right columns across the
// horizontal axis, corners take the opposite interior corner. Interior texels map to
// themselves.
__host__ __device__ inline int border_source(int t) {
    const int r = t >> 3, c = t & 7, n = kN;
    int sr = r, sc = c;
    if (r == 0 && c == 0) sr = n, sc = n;
    else if (r == 0 && c == n + 1) sr = n, sc = 1;
    else if (r == n + 1 && c == 0) sr = 1, sc = n;
    else if (r == n + 1 && c == n + 1) sr = 1, sc = 1;
    else if (r == 0) sr = 1, sc = n + 1 - c;
    else if (r == n + 1) sr = n, sc = n + 1 - c;
    else if (c == 0) sr = n + 1 - r, sc = 1;
    else if (c == n + 1) sr = n + 1 - r, sc = n;
    return sr * 8 + sc;
}

// tensor-core inference (denoiser_tc.cu)
struct TcState {
    void* wimg = nullptr;      // the three layers' weights as shared-memory operand images (bf16)
    size_t wimg_bytes = 0;
    uint32_t* status = nullptr;  // device word; bit 1: a bounded wait gave up (sticky)
    int sms = 0;
};
cudaError_t tc_create(TcState& s);
void tc_destroy(TcState& s);
// builds the weight images from the kernels' weight copy `use` (bf16-rounded weights, biases)
cudaError_t tc_prepare(TcState& s, const float* use, cudaStream_t st);
// feat: work space of P * 64 * 16 bytes for the feature texels; out may be m.irr (in place)
cudaError_t tc_forward(TcState& s, const MapsView& m, float depth_scale, const float* use, void* feat, float4* out,
                       cudaStream_t st);

}  // namespace dn
}  // namespace sdfddgi
