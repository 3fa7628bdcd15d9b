// volume.cu -- the device SDF store.
//
// Besides the plain [z][y][x] array, the scene keeps the signed-distance values in an
// "xy-quad" layout: quad (x, y, z) holds the four values (x, y), (x+1, y), (x, y+1),
// (x+1, y+1) of slice z. A trilinear sample then reads its eight corners with two vector
// loads (slices z and z+1) instead of eight scalar loads, which is what bounds the
// sphere-trace kernels. The quads are stored in z-pairs, [z/2][y][x][z%2]: the quads of
// slices 2m and 2m+1 of one (x, y) sit side by side, so a sample in a cell of even padded z
// finds both of its quads in one 32-byte sector (a quarter fewer sectors per sample on
// average). The store has a one-voxel apron on every side holding copies of the edge
// values (clamp to edge), so that the traces index cells -1 .. n-1 without clamping:
// lerp(a, a, f) = a exactly, so the samples equal those of the clamped rule. The values are
// the same float32 / binary16 numbers, only replicated, so results are unchanged.
#include <algorithm>

#include "internal.h"

namespace sdfddgi {

template <typename T, typename Q>
__global__ void build_quads_kernel(const T* __restrict__ sdf, Q* __restrict__ quads, int nx, int ny, int nz, int qx) {
    const int qy = ny + 2, qz = nz + 2;  // padded extents
    const size_t n = (size_t)qx * qy * qz;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int X = (int)(i % qx), Y = (int)((i / qx) % qy), Z = (int)(i / ((size_t)qx * qy));
        // padded coordinate P holds voxel clamp(P - 1, 0, n - 1)
        const int x0 = min(max(X - 1, 0), nx - 1), x1 = min(X, nx - 1);
        const int y0 = min(max(Y - 1, 0), ny - 1), y1 = min(Y, ny - 1);
        const size_t z = (size_t)min(max(Z - 1, 0), nz - 1);
        const size_t r0 = (z * ny + y0) * nx, r1 = (z * ny + y1) * nx;
        Q q;
        T* e = reinterpret_cast<T*>(&q);
        e[0] = sdf[r0 + x0];
        e[1] = sdf[r0 + x1];
        e[2] = sdf[r1 + x0];
        e[3] = sdf[r1 + x1];
        quads[quad_index((size_t)X, (size_t)Y, (size_t)Z, (size_t)qx, (size_t)qy)] = q;
    }
}

size_t quad_bytes(int dtype, const int dims[3]) {
    const size_t pairs = ((size_t)dims[2] + 3) / 2;
    return 2 * pairs * (size_t)padded_qx(dims[0]) * ((size_t)dims[1] + 2) * (dtype == SDFDDGI_F16 ? 8 : 16);
}

cudaError_t build_quads(const void* sdf, void* quads, int dtype, const int dims[3], cudaStream_t stream) {
    const size_t n = (size_t)padded_qx(dims[0]) * ((size_t)dims[1] + 2) * ((size_t)dims[2] + 2);
    const int threads = 256;
    const int blocks = (int)std::min<size_t>((n + threads - 1) / threads, 148 * 64);
    if (dtype == SDFDDGI_F16)
        build_quads_kernel<__half, uint2><<<blocks, threads, 0, stream>>>(
            static_cast<const __half*>(sdf), static_cast<uint2*>(quads), dims[0], dims[1], dims[2], padded_qx(dims[0]));
    else
        build_quads_kernel<float, float4><<<blocks, threads, 0, stream>>>(
            static_cast<const float*>(sdf), static_cast<float4*>(quads), dims[0], dims[1], dims[2], padded_qx(dims[0]));
    return cudaGetLastError();
}

}  // namespace sdfddgi
