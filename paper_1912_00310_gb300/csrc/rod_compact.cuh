// rod_compact.cuh -- pieces shared by the gradient kernels (k_adjoint.cu, k_tangent.cu): small
// FP32 vector helpers with explicit fused multiply-adds, and the compact shared-memory rod.
//
// Compact rod: one float4 per cell in cell order (x fastest, then y, then z), followed by one zero
// slot that stands for every neighbour beyond a free face.  Consecutive threads then read
// consecutive float4s; a ghost-padded layout of a thin rod (the b = 4 rod is two cells wide) uses
// only part of each row's banks and doubled the wavefronts of every neighbour load.
#pragma once

#include "physics.cuh"

namespace llg {
namespace grad {

__device__ __forceinline__ float3 zero3() { return make_float3(0.f, 0.f, 0.f); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b)
{
    return make_float3(fmaf(a.y, b.z, -a.z * b.y), fmaf(a.z, b.x, -a.x * b.z), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float dot3(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 scale3(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }

// Neighbour indices of a cell, in the order x-, x+, y-, y+, z-, z+; `zero` (the slot after the
// last cell) beyond a free face.
struct Nbr {
    int i[6];
};

__device__ __forceinline__ Nbr neighbours(int c, int nx, int ny, int nz, int zero)
{
    const int x = c % nx, y = (c / nx) % ny, z = c / (nx * ny), sxy = nx * ny;
    Nbr n;
    n.i[0] = x > 0 ? c - 1 : zero;
    n.i[1] = x < nx - 1 ? c + 1 : zero;
    n.i[2] = y > 0 ? c - nx : zero;
    n.i[3] = y < ny - 1 ? c + nx : zero;
    n.i[4] = z > 0 ? c - sxy : zero;
    n.i[5] = z < nz - 1 ? c + sxy : zero;
    return n;
}

// The neighbour sum in the order x-, x+, y-, y+, z-, z+ (every engine's order).
__device__ __forceinline__ float3 neighbour_sum(const float4 *A, const Nbr &n)
{
    float3 nb = add3(xyz(A[n.i[0]]), xyz(A[n.i[1]]));
    nb = add3(nb, xyz(A[n.i[2]]));
    nb = add3(nb, xyz(A[n.i[3]]));
    nb = add3(nb, xyz(A[n.i[4]]));
    return add3(nb, xyz(A[n.i[5]]));
}

}  // namespace grad
}  // namespace llg
