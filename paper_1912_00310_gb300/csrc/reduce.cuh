// reduce.cuh -- the cell average of m_z used for every M(H) sample (the paragraph defining m_H).
// One warp per realisation: lane l accumulates cells l, l+32, l+64, ... in increasing order in
// FP32, then a butterfly of xor-shuffles with offsets 16, 8, 4, 2, 1; lane 0's total divided by
// the cell count is the sample.  Every engine uses this order, so the samples of two engines that
// hold bitwise-equal states are bitwise equal.
#pragma once

#include <cuda_runtime.h>

namespace llg {

__device__ __forceinline__ float warp_cell_mean(float part, int ncells)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    return part / (float)ncells;
}

}  // namespace llg
