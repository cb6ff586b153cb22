// sweep32.cuh -- the Zeeman sweep of physics.cuh's SweepOf with the phase in 32 bits, for kernels
// specialised on the sweep shape (SHAPE 0 triangle, 1 cosine).  The host uses these instances
// only for periods below 2^31 steps.  Same values as SweepOf: the triangle coordinate
// min(ph, period - ph) and the cosine argument convert the same integers to float.
#pragma once

#include "physics.cuh"

namespace llg {

template <int SHAPE>
struct Sweep32 {
    int ph, period;
    float a, c;
    __device__ __forceinline__ void init(long long n, const KParams &p)
    {
        long long per;
        if constexpr (SHAPE == 0) {
            per = 2 * p.n_half;
            a = p.H0;
        } else {
            per = p.period;
            a = p.amp;
        }
        c = p.slope;
        period = (int)per;
        ph = per > 0 ? (int)(n % per) : 0;
    }
    __device__ __forceinline__ float value() const
    {
        if constexpr (SHAPE == 1) return a * cospif(2.0f * ((float)ph / (float)period));
        const int tri = min(ph, period - ph);
        return fmaf(c, (float)tri, a);
    }
    __device__ __forceinline__ void inc()
    {
        if (period > 0 && ++ph == period) ph = 0;
    }
    __device__ __forceinline__ void dec()
    {
        if (period > 0) ph = (ph == 0 ? period : ph) - 1;
    }
};

// SHAPE -1: the 64-bit sweep of physics.cuh (any period, shape at run time).
template <int SHAPE>
struct SweepSel {
    using type = Sweep32<SHAPE>;
};
template <>
struct SweepSel<-1> {
    using type = Sweep;
};

// Whether the 32-bit instances cover a sweep: its period (or the held field's zero) below 2^31.
inline bool sweep_fits_32(const KParams &p)
{
    const long long per = p.shape == 1 ? p.period : 2 * p.n_half;
    return per >= 0 && per < (1LL << 31);
}

}  // namespace llg
