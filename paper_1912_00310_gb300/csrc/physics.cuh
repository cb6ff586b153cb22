// physics.cuh -- device arithmetic of one stochastic Heun step of Eq. 1 (FP32), shared by every
// engine of the library: the Philox4x32-10 noise source, the Box-Muller thermal normals, the
// effective field (easy axis z or a per-cell axis), the LLG torque, the renormalisation and the
// field sweep (triangle or sinusoid) evaluated from an integer phase.
//
// Eq. 1 for the unit vector m = M/Ms:  dm/dt = -g1 m x H - alpha g1 m x (m x H),
// g1 = mu0 ge / (1 + alpha^2).  Writing s(m, H) = m x H + alpha m x (m x H), the right-hand side
// is f = -g1 s, so the Heun predictor is m~ = normalise(m - dt g1 s(m, H_n)) and the corrector
// m' = normalise(m - (dt g1 / 2) (s(m, H_n) + s(m~, H~_n+1))).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "llg_internal.h"

namespace llg {

// ------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two 32x32->64 multiplies,
// a half swap and a key xor, the key bumped by the Weyl constants between rounds.
// ------------------------------------------------------------------------------------------
constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox_round(uint4 c, uint32_t k0, uint32_t k1)
{
    const unsigned long long p0 = (unsigned long long)kPhiloxM0 * c.x;
    const unsigned long long p1 = (unsigned long long)kPhiloxM1 * c.z;
    return make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1,
                      (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
}

// Key bumped round by round (for keys that differ between the cells of a thread).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += kPhiloxW0;
            k1 += kPhiloxW1;
        }
        c = philox_round(c, k0, k1);
    }
    return c;
}

// The ten round keys of one key, computed once (for a key shared by all cells of a CTA, where
// they stay in uniform registers across the step loop).
struct PhiloxKeys {
    uint32_t k0[10], k1[10];
};

__device__ __forceinline__ PhiloxKeys philox_keys(uint32_t k0, uint32_t k1)
{
    PhiloxKeys K;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        K.k0[r] = k0 + (uint32_t)r * kPhiloxW0;
        K.k1[r] = k1 + (uint32_t)r * kPhiloxW1;
    }
    return K;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys &K)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) c = philox_round(c, K.k0[r], K.k1[r]);
    return c;
}

// Uniform in (0,1): (floor(x / 256) + 1/2) * 2^-24, exact in FP32.
__device__ __forceinline__ float uniform24(uint32_t x)
{
    return fmaf(__uint2float_rn(x >> 8), 0x1p-24f, 0x1p-25f);
}

// Thermal field from the four Philox words of (seed, realisation, cell, step): sigma times
// three standard normals from Box-Muller on (u0, u1) and (u2, u3).  The angle is taken as
// 2 pi (u - 1/2), inside the accurate range of the hardware sine, which negates both members of
// each pair.
__device__ __forceinline__ float3 box_muller3(uint4 x, float sigma)
{
    const float u0 = uniform24(x.x), u1 = uniform24(x.y);
    const float u2 = uniform24(x.z), u3 = uniform24(x.w);
    const float kNeg2Ln2 = -1.3862943611198906f;  // -2 ln 2 : -2 ln u = -2 ln2 log2 u
    const float v0 = fmaxf(kNeg2Ln2 * __log2f(u0), 1e-30f);
    const float v2 = fmaxf(kNeg2Ln2 * __log2f(u2), 1e-30f);
    const float r0 = -sigma * v0 * rsqrtf(v0);
    const float r2 = -sigma * v2 * rsqrtf(v2);
    const float kTwoPi = 6.283185307179586f;
    float s1, c1;
    __sincosf(kTwoPi * (u1 - 0.5f), &s1, &c1);
    const float c3 = __cosf(kTwoPi * (u3 - 0.5f));
    return make_float3(r0 * c1, r0 * s1, r2 * c3);
}

__device__ __forceinline__ uint4 noise_counter(uint32_t cell, unsigned long long step)
{
    return make_uint4(cell, (uint32_t)step, (uint32_t)(step >> 32), 0u);
}

__device__ __forceinline__ float3 thermal_field(uint32_t seed, uint32_t real, uint32_t cell,
                                                unsigned long long step, float sigma)
{
    return box_muller3(philox4x32_10(noise_counter(cell, step), seed, real), sigma);
}

__device__ __forceinline__ float3 thermal_field(const PhiloxKeys &K, uint32_t cell,
                                                unsigned long long step, float sigma)
{
    return box_muller3(philox4x32_10(noise_counter(cell, step), K), sigma);
}

// s(m, H) = m x H + alpha m x (m x H)
__device__ __forceinline__ float3 llg_torque(float3 m, float3 H, float alpha)
{
    const float ax = fmaf(m.y, H.z, -m.z * H.y);
    const float ay = fmaf(m.z, H.x, -m.x * H.z);
    const float az = fmaf(m.x, H.y, -m.y * H.x);
    const float bx = fmaf(m.y, az, -m.z * ay);
    const float by = fmaf(m.z, ax, -m.x * az);
    const float bz = fmaf(m.x, ay, -m.y * ax);
    return make_float3(fmaf(alpha, bx, ax), fmaf(alpha, by, ay), fmaf(alpha, bz, az));
}

__device__ __forceinline__ float3 normalised(float3 v)
{
    const float r = rsqrtf(fmaf(v.x, v.x, fmaf(v.y, v.y, v.z * v.z)));
    return make_float3(v.x * r, v.y * r, v.z * r);
}

__device__ __forceinline__ float3 axpy(float a, float3 x, float3 y)
{
    return make_float3(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z));
}

__device__ __forceinline__ float3 add3(float3 a, float3 b)
{
    return make_float3(a.x + b.x, a.y + b.y, a.z + b.z);
}

__device__ __forceinline__ float3 xyz(float4 v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float4 pad4(float3 v) { return make_float4(v.x, v.y, v.z, 0.f); }

// Effective field from the neighbour sum nb = sum_j m_j: c_ex nb + h_th + (c_an m_z + Hz) z.
__device__ __forceinline__ float3 effective_field(float3 nb, float3 m, float3 hth, float c_ex,
                                                  float c_an, float Hz)
{
    return make_float3(fmaf(c_ex, nb.x, hth.x), fmaf(c_ex, nb.y, hth.y),
                       fmaf(c_ex, nb.z, fmaf(c_an, m.z, hth.z + Hz)));
}

// Effective field with a per-cell easy axis u (the dispersed-axis mode):
// c_ex nb + h_th + c_an (m.u) u + Hz z.  A separate form, not effective_field with u = z: the
// z-axis form fuses c_an m_z into one rounding, which keeps the default path unchanged.
__device__ __forceinline__ float3 effective_field_axis(float3 nb, float3 m, float3 hth, float c_ex,
                                                       float c_an, float Hz, float3 u)
{
    const float a = c_an * fmaf(m.x, u.x, fmaf(m.y, u.y, m.z * u.z));
    return make_float3(fmaf(c_ex, nb.x, fmaf(a, u.x, hth.x)), fmaf(c_ex, nb.y, fmaf(a, u.y, hth.y)),
                       fmaf(c_ex, nb.z, fmaf(a, u.z, hth.z + Hz)));
}

// The effective field of the z-axis mode (AX = false; u unused) or of the dispersed-axis mode.
template <bool AX>
__device__ __forceinline__ float3 effective_field_sel(float3 nb, float3 m, float3 hth, const KParams &p,
                                                      float Hz, float3 u)
{
    if constexpr (AX)
        return effective_field_axis(nb, m, hth, p.c_ex, p.c_an, Hz, u);
    else
        return effective_field(nb, m, hth, p.c_ex, p.c_an, Hz);
}

// Easy axis of one cell of one realisation: uniform over the solid angle of the cone of
// half-angle theta_max about z, drawn from Philox4x32-10 with key (seed, realisation) and counter
// (cell, 0, 0, 1) (the thermal draws use tag word 0).  w_max = 1 - cos(theta_max); on a
// spherical cap 1 - cos(theta) is uniform on [0, w_max] and the azimuth is uniform.
__device__ __forceinline__ float3 easy_axis(uint32_t seed, uint32_t real, uint32_t cell, float w_max)
{
    const uint4 x = philox4x32_10(make_uint4(cell, 0u, 0u, 1u), seed, real);
    const float w = w_max * uniform24(x.x);
    float sp, cp;
    sincospif(2.0f * uniform24(x.y), &sp, &cp);
    const float st = sqrtf(w * (2.0f - w));
    return make_float3(st * cp, st * sp, 1.0f - w);
}

// Zeeman field along z at step n, tracked by its phase (n mod period) in steps:
//   shape 0: triangle, H0 + slope * tri(ph) with tri = ph for ph <= n_half, period - ph after
//            (period = 2 n_half; n_half = 0 holds H0);
//   shape 1: cosine, amp * cos(2 pi ph / period) (the paper's sinusoidal field with its phase
//            chosen to start at +amp).
// (a, c) = (H0, slope) for the triangle, (amp, unused) for the cosine; period 0 holds H0.  The
// triangle coordinate is min(ph, period - ph) since its period is 2 n_half.  SHAPE = 0 or 1 fixes
// the shape at compile time (the hot resident kernel, whose registers are all in use across the
// step loop, instantiates one per shape); -1 branches on p.shape.
template <int SHAPE>
struct SweepOf {
    long long ph, period;
    float a, c;
    int shape;

    __host__ __device__ __forceinline__ void init(long long n, const KParams &p)
    {
        if constexpr (SHAPE == 0) {
            period = 2 * p.n_half;
            a = p.H0;
        } else if constexpr (SHAPE == 1) {
            period = p.period;
            a = p.amp;
        } else {
            period = p.shape == 1 ? p.period : 2 * p.n_half;
            a = p.shape == 1 ? p.amp : p.H0;
        }
        shape = p.shape;
        c = p.slope;
        ph = period > 0 ? n % period : 0;
    }
    __device__ __forceinline__ float value() const
    {
        if (SHAPE == 1 || (SHAPE < 0 && shape == 1)) return a * cospif(2.0f * ((float)ph / (float)period));
        const long long tri = min(ph, period - ph);
        return fmaf(c, (float)tri, a);
    }
    __host__ __device__ __forceinline__ void inc()
    {
        if (period > 0 && ++ph == period) ph = 0;
    }
    __host__ __device__ __forceinline__ void dec()
    {
        if (period > 0) ph = (ph == 0 ? period : ph) - 1;
    }
};
using Sweep = SweepOf<-1>;

}  // namespace llg
