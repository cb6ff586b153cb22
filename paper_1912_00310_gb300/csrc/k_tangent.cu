// k_tangent.cu -- forward-mode (tangent) gradient of the sampled loop with respect to the
// calibration scale factors theta = (s_K, s_alpha, s_Ms), the second method of the pathwise
// gradient of llg_loop_area_grad (the first is the reverse-mode adjoint of k_adjoint.cu).
//
// With three parameters, carrying the three tangents dm/dtheta_j forward beside m costs one pass
// and no stored window: per cell and step the Heun map of Eq. 1 and its derivative
//   H   = c_ex N(m) + (c_an m_z + H_z) z + sigma xi       dH_j = dc_ex_j N(m) + c_ex N(dm_j)
//                                                              + (dc_an_j m_z + c_an dm_j,z) z + dsigma_j xi
//   c0  = m x H,  s0 = c0 + alpha m x c0                  ds0_j = dc0_j + dalpha_j m x c0
//                                                              + alpha (dm_j x c0 + m x dc0_j)
//   p   = m - a s0,  m~ = p / |p|                         dm~_j = (dp_j - m~ (m~.dp_j)) / |p|
//   (the same at m~ with the step's field H~ and the same thermal field)
//   q   = m - (a/2)(s0 + s1),  m' = q / |q|               dm'_j = (dq_j - m' (m'.dq_j)) / |q|
// with a = dt g1, g1 = g0/(1 + alpha^2), sigma ~ sqrt(alpha / Ms), c_ex ~ 1/Ms, c_an ~ K/Ms; the
// thermal normals xi are the pathwise constants (dsigma_j xi = (dsigma_j / sigma) h).  The primal
// uses the forward engines' exact arithmetic, so its samples -- and the loss -- are bitwise those
// of a forward run.  At each sample of the window the kernel writes the cell average of m_z and of
// the three dm_z/dtheta_j; the host forms dL/dtheta_j = sum_k (dL/dmbar_k) dmbar_k/dtheta_j.
//
// One CTA per rod and parameter (grid n_real x 3): CTA (r, j) recomputes rod r's primal, with the
// forward engines' arithmetic (every CTA of a rod holds bitwise the same m), and carries the tangent
// dm/dtheta_j; one or two cells per thread.  The rod sits in shared memory compactly, one float4
// per cell in cell order plus one zero slot that stands for every neighbour beyond a free face (each
// thread keeps its six neighbour indices): consecutive threads read consecutive float4s, without
// the bank conflicts of a ghost-padded layout whose rows are only partly used.  Four such arrays:
// m and dm/dtheta_j for the state and for the predictor (64 bytes a cell); rods of at most 1408
// cells, the b = 2 rod included.
#include <cmath>

#include "llg_internal.h"
#include "physics.cuh"
#include "reduce.cuh"
#include "rod_compact.cuh"
#include "sweep32.cuh"

namespace llg {
namespace {

using grad::Nbr;
using grad::neighbours;
__device__ __forceinline__ float3 zr3() { return grad::zero3(); }
__device__ __forceinline__ float3 crs(float3 a, float3 b) { return grad::cross3(a, b); }
__device__ __forceinline__ float dt3(float3 a, float3 b) { return grad::dot3(a, b); }
__device__ __forceinline__ float3 sc3(float s, float3 a) { return grad::scale3(s, a); }
__device__ __forceinline__ float3 sb3(float3 a, float3 b) { return grad::sub3(a, b); }

// Derivatives of the simulation coefficients with respect to theta_j at the current scale.
struct TanCoeffs {
    float dcex[3], dcan[3], dalpha[3], da[3], rsig[3];  // rsig = dsigma_j / sigma
};

struct TanParams {
    KParams p;
    TanCoeffs d;
    long long step0;
    int n_steps;
    long long k_first;  // first sample number of the window
    int n_k;            // samples in the window
};

// CPT cells per thread (cell c + k * blockDim.x, k < CPT); MAXT the largest CTA of the instance;
// SHAPE the sweep shape with 32-bit bookkeeping (0 triangle, 1 cosine), or -1 for the 64-bit sweep
// of any period.  Each thread's dependent chain is the primal plus one tangent.
template <bool AX, int CPT, int MAXT, int SHAPE>
__global__ void __launch_bounds__(MAXT, MAXT <= 256 ? 1 : 0) tangent_kernel(TanParams tp, float *__restrict__ m_glob,
                                                      float *__restrict__ samples, float *__restrict__ dsamples,
                                                      int *__restrict__ status)
{
    extern __shared__ float4 sm4[];
    const KParams &p = tp.p;
    const TanCoeffs &d = tp.d;
    const int ncell = p.ncells;
    const int S = ncell + 1;  // cells and the zero slot
    // state m, its tangent, predictor, its tangent
    float4 *M = sm4, *Md = sm4 + S, *P = sm4 + 2 * S, *Pd = sm4 + 3 * S;
    const int rod = blockIdx.x, j = blockIdx.y;  // j: the parameter whose tangent this CTA carries
    for (int i = threadIdx.x; i < 4 * S; i += blockDim.x) sm4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    const uint32_t real = p.real0 + (uint32_t)rod;
    const PhiloxKeys keys = philox_keys(p.seed, real);  // the rod's round keys, formed once
    // this CTA's coefficient derivatives (a uniform index into the parameter block)
    const float dcex = d.dcex[j], dcan = d.dcan[j], dalpha = d.dalpha[j], da = d.da[j], rsig = d.rsig[j];
    Nbr nb[CPT];
    float3 m[CPT], dm[CPT], u[CPT], hpre[CPT];  // the tangent starts at zero: m0 is fixed
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        const int c = threadIdx.x + k * blockDim.x;
        nb[k] = neighbours(0, p.nx, p.ny, p.nz, ncell);
        m[k] = dm[k] = hpre[k] = zr3();
        u[k] = make_float3(0.f, 0.f, 1.f);
        if (c < ncell) {
            nb[k] = neighbours(c, p.nx, p.ny, p.nz, ncell);
            const float *src = m_glob + ((size_t)rod * ncell + c) * 3;
            m[k] = make_float3(src[0], src[1], src[2]);
            if (AX) u[k] = xyz(__ldg(p.axis + (size_t)rod * ncell + c));
            // thermal field of the next step, drawn before the step's last barrier
            hpre[k] = thermal_field(keys, (uint32_t)c, (unsigned long long)tp.step0, p.sigma);
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < CPT; ++k)
        if (threadIdx.x + k * blockDim.x < ncell) M[threadIdx.x + k * blockDim.x] = pad4(m[k]);
    __syncthreads();
    const float alpha = p.alpha, a = -p.neg_dt_g1;
    const int lane = threadIdx.x & 31;
    typename SweepSel<SHAPE>::type field;
    field.init(tp.step0, p);
    float Hn = field.value();
    // steps to the next sample (32-bit countdown; the host keeps sample_every below 2^31)
    const long long se = p.sample_every;
    long long k_next = se > 0 ? tp.step0 / se + 1 : 0;
    int to_sample = se > 0 ? (int)(k_next * se - tp.step0) : -1;
    // the field-tangent and torque-tangent of one half step: dH = dc_ex N + c_ex Nd + rsig h +
    // the anisotropy tangent; ds = dc + dalpha m x c + alpha (dm x c + m x dc), dc = dm x H + m x dH
    auto half_tan = [&](float3 mm, float3 dmm, float3 N, float3 Nd, float3 h, float3 H, float3 uu) {
        float3 dH = add3(sc3(dcex, N), sc3(p.c_ex, Nd));
        dH = add3(dH, sc3(rsig, h));
        if constexpr (AX) {
            const float mu = dt3(mm, uu), dmu = dt3(dmm, uu);
            dH = add3(dH, sc3(fmaf(dcan, mu, p.c_an * dmu), uu));
        } else {
            dH.z = fmaf(dcan, mm.z, fmaf(p.c_an, dmm.z, dH.z));
        }
        const float3 cc = crs(mm, H);
        const float3 dc = add3(crs(dmm, H), crs(mm, dH));
        return add3(add3(dc, sc3(dalpha, crs(mm, cc))), sc3(alpha, add3(crs(dmm, cc), crs(mm, dc))));
    };
    for (int s = 0; s < tp.n_steps; ++s) {
        const unsigned long long n = (unsigned long long)(tp.step0 + s);
        field.inc();
        const float Hn1 = field.value();
        float3 acc[CPT], dacc[CPT], t[CPT], dtt[CPT];
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            acc[k] = dacc[k] = t[k] = dtt[k] = zr3();
            const int c = threadIdx.x + k * blockDim.x;
            if (c >= ncell) continue;
            const float3 N = grad::neighbour_sum(M, nb[k]), Nd = grad::neighbour_sum(Md, nb[k]);
            const float3 H = effective_field_sel<AX>(N, m[k], hpre[k], p, Hn, u[k]);
            const float3 s0 = llg_torque(m[k], H, alpha);
            const float3 ds0 = half_tan(m[k], dm[k], N, Nd, hpre[k], H, u[k]);
            const float3 pv = axpy(p.neg_dt_g1, s0, m[k]);
            const float r = rsqrtf(fmaf(pv.x, pv.x, fmaf(pv.y, pv.y, pv.z * pv.z)));
            t[k] = make_float3(pv.x * r, pv.y * r, pv.z * r);  // normalised(pv), the engines' arithmetic
            acc[k] = axpy(p.neg_hdt_g1, s0, m[k]);
            const float3 dp = sb3(sb3(dm[k], sc3(da, s0)), sc3(a, ds0));
            dtt[k] = sc3(r, sb3(dp, sc3(dt3(t[k], dp), t[k])));
            dacc[k] = sb3(sb3(dm[k], sc3(0.5f * da, s0)), sc3(0.5f * a, ds0));
            Pd[c] = pad4(dtt[k]);
            P[c] = pad4(t[k]);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            const int c = threadIdx.x + k * blockDim.x;
            if (c >= ncell) continue;
            const float3 N = grad::neighbour_sum(P, nb[k]), Nd = grad::neighbour_sum(Pd, nb[k]);
            const float3 H = effective_field_sel<AX>(N, t[k], hpre[k], p, Hn1, u[k]);
            const float3 s1 = llg_torque(t[k], H, alpha);
            const float3 ds1 = half_tan(t[k], dtt[k], N, Nd, hpre[k], H, u[k]);
            const float3 qv = axpy(p.neg_hdt_g1, s1, acc[k]);
            const float r = rsqrtf(fmaf(qv.x, qv.x, fmaf(qv.y, qv.y, qv.z * qv.z)));
            m[k] = make_float3(qv.x * r, qv.y * r, qv.z * r);
            const float3 dq = sb3(sb3(dacc[k], sc3(0.5f * da, s1)), sc3(0.5f * a, ds1));
            dm[k] = sc3(r, sb3(dq, sc3(dt3(m[k], dq), m[k])));
            Md[c] = pad4(dm[k]);
            M[c] = pad4(m[k]);
            hpre[k] = thermal_field(keys, (uint32_t)c, n + 1, p.sigma);
        }
        __syncthreads();
        Hn = Hn1;
        if (--to_sample == 0) {
            to_sample = (int)se;
            const long long kk = k_next++ - tp.k_first;
            if (kk >= 0 && kk < tp.n_k && threadIdx.x < 32) {
                // the first warp: the canonical reduction of m_z (every engine's) and of the
                // tangent's z component
                float part = 0.f, pd = 0.f;
                for (int cc = lane; cc < ncell; cc += 32) {
                    pd += Md[cc].z;
                    part += M[cc].z;
                }
                const float dmean = warp_cell_mean(pd, ncell);
                const float mean = warp_cell_mean(part, ncell);
                if (lane == 0) {
                    dsamples[((size_t)rod * tp.n_k + kk) * 3 + j] = dmean;
                    if (j == 0) {
                        samples[(size_t)rod * tp.n_k + kk] = mean;
                        if (!isfinite(mean)) atomicOr(status, 1);
                    }
                }
            }
        }
    }
}

}  // namespace

bool tangent_supported(const KParams &p, int dev)
{
    int smem_optin = 0;
    if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
    return p.periodic == 0 && p.ncells <= 1408 && 4 * (size_t)(p.ncells + 1) * sizeof(float4) <= (size_t)smem_optin;
}

cudaError_t tangent_forward(const KParams &p, const double dcoef[15], int n_real, long long step0, long long n_steps,
                            long long k_first, int n_k, float *m_work, float *samples, float *dsamples, int *status,
                            cudaStream_t st)
{
    if (n_steps < 0 || n_steps > 0x7fffffffLL || n_k < 1 || n_real < 1 || p.sample_every >= (1LL << 31))
        return cudaErrorInvalidValue;
    TanParams tp;
    tp.p = p;
    for (int j = 0; j < 3; ++j) {
        tp.d.dcex[j] = (float)dcoef[j];
        tp.d.dcan[j] = (float)dcoef[3 + j];
        tp.d.dalpha[j] = (float)dcoef[6 + j];
        tp.d.da[j] = (float)dcoef[9 + j];
        tp.d.rsig[j] = (float)dcoef[12 + j];
    }
    tp.step0 = step0;
    tp.n_steps = (int)n_steps;
    tp.k_first = k_first;
    tp.n_k = n_k;
    const size_t smem = 4 * (size_t)(p.ncells + 1) * sizeof(float4);
    const dim3 grid((unsigned)n_real, 3);
    auto go = [&](auto kern, int threads) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, threads, smem, st>>>(tp, m_work, samples, dsamples, status);
        return cudaGetLastError();
    };
    const int t1 = (p.ncells + 31) / 32 * 32;             // one cell per thread
    const int t2 = ((p.ncells + 1) / 2 + 31) / 32 * 32;   // two cells per thread
    // the sweep shape at compile time where its period fits 32 bits
    const int shape = sweep_fits_32(p) ? (p.shape == 1 ? 1 : 0) : -1;
    auto by_shape = [&](auto k0, auto k1, auto kg, int threads) {
        return shape == 0 ? go(k0, threads) : shape == 1 ? go(k1, threads) : go(kg, threads);
    };
#define LLG_TAN(AXV, C, T) tangent_kernel<AXV, C, T, 0>, tangent_kernel<AXV, C, T, 1>, tangent_kernel<AXV, C, T, -1>
    if (t1 <= 192) return p.axis ? by_shape(LLG_TAN(true, 1, 192), t1) : by_shape(LLG_TAN(false, 1, 192), t1);
    if (t1 <= 768) return p.axis ? by_shape(LLG_TAN(true, 1, 768), t1) : by_shape(LLG_TAN(false, 1, 768), t1);
    if (t2 <= 704) return p.axis ? by_shape(LLG_TAN(true, 2, 704), t2) : by_shape(LLG_TAN(false, 2, 704), t2);
#undef LLG_TAN
    return cudaErrorInvalidValue;
}

}  // namespace llg
