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
// One CTA per rod, three threads per cell (one per tangent), the rod in shared memory with a zero
// ghost layer: the state m and the three tangents in four float4 arrays, the same for the
// predictor (64 bytes a cell and buffer); rods of at most 256 cells.
#include <cmath>

#include "llg_internal.h"
#include "physics.cuh"
#include "reduce.cuh"

namespace llg {
namespace {

__device__ __forceinline__ float3 zr3() { return make_float3(0.f, 0.f, 0.f); }
__device__ __forceinline__ float3 crs(float3 a, float3 b)
{
    return make_float3(fmaf(a.y, b.z, -a.z * b.y), fmaf(a.z, b.x, -a.x * b.z), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float dt3(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 sc3(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float3 sb3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }

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

__device__ __forceinline__ float3 nbr(const float4 *A, int q, int sy, int sz)
{
    float3 nb = add3(xyz(A[q - 1]), xyz(A[q + 1]));
    nb = add3(nb, xyz(A[q - sy]));
    nb = add3(nb, xyz(A[q + sy]));
    nb = add3(nb, xyz(A[q - sz]));
    return add3(nb, xyz(A[q + sz]));
}

// Three groups of warps per rod: group j carries the tangent dm/dtheta_j (threads g*TPG ..
// g*TPG + TPG - 1, TPG = the rod's cells rounded up to a warp), and every group recomputes the
// primal with the same arithmetic (so all three hold bitwise the same m); group 0 writes the
// primal state to shared memory, group j its tangent.  Each thread's dependent chain is the
// primal plus one tangent, and a rod has three times the warps to hide latency.
// MAXT: the largest CTA of the instance (3 x 256 for rods up to 256 cells; 3 x 64 = 192 for the
// smallest).
template <bool AX, int MAXT>
__global__ void __launch_bounds__(MAXT) tangent_kernel(TanParams tp, float *__restrict__ m_glob,
                                                      float *__restrict__ samples, float *__restrict__ dsamples,
                                                      int *__restrict__ status)
{
    extern __shared__ float4 sm4[];
    const KParams &p = tp.p;
    const TanCoeffs &d = tp.d;
    const int px = p.nx + 2, py = p.ny + 2;
    const int sy = px, sz = px * py;
    const int rod_pad = sz * (p.nz + 2);
    // state and predictor, each as m and the three tangents
    float4 *M = sm4, *P = sm4 + 4 * rod_pad;
    const int rod = blockIdx.x;
    const int ncell = p.ncells;
    const int tpg = blockDim.x / 3;            // threads per group (a multiple of 32)
    const int grp = threadIdx.x / tpg;         // the tangent this thread carries (warp-uniform)
    const int c = threadIdx.x - grp * tpg;
    const bool act = c < ncell;
    for (int i = threadIdx.x; i < 8 * rod_pad; i += blockDim.x) sm4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    int q = 0;
    if (act) {
        const int x = c % p.nx, y = (c / p.nx) % p.ny, z = c / (p.nx * p.ny);
        q = (x + 1) + sy * (y + 1) + sz * (z + 1);
    }
    const uint32_t real = p.real0 + (uint32_t)rod;
    // this group's coefficient derivatives (a uniform index into the parameter block)
    const float dcex = d.dcex[grp], dcan = d.dcan[grp], dalpha = d.dalpha[grp], da = d.da[grp],
                rsig = d.rsig[grp];
    float4 *Md = M + (grp + 1) * rod_pad, *Pd = P + (grp + 1) * rod_pad;
    float3 m = zr3(), dm = zr3();  // the tangent starts at zero: m0 is fixed
    if (act) m = make_float3(m_glob[((size_t)rod * ncell + c) * 3], m_glob[((size_t)rod * ncell + c) * 3 + 1],
                             m_glob[((size_t)rod * ncell + c) * 3 + 2]);
    float3 u = make_float3(0.f, 0.f, 1.f);
    if (AX && act) u = xyz(__ldg(p.axis + (size_t)rod * ncell + c));
    __syncthreads();
    if (act && grp == 0) M[q] = pad4(m);
    __syncthreads();
    const float alpha = p.alpha, a = -p.neg_dt_g1;
    const int lane = threadIdx.x & 31, wig = c >> 5;  // lane, warp within the group
    Sweep field;
    field.init(tp.step0, p);
    float Hn = field.value();
    // the field-tangent and torque-tangent of one half step: dH = dc_ex N + c_ex Nd + rsig h +
    // the anisotropy tangent; ds = dc + dalpha m x c + alpha (dm x c + m x dc), dc = dm x H + m x dH
    auto half_tan = [&](float3 mm, float3 dmm, float3 N, float3 Nd, float3 h, float3 H, float3 *dsv) {
        float3 dH = add3(sc3(dcex, N), sc3(p.c_ex, Nd));
        dH = add3(dH, sc3(rsig, h));
        if constexpr (AX) {
            const float mu = dt3(mm, u), dmu = dt3(dmm, u);
            dH = add3(dH, sc3(fmaf(dcan, mu, p.c_an * dmu), u));
        } else {
            dH.z = fmaf(dcan, mm.z, fmaf(p.c_an, dmm.z, dH.z));
        }
        const float3 cc = crs(mm, H);
        const float3 dc = add3(crs(dmm, H), crs(mm, dH));
        *dsv = add3(add3(dc, sc3(dalpha, crs(mm, cc))), sc3(alpha, add3(crs(dmm, cc), crs(mm, dc))));
    };
    float3 hpre = zr3();  // thermal field of the next step, drawn before the step's last barrier
    if (act) hpre = thermal_field(p.seed, real, (uint32_t)c, (unsigned long long)tp.step0, p.sigma);
    for (int s = 0; s < tp.n_steps; ++s) {
        const unsigned long long n = (unsigned long long)(tp.step0 + s);
        field.inc();
        const float Hn1 = field.value();
        float3 acc = zr3(), dacc = zr3(), h = hpre, t = zr3(), dtt = zr3();
        if (act) {
            const float3 N = nbr(M, q, sy, sz), Nd = nbr(Md, q, sy, sz);
            const float3 H = effective_field_sel<AX>(N, m, h, p, Hn, u);
            const float3 s0 = llg_torque(m, H, alpha);
            float3 ds0;
            half_tan(m, dm, N, Nd, h, H, &ds0);
            const float3 pv = axpy(p.neg_dt_g1, s0, m);
            const float r = rsqrtf(fmaf(pv.x, pv.x, fmaf(pv.y, pv.y, pv.z * pv.z)));
            t = make_float3(pv.x * r, pv.y * r, pv.z * r);  // normalised(pv), the engines' arithmetic
            acc = axpy(p.neg_hdt_g1, s0, m);
            const float3 dp = sb3(sb3(dm, sc3(da, s0)), sc3(a, ds0));
            dtt = sc3(r, sb3(dp, sc3(dt3(t, dp), t)));
            dacc = sb3(sb3(dm, sc3(0.5f * da, s0)), sc3(0.5f * a, ds0));
            Pd[q] = pad4(dtt);
            if (grp == 0) P[q] = pad4(t);
        }
        __syncthreads();
        if (act) {
            const float3 N = nbr(P, q, sy, sz), Nd = nbr(Pd, q, sy, sz);
            const float3 H = effective_field_sel<AX>(N, t, h, p, Hn1, u);
            const float3 s1 = llg_torque(t, H, alpha);
            float3 ds1;
            half_tan(t, dtt, N, Nd, h, H, &ds1);
            const float3 qv = axpy(p.neg_hdt_g1, s1, acc);
            const float r = rsqrtf(fmaf(qv.x, qv.x, fmaf(qv.y, qv.y, qv.z * qv.z)));
            m = make_float3(qv.x * r, qv.y * r, qv.z * r);
            const float3 dq = sb3(sb3(dacc, sc3(0.5f * da, s1)), sc3(0.5f * a, ds1));
            dm = sc3(r, sb3(dq, sc3(dt3(m, dq), m)));
            Md[q] = pad4(dm);
            if (grp == 0) M[q] = pad4(m);
            hpre = thermal_field(p.seed, real, (uint32_t)c, n + 1, p.sigma);
        }
        __syncthreads();
        Hn = Hn1;
        const long long done = (long long)n + 1;
        if (p.sample_every > 0 && done % p.sample_every == 0) {
            const long long kk = done / p.sample_every - tp.k_first;
            if (kk >= 0 && kk < tp.n_k && wig == 0) {
                // the first warp of each group: the canonical reduction of m_z (group 0, as every
                // engine) or of its tangent's z component
                const float4 *A = grp == 0 ? M : Md;
                float part = 0.f, pd = 0.f;
                for (int cc = lane; cc < ncell; cc += 32) {
                    const int x = cc % p.nx, y = (cc / p.nx) % p.ny, z = cc / (p.nx * p.ny);
                    const int qq = (x + 1) + sy * (y + 1) + sz * (z + 1);
                    pd += Md[qq].z;
                    if (grp == 0) part += A[qq].z;
                }
                const float dmean = warp_cell_mean(pd, ncell);
                const float mean = grp == 0 ? warp_cell_mean(part, ncell) : 0.f;
                if (lane == 0) {
                    dsamples[((size_t)rod * tp.n_k + kk) * 3 + grp] = dmean;
                    if (grp == 0) {
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
    const size_t rod_pad = (size_t)(p.nx + 2) * (p.ny + 2) * (p.nz + 2);
    return p.periodic == 0 && p.ncells <= 256 && 8 * rod_pad * sizeof(float4) <= (size_t)smem_optin;
}

cudaError_t tangent_forward(const KParams &p, const double dcoef[15], int n_real, long long step0, long long n_steps,
                            long long k_first, int n_k, float *m_work, float *samples, float *dsamples, int *status,
                            cudaStream_t st)
{
    if (n_steps < 0 || n_steps > 0x7fffffffLL || n_k < 1) return cudaErrorInvalidValue;
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
    const size_t rod_pad = (size_t)(p.nx + 2) * (p.ny + 2) * (p.nz + 2);
    const size_t smem = 8 * rod_pad * sizeof(float4);
    const int threads = 3 * ((p.ncells + 31) / 32 * 32);  // three groups, one per tangent
    auto go = [&](auto kern) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<n_real, threads, smem, st>>>(tp, m_work, samples, dsamples, status);
        return cudaGetLastError();
    };
    if (threads <= 3 * 64) return p.axis ? go(tangent_kernel<true, 192>) : go(tangent_kernel<false, 192>);
    if (threads <= 3 * 256) return p.axis ? go(tangent_kernel<true, 768>) : go(tangent_kernel<false, 768>);
    return cudaErrorInvalidValue;
}

}  // namespace llg
