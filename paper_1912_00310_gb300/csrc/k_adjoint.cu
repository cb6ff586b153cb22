// k_adjoint.cu -- pathwise adjoint of the stochastic Heun step of Eq. 1: the gradient of a loss of
// the sampled M(H) loop with respect to the calibration scale factors (s_K, s_alpha, s_Ms) with
// the thermal normals held fixed (the same Philox draws replayed).
//
// Forward (per cell i, step n; N_i(m) = sum of the neighbours' m):
//   H  = c_ex N(m) + (c_an m_z + h_n) z + sigma xi          c0 = m x H,  s0 = c0 + alpha m x c0
//   p  = m - a s0,  m~ = p/|p|                              (a = dt g1, g1 = g0/(1 + alpha^2))
//   H~ = c_ex N(m~) + (c_an m~_z + h_n+1) z + sigma xi       c1 = m~ x H~, s1 = c1 + alpha m~ x c1
//   q  = m - (a/2)(s0 + s1),  m' = q/|q|
// Reverse (given g' = dL/dm'):
//   g_q = (g' - m'(m'.g'))/|q|;  g_m = g_q;  g_s0 = g_s1 = -(a/2) g_q;  g_a += -(s0 + s1).g_q/2
//   through s1: g_c1 = g_s1 + alpha g_s1 x m~;  g_m~ = alpha c1 x g_s1 + H~ x g_c1;
//               g_H~ = g_c1 x m~;  g_alpha += (m~ x c1).g_s1
//   through H~: g_m~_i += c_ex sum_j g_H~_j (neighbours), g_m~_z += c_an g_H~_z;
//               g_cex += g_H~.N(m~), g_can += g_H~_z m~_z, g_sigma += g_H~.xi
//   (with a per-cell easy axis u the anisotropy term is c_an (m.u) u: g_m~ += c_an (g_H~.u) u and
//   g_can += (g_H~.u)(m~.u))
//   g_p = (g_m~ - m~(m~.g_m~))/|p|;  g_m += g_p;  g_s0 += -a g_p;  g_a += -s0.g_p
//   through s0 and H: as through s1 and H~, with m, c0, H
// and dL/dm of the previous state is g_m.  The host maps (g_alpha, g_a, g_cex, g_can, g_sigma)
// to the scale factors (g_sigma is accumulated as g_H.h_th, i.e. sigma dL/dsigma).
//
// One CTA per rod, one cell per thread, the rod in shared memory (compact, with one zero slot for
// the neighbours beyond a free face).  The
// kernel has two phases: recompute the states of a checkpoint segment forward from its checkpoint
// (bitwise the forward run: same arithmetic) into global memory, and walk stored states backward.
// With memory to spare (the whole window's states, 12 bytes per cell, realisation and step), one
// launch recomputes every segment at once (a CTA per rod and segment) and one launch walks the
// whole window back, so the recomputation leaves the sequential critical path; otherwise each
// segment is recomputed and reversed in turn in one launch.  The parameter partial sums are FP32
// within blocks of 64 steps (aligned to absolute step numbers) and FP64 across blocks and in the
// per-CTA reduction.
#include <cmath>

#include "llg_internal.h"
#include "physics.cuh"
#include "rod_compact.cuh"
#include "sweep32.cuh"

namespace llg {
namespace {

using grad::cross3;
using grad::dot3;
using grad::scale3;
using grad::sub3;
using grad::Nbr;
using grad::neighbours;
__device__ __forceinline__ float3 zero3a() { return grad::zero3(); }

constexpr long long kAdjBlock = 64;  // steps per FP32 block of the parameter partial sums

struct AdjParams {
    KParams p;
    long long seg_start;  // first step of the segment
    int seg_len;          // steps in the segment
    long long win_end;    // last step index + 1 of the window (samples at (start, win_end])
    long long k_first;    // sample number of w[0]
    int n_k;
    float inj_scale;      // 1 / (n_real * ncells)
    int phases;           // bit 0: recompute the segment forward; bit 1: walk it backward
    int seg_stride;       // recompute with gridDim.y > 1: segment blockIdx.y starts seg_stride
                          // steps after seg_start (its checkpoint and states offset to match)
    long long n_total;    // ... and the window has n_total steps (the last segment is shorter)
};

// MAXT: the largest CTA the instance runs with (256 for rods up to 256 cells, which then get up to
// 255 registers per thread, 1024 otherwise); SHAPE: the sweep shape with 32-bit bookkeeping (0
// triangle, 1 cosine) or -1 for the 64-bit sweep of any period.
template <bool AX, int MAXT, int SHAPE>
__global__ void __launch_bounds__(MAXT) adjoint_segment_kernel(
    AdjParams ap, const float *__restrict__ ckpt, float *__restrict__ seg, float *__restrict__ lam,
    const double *__restrict__ w, double *__restrict__ partial)
{
    extern __shared__ float4 sm4[];
    const KParams &p = ap.p;
    const int ncell = p.ncells;
    const int S = ncell + 1;  // cells and the zero slot
    float4 *M = sm4, *P = M + S, *GT = P + S, *GH = GT + S;
    const int rod = blockIdx.x;
    const int c = threadIdx.x;
    const bool act = c < ncell;
    for (int i = threadIdx.x; i < 4 * S; i += blockDim.x) sm4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    const Nbr nb = neighbours(act ? c : 0, p.nx, p.ny, p.nz, ncell);
    const int q = c;  // this cell's slot
    const uint32_t real = p.real0 + (uint32_t)rod;
    const PhiloxKeys keys = philox_keys(p.seed, real);  // the rod's round keys, formed once
    const size_t state = (size_t)ncell * 3;
    const size_t rod_off = (size_t)rod * state;
    const int n_rods = gridDim.x;
    long long seg_start = ap.seg_start;
    int seg_len = ap.seg_len;
    if (gridDim.y > 1) {  // one segment of a window recomputed all at once
        const long long off = (long long)blockIdx.y * ap.seg_stride;
        seg_start += off;
        seg_len = (int)min((long long)ap.seg_stride, ap.n_total - off);
        ckpt += (size_t)blockIdx.y * n_rods * state;
        seg += (size_t)off * n_rods * state;
    }
    float3 m = zero3a();
    if (act && (ap.phases & 1))
        m = make_float3(ckpt[rod_off + 3 * c], ckpt[rod_off + 3 * c + 1], ckpt[rod_off + 3 * c + 2]);
    float3 u = make_float3(0.f, 0.f, 1.f);  // easy axis (dispersed-axis mode, AX)
    if (AX && act) u = xyz(__ldg(p.axis + (size_t)rod * ncell + c));
    auto field_of = [&](float3 nb, float3 mm, float3 hh, float Hz) {
        return effective_field_sel<AX>(nb, mm, hh, p, Hz, u);
    };
    __syncthreads();

    // ---- forward recomputation of the segment: seg[j] = state before step seg_start + j ----
    typename SweepSel<SHAPE>::type field;
    field.init(seg_start, p);
    float Hn = field.value();
    for (int j = 0; j < ((ap.phases & 1) ? seg_len : 0); ++j) {
        const unsigned long long n = (unsigned long long)(seg_start + j);
        field.inc();
        const float Hn1 = field.value();
        float *sj = seg + (size_t)j * n_rods * state + rod_off;
        float3 acc = zero3a(), h = zero3a();
        if (act) {
            sj[3 * c] = m.x;
            sj[3 * c + 1] = m.y;
            sj[3 * c + 2] = m.z;
            M[q] = pad4(m);
        }
        __syncthreads();
        if (act) {
            h = thermal_field(keys, (uint32_t)c, n, p.sigma);
            const float3 H = field_of(grad::neighbour_sum(M, nb), m, h, Hn);
            const float3 s0 = llg_torque(m, H, p.alpha);
            P[q] = pad4(normalised(axpy(p.neg_dt_g1, s0, m)));
            acc = axpy(p.neg_hdt_g1, s0, m);
        }
        __syncthreads();
        if (act) {
            const float3 t = xyz(P[q]);
            const float3 H = field_of(grad::neighbour_sum(P, nb), t, h, Hn1);
            m = normalised(axpy(p.neg_hdt_g1, llg_torque(t, H, p.alpha), acc));
        }
        __syncthreads();
        Hn = Hn1;
    }

    if (!(ap.phases & 2)) return;
    // ---- backward through the segment ----
    float3 g = zero3a();  // dL/d(state after the step being reversed)
    if (act) g = make_float3(lam[rod_off + 3 * c], lam[rod_off + 3 * c + 1], lam[rod_off + 3 * c + 2]);
    // parameter partial sums: FP32 within blocks of kAdjBlock steps (aligned to absolute step
    // numbers, so both reverse schedules form the same block sums), FP64 across blocks -- the
    // GPU's FP64 rate is a small fraction of its FP32 rate, and a per-step FP64 update made the
    // reverse step wait on it
    double g_alpha = 0.0, g_a = 0.0, g_cex = 0.0, g_can = 0.0, g_sigma = 0.0;
    float f_alpha = 0.f, f_a = 0.f, f_cex = 0.f, f_can = 0.f, f_sigma = 0.f;
    auto flush = [&]() {
        g_alpha += (double)f_alpha;
        g_a += (double)f_a;
        g_cex += (double)f_cex;
        g_can += (double)f_can;
        g_sigma += (double)f_sigma;
        f_alpha = f_a = f_cex = f_can = f_sigma = 0.f;
    };
    const float a = -p.neg_dt_g1;  // dt g1
    const float ha = -p.neg_hdt_g1;
    const float alpha = p.alpha;
    field.init(seg_start + seg_len - 1, p);
    // sample bookkeeping of the reverse walk in 32 bits: done = n + 1 runs down from
    // seg_start + seg_len; r = done mod sample_every, kd = done / sample_every (the host keeps
    // sample_every below 2^31)
    const long long se = p.sample_every;
    int r_s = se > 0 ? (int)((seg_start + seg_len) % se) : -1;
    long long kd = se > 0 ? (seg_start + seg_len) / se : 0;
    // Three barriers per reversed step.  The state before step j sits in M from the previous
    // iteration (it is stored there with the last shared write of that iteration, after every
    // read of M), and the stored state of the next step to reverse is loaded one step ahead (a
    // stored window is larger than L2, so each load would otherwise wait on HBM).
    float3 m_cur = zero3a(), m_ahead = zero3a();
    if (act && seg_len > 0) {
        const float *sl = seg + (size_t)(seg_len - 1) * n_rods * state + rod_off;
        m_cur = make_float3(sl[3 * c], sl[3 * c + 1], sl[3 * c + 2]);
        M[q] = pad4(m_cur);
    }
    __syncthreads();
    for (int j = seg_len - 1; j >= 0; --j) {
        const long long n = seg_start + j;
        const float hn = field.value();
        auto f1 = field;
        f1.inc();
        const float hn1 = f1.value();
        // loss gradient of the state after step n, if it is a sample of the window
        if (r_s == 0 && n + 1 <= ap.win_end) {
            const long long k = kd - ap.k_first;
            if (k >= 0 && k < ap.n_k) g.z += (float)w[k] * ap.inj_scale;
        }
        if (r_s == 0) {
            r_s = (int)se - 1;
            --kd;
        } else if (r_s > 0) {
            --r_s;
        }
        float3 mi = zero3a(), h = zero3a(), H = zero3a(), c0 = zero3a(), s0 = zero3a(), t = zero3a();
        float pn = 1.f;  // 1 / |p|
        if (act) {
            mi = m_cur;
            if (j > 0) {
                const float *sn = seg + (size_t)(j - 1) * n_rods * state + rod_off;
                m_ahead = make_float3(sn[3 * c], sn[3 * c + 1], sn[3 * c + 2]);
            }
        }
        float3 Nm = zero3a();
        if (act) {
            h = thermal_field(keys, (uint32_t)c, (unsigned long long)n, p.sigma);
            Nm = grad::neighbour_sum(M, nb);
            H = field_of(Nm, mi, h, hn);
            c0 = cross3(mi, H);
            s0 = llg_torque(mi, H, alpha);
            const float3 pv = axpy(p.neg_dt_g1, s0, mi);
            pn = rsqrtf(dot3(pv, pv));  // 1 / |p|
            t = normalised(pv);
            P[q] = pad4(t);
        }
        __syncthreads();
        float3 gHt = zero3a(), Nt = zero3a(), c1 = zero3a(), gq = zero3a(), gmt = zero3a(), Ht = zero3a();
        float3 s1 = zero3a();
        if (act) {
            Nt = grad::neighbour_sum(P, nb);
            Ht = field_of(Nt, t, h, hn1);
            c1 = cross3(t, Ht);
            s1 = llg_torque(t, Ht, alpha);
            const float3 qv = axpy(p.neg_hdt_g1, add3(s0, s1), mi);
            const float rq = rsqrtf(dot3(qv, qv));  // 1 / |q|: m' = rq q, the forward's normalisation
            const float3 mp = scale3(rq, qv);
            gq = scale3(rq, sub3(g, scale3(dot3(mp, g), mp)));
            const float3 gs1 = scale3(-ha, gq);
            f_a -= 0.5f * dot3(add3(s0, s1), gq);
            const float3 gc1 = add3(gs1, scale3(alpha, cross3(gs1, t)));
            gmt = add3(scale3(alpha, cross3(c1, gs1)), cross3(Ht, gc1));
            gHt = cross3(gc1, t);
            f_alpha += dot3(cross3(t, c1), gs1);
            GT[q] = pad4(gHt);
        }
        __syncthreads();
        float3 gH = zero3a(), gm = zero3a();
        if (act) {
            gmt = axpy(p.c_ex, grad::neighbour_sum(GT, nb), gmt);
            if constexpr (AX) {
                const float gu = dot3(gHt, u);
                gmt = axpy(p.c_an * gu, u, gmt);
                f_can += gu * dot3(t, u);
            } else {
                gmt.z = fmaf(p.c_an, gHt.z, gmt.z);
                f_can += gHt.z * t.z;
            }
            f_cex += dot3(gHt, Nt);
            f_sigma += dot3(gHt, h);  // d/dsigma = (1/sigma) g_H.h, divided on the host
            const float3 gp = scale3(pn, sub3(gmt, scale3(dot3(t, gmt), t)));
            gm = add3(gq, gp);                                     // q = m - ..., p = m - a s0
            const float3 gs0 = add3(scale3(-ha, gq), scale3(-a, gp));  // from q and from p
            f_a -= dot3(s0, gp);
            const float3 gc0 = add3(gs0, scale3(alpha, cross3(gs0, mi)));
            gm = add3(gm, add3(scale3(alpha, cross3(c0, gs0)), cross3(H, gc0)));
            gH = cross3(gc0, mi);
            f_alpha += dot3(cross3(mi, c0), gs0);
            GH[q] = pad4(gH);
            if (j > 0) M[q] = pad4(m_ahead);  // M was last read before the previous barrier
        }
        __syncthreads();
        if (act) {
            gm = axpy(p.c_ex, grad::neighbour_sum(GH, nb), gm);
            if constexpr (AX) {
                const float gu = dot3(gH, u);
                gm = axpy(p.c_an * gu, u, gm);
                f_can += gu * dot3(mi, u);
            } else {
                gm.z = fmaf(p.c_an, gH.z, gm.z);
                f_can += gH.z * mi.z;
            }
            f_cex += dot3(gH, Nm);
            f_sigma += dot3(gH, h);
            g = gm;
            m_cur = m_ahead;
            if (n % kAdjBlock == 0) flush();
        }
        // no barrier here: the next iteration's first shared write (P) follows reads of P that
        // ended before this iteration's second barrier, and GH is next written after two barriers
        // step back the field phase
        field.dec();
    }
    flush();
    if (act) {
        lam[rod_off + 3 * c] = g.x;
        lam[rod_off + 3 * c + 1] = g.y;
        lam[rod_off + 3 * c + 2] = g.z;
    }
    // per-CTA partial sums of the parameter adjoints, fixed order
    __shared__ double red[5][32];
    double v[5] = {g_alpha, g_a, g_cex, g_can, g_sigma};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        double x = v[k];
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double s = 0.0;
        for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) s += red[threadIdx.x][wi];
        partial[(size_t)rod * 5 + threadIdx.x] += s;
    }
}

}  // namespace

bool adjoint_supported(const KParams &p, int dev)
{
    int smem_optin = 0;
    if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
    return p.periodic == 0 && p.ncells <= 1024 && 4 * (size_t)(p.ncells + 1) * sizeof(float4) <= (size_t)smem_optin;
}

namespace {
cudaError_t launch_adjoint(const AdjParams &ap, int n_real, int n_seg, const float *ckpt, float *seg, float *lam,
                           const double *w, double *partial, cudaStream_t st)
{
    const KParams &p = ap.p;
    const size_t smem = 4 * (size_t)(p.ncells + 1) * sizeof(float4);
    const int threads = (p.ncells + 31) / 32 * 32;
    const dim3 grid((unsigned)n_real, (unsigned)n_seg);
    if (p.sample_every >= (1LL << 31)) return cudaErrorInvalidValue;
    // the sweep shape at compile time where its period fits 32 bits
    const int shape = sweep_fits_32(p) ? (p.shape == 1 ? 1 : 0) : -1;
    auto go = [&](auto kern) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, threads, smem, st>>>(ap, ckpt, seg, lam, w, partial);
        return cudaGetLastError();
    };
    auto by_shape = [&](auto k0, auto k1, auto kg) { return shape == 0 ? go(k0) : shape == 1 ? go(k1) : go(kg); };
#define LLG_ADJ(AXV, T) \
    adjoint_segment_kernel<AXV, T, 0>, adjoint_segment_kernel<AXV, T, 1>, adjoint_segment_kernel<AXV, T, -1>
    if (threads <= 256) return p.axis ? by_shape(LLG_ADJ(true, 256)) : by_shape(LLG_ADJ(false, 256));
    return p.axis ? by_shape(LLG_ADJ(true, 1024)) : by_shape(LLG_ADJ(false, 1024));
#undef LLG_ADJ
}

AdjParams adj_params(const KParams &p, int n_real, long long seg_start, int seg_len, long long win_end,
                     long long k_first, int n_k, int phases)
{
    AdjParams ap;
    ap.p = p;
    ap.seg_start = seg_start;
    ap.seg_len = seg_len;
    ap.win_end = win_end;
    ap.k_first = k_first;
    ap.n_k = n_k;
    ap.inj_scale = 1.0f / ((float)n_real * (float)p.ncells);
    ap.phases = phases;
    ap.seg_stride = 0;
    ap.n_total = 0;
    return ap;
}
}  // namespace

cudaError_t adjoint_segment(const KParams &p, int n_real, long long seg_start, int seg_len, long long win_end,
                            long long k_first, int n_k, const float *ckpt, float *seg, float *lam,
                            const double *w, double *partial, cudaStream_t st)
{
    const AdjParams ap = adj_params(p, n_real, seg_start, seg_len, win_end, k_first, n_k, 3);
    return launch_adjoint(ap, n_real, 1, ckpt, seg, lam, w, partial, st);
}

cudaError_t adjoint_recompute_all(const KParams &p, int n_real, long long step0, long long n_steps, int ckpt_every,
                                  const float *ckpt, float *states, cudaStream_t st)
{
    const long long n_seg = (n_steps + ckpt_every - 1) / ckpt_every;
    if (n_seg < 1 || n_seg > 65535) return cudaErrorInvalidValue;
    AdjParams ap = adj_params(p, n_real, step0, ckpt_every, step0 + n_steps, 0, 0, 1);
    ap.seg_stride = ckpt_every;
    ap.n_total = n_steps;
    return launch_adjoint(ap, n_real, (int)n_seg, ckpt, states, nullptr, nullptr, nullptr, st);
}

cudaError_t adjoint_backward_all(const KParams &p, int n_real, long long step0, long long n_steps, long long k_first,
                                 int n_k, const float *states, float *lam, const double *w, double *partial,
                                 cudaStream_t st)
{
    if (n_steps < 1 || n_steps > 0x7fffffffLL) return cudaErrorInvalidValue;
    const AdjParams ap = adj_params(p, n_real, step0, (int)n_steps, step0 + n_steps, k_first, n_k, 2);
    return launch_adjoint(ap, n_real, 1, nullptr, const_cast<float *>(states), lam, w, partial, st);
}

}  // namespace llg
