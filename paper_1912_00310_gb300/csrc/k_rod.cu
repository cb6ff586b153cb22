// k_rod.cu -- the resident engine: whole rods live in shared memory for an entire launch of
// thousands of Heun steps of Eq. 1, and only the sampled M(H) values reach HBM.
//
// Two kernels, chosen by rod size:
//
//  rod_twophase_kernel  (rods whose state and predictor state both fit: b >= 2 in the paper's
//      ladder), in k_rod_small.cu.  Several rods per CTA, each padded with a zero ghost layer.
//
//  rod_pipelined_kernel (the b = 1 rod, 8x24x56 = 10752 cells: M alone is 129 KB, M and a full
//      predictor copy do not fit).  One rod per CTA.  Each thread owns rows along x (fixed y, z);
//      the CTA sweeps the x planes in lock step, computing the predictor at plane x and the
//      corrector at plane x-1 in the same iteration, so only two planes of predictor state are
//      ever needed (double-buffered by the parity of the plane counter).  The x-neighbours come
//      from registers, the y- and z-neighbours from shared memory.  When nx >= 3 the corrector of
//      the last plane of step n shares its iteration with the predictor of plane 0 of step n+1,
//      so every iteration does both halves of the work: nx barriers per step.
//
//  rod_pipelined_nx_kernel: the same schedule with the plane count (and, for the b = 1 rod, the
//      whole shape) and the sweep shape fixed at compile time, unrolled over the planes and run
//      over a co-resident grid with a balanced schedule of rod-steps (McNaughton's wrap-around
//      rule) when the rods do not fill whole waves.
//
// The thread count of the plane-pipelined kernels balances the rows over the SM's four
// schedulers (pipelined_threads).  The dispersed-axis mode (per-cell easy axes in global memory)
// runs the AX instances: of the two-phase kernel, of the runtime-size plane-pipelined kernel and,
// for the b = 1 rod at three rows per thread, of the shape-specialised one.
//
// Both kernels add the neighbours in the order x-, x+, y-, y+, z-, z+ with exact zeros for
// missing ones and use the same physics.cuh arithmetic as the plain engine, so all engines
// produce bitwise-identical trajectories.  Samples use the canonical warp reduction (reduce.cuh).
#include <algorithm>
#include <cstring>

#include "llg_internal.h"
#include "physics.cuh"
#include "reduce.cuh"

namespace llg {
namespace {

// At most 768 threads per CTA leaves 85 registers per thread, enough for the per-cell Heun
// state (predictor accumulator and thermal field) of two cells or rows without spilling.
constexpr int kMaxThreads = 768;

__device__ __forceinline__ float3 zero3() { return make_float3(0.f, 0.f, 0.f); }

// ------------------------------------------------------------------------------------------
// plane-pipelined kernel
// ------------------------------------------------------------------------------------------
// Shared memory (float4 = x, y, z, 0): M[nx][PL] (state) and S[2][PL] (predictor planes),
// PL = (nz + 2) * ny: each plane holds the rows (y, z) at offset q = (z + 1) * ny + y, with zero
// ghost lines at z = -1 and z = nz; the y faces are handled by 0/1 weights.
// Threads per CTA of the plane-pipelined kernel for R rows per thread.  The register file is split
// over the four SM sub-partitions (16384 registers each), so the per-thread budget is set by the
// warps per sub-partition: 768 or 672 threads -> 80 registers, 512 -> 128, 384 -> 168.
__host__ __device__ constexpr int pipelined_max_threads(int R)
{
    return R == 1 ? 768 : (R == 2 ? 672 : (R == 3 ? 512 : 384));
}

template <int R, bool AX>
__global__ void __launch_bounds__(pipelined_max_threads(R), 1) rod_pipelined_kernel(KParams p, float *__restrict__ m_glob,
                                                               long long step0, long long n_steps,
                                                               float *__restrict__ samples,
                                                               int *__restrict__ status)
{
    extern __shared__ float4 sm4[];
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int rows = ny * nz;
    const int PL = (nz + 2) * ny;
    float4 *M = sm4;
    float4 *S = sm4 + nx * PL;
    const int T = blockDim.x;
    const int rod = blockIdx.x;
    const int ncell = p.ncells;

    for (int i = threadIdx.x; i < (nx + 2) * PL; i += T) sm4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    {
        const float *g = m_glob + (size_t)rod * ncell * 3;
        for (int c = threadIdx.x; c < ncell; c += T) {
            const int x = c % nx, rr = c / nx;
            M[x * PL + ny + rr] = make_float4(g[3 * (size_t)c], g[3 * (size_t)c + 1], g[3 * (size_t)c + 2], 0.f);
        }
    }

    int q[R];
    float wm[R], wp[R];
    bool act[R];
    uint32_t cbase[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const int r = threadIdx.x + j * T;
        act[j] = r < rows;
        const int rr = act[j] ? r : 0;
        const int y = rr % ny;
        q[j] = ny + rr;
        wm[j] = y > 0 ? 1.f : 0.f;
        wp[j] = y < ny - 1 ? 1.f : 0.f;
        cbase[j] = (uint32_t)(rr * nx);  // cell index x + nx * (y + ny * z), rr = y + ny * z
    }
    const PhiloxKeys keys = philox_keys(p.seed, p.real0 + (uint32_t)rod);
    const float4 *axr = AX ? p.axis + (size_t)rod * ncell : nullptr;  // this rod's easy axes

    float3 mprev[R], mcur[R], mta[R], mtb[R], acc[R], hth[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        mprev[j] = mcur[j] = mta[j] = mtb[j] = acc[j] = hth[j] = zero3();
    }
    __syncthreads();

    const bool merged = nx >= 3;
    bool pa = n_steps > 0, ca = false;
    long long sp = 0, sc = 0;
    int xp = 0, xc = 0;
    Sweep fpred, fcorr;
    fpred.init(step0, p);
    fcorr.init(step0 + 1, p);
    float Hp = fpred.value(), Hc = fcorr.value();
    const long long se = p.sample_every;
    long long next_sample = (samples && se > 0) ? (step0 / se + 1) * se : -1;
    const int lane = threadIdx.x & 31;

    while (pa || ca) {
        float3 mt_new[R], acc_new[R], h_new[R];
        if (pa) {
            const unsigned long long n = (unsigned long long)(step0 + sp);
            const float4 *Mp = M + xp * PL;
            float4 *Sw = S + (int)((sp * nx + xp) & 1) * PL;
            const bool has_next = xp + 1 < nx;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                if (!act[j]) continue;
                const int qq = q[j];
                if (xp == 0) {
                    mcur[j] = xyz(Mp[qq]);
                    mprev[j] = zero3();
                }
                const float3 mnext = has_next ? xyz(Mp[qq + PL]) : zero3();
                h_new[j] = thermal_field(keys, cbase[j] + (uint32_t)xp, n, p.sigma);
                float3 nb = add3(mprev[j], mnext);
                nb = axpy(wm[j], xyz(Mp[qq - 1]), nb);
                nb = axpy(wp[j], xyz(Mp[qq + 1]), nb);
                nb = add3(nb, xyz(Mp[qq - ny]));
                nb = add3(nb, xyz(Mp[qq + ny]));
                const float3 u = AX ? xyz(__ldg(axr + cbase[j] + xp)) : zero3();
                const float3 H = effective_field_sel<AX>(nb, mcur[j], h_new[j], p, Hp, u);
                const float3 s0 = llg_torque(mcur[j], H, p.alpha);
                mt_new[j] = normalised(axpy(p.neg_dt_g1, s0, mcur[j]));
                acc_new[j] = axpy(p.neg_hdt_g1, s0, mcur[j]);
                Sw[qq] = pad4(mt_new[j]);
                mprev[j] = mcur[j];
                mcur[j] = mnext;
            }
        }
        if (ca) {
            const float4 *Sr = S + (int)((sc * nx + xc) & 1) * PL;
            float4 *Mw = M + xc * PL;
            const bool has_next = xc + 1 < nx;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                if (!act[j]) continue;
                const int qq = q[j];
                const float3 tnext = has_next ? mt_new[j] : zero3();
                float3 nb = add3(mta[j], tnext);
                nb = axpy(wm[j], xyz(Sr[qq - 1]), nb);
                nb = axpy(wp[j], xyz(Sr[qq + 1]), nb);
                nb = add3(nb, xyz(Sr[qq - ny]));
                nb = add3(nb, xyz(Sr[qq + ny]));
                const float3 u = AX ? xyz(__ldg(axr + cbase[j] + xc)) : zero3();
                const float3 H = effective_field_sel<AX>(nb, mtb[j], hth[j], p, Hc, u);
                const float3 s1 = llg_torque(mtb[j], H, p.alpha);
                Mw[qq] = pad4(normalised(axpy(p.neg_hdt_g1, s1, acc[j])));
            }
        }
        if (pa) {
#pragma unroll
            for (int j = 0; j < R; ++j) {
                mta[j] = xp == 0 ? zero3() : mtb[j];
                mtb[j] = mt_new[j];
                acc[j] = acc_new[j];
                hth[j] = h_new[j];
            }
        }
        __syncthreads();
        if (ca && xc == nx - 1 && step0 + sc + 1 == next_sample) {
            const long long k = next_sample / se;
            if (k < p.n_samples && threadIdx.x < 32) {
                float part = 0.f;
                for (int c = lane; c < ncell; c += 32) part += M[(c % nx) * PL + ny + c / nx].z;
                const float mean = warp_cell_mean(part, ncell);
                if (lane == 0) {
                    samples[(size_t)rod * p.n_samples + k] = mean;
                    if (!isfinite(mean)) atomicOr(status, 1);
                }
            }
            next_sample += se;
            __syncthreads();
        }
        // advance the schedule; the corrector takes the predictor's old position
        const bool old_pa = pa;
        const long long old_sp = sp;
        const int old_xp = xp;
        if (merged) {
            if (pa && ++xp == nx) {
                xp = 0;
                ++sp;
                fpred.inc();
                Hp = fpred.value();
                pa = sp < n_steps;
            }
        } else if (pa) {
            if (++xp == nx) pa = false;  // one corrector-only iteration closes the step
        } else if (ca) {
            ++sp;
            xp = 0;
            fpred.inc();
            Hp = fpred.value();
            pa = sp < n_steps;
        }
        ca = old_pa;
        if (old_pa) {
            if (old_sp != sc) {
                sc = old_sp;
                fcorr.inc();
                Hc = fcorr.value();
            }
            xc = old_xp;
        }
    }

    {
        float *g = m_glob + (size_t)rod * ncell * 3;
        for (int c = threadIdx.x; c < ncell; c += T) {
            const float4 v = M[(c % nx) * PL + ny + c / nx];
            g[3 * (size_t)c] = v.x;
            g[3 * (size_t)c + 1] = v.y;
            g[3 * (size_t)c + 2] = v.z;
        }
    }
}

// ------------------------------------------------------------------------------------------
// plane-pipelined kernel with a compile-time plane count (the b = 1 rod has NX = 8): the x sweep
// of a step is unrolled, so the plane windows rotate by register renaming and the slot parity
// is a constant.  Same schedule and arithmetic as rod_pipelined_kernel.
// ------------------------------------------------------------------------------------------
// NY, NZ > 0: the rod's y and z extents are compile-time constants (the b = 1 rod), so every
// shared-memory offset of the stencil is an immediate.
template <int R, int NX, int NY = 0, int NZ = 0, int SHAPE = -1, bool AX = false>
struct PipelinedRod {
    float4 *M, *S;
    int ny_rt, PL_rt, ncell;
    __device__ __forceinline__ int ny() const
    {
        if constexpr (NY > 0) return NY;
        return ny_rt;
    }
    __device__ __forceinline__ int PL() const
    {
        if constexpr (NY > 0 && NZ > 0) return (NZ + 2) * NY;
        return PL_rt;
    }
    int q[R];
    float wm[R], wp[R];
    bool act[R];
    uint32_t cbase[R];

    __device__ void setup(float4 *sm, const KParams &p)
    {
        ny_rt = p.ny;
        PL_rt = (p.nz + 2) * p.ny;
        ncell = p.ncells;
        M = sm;
        S = sm + NX * PL();
        const int ny = this->ny();
        const int rows = ny * p.nz;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int r = threadIdx.x + j * blockDim.x;
            act[j] = r < rows;
            const int rr = act[j] ? r : 0;
            const int y = rr % ny;
            q[j] = ny + rr;
            wm[j] = y > 0 ? 1.f : 0.f;
            wp[j] = y < ny - 1 ? 1.f : 0.f;
            cbase[j] = (uint32_t)(rr * NX);
        }
    }

    // Sample k of rod `rod`: the canonical warp reduction of m_z over the cells in M, then a
    // barrier (the next iteration overwrites plane 0).
    __device__ __forceinline__ void sample(const KParams &p, int rod, long long k, float *__restrict__ samples,
                                        int *__restrict__ status)
    {
        const int ny = this->ny(), PL = this->PL();
        if (k < p.n_samples && threadIdx.x < 32) {
            const int lane = threadIdx.x;
            float part = 0.f;
            for (int c = lane; c < ncell; c += 32) part += M[(c % NX) * PL + ny + c / NX].z;
            const float mean = warp_cell_mean(part, ncell);
            if (lane == 0) {
                samples[(size_t)rod * p.n_samples + k] = mean;
                if (!isfinite(mean)) atomicOr(status, 1);
            }
        }
        __syncthreads();
    }

    // Load rod `rod` from global memory (L2, bypassing L1: another SM may have written it during
    // this launch), advance it from step s0 by ns steps, store it back.
    __device__ __forceinline__ void run(const KParams &p, float *__restrict__ m_glob, int rod, long long s0,
                                        long long ns, float *__restrict__ samples, int *__restrict__ status)
    {
        const int ny = this->ny(), PL = this->PL();
        {
            const float *g = m_glob + (size_t)rod * ncell * 3;
            for (int c = threadIdx.x; c < ncell; c += blockDim.x)
                M[(c % NX) * PL + ny + c / NX] = make_float4(__ldcg(g + 3 * (size_t)c), __ldcg(g + 3 * (size_t)c + 1),
                                                             __ldcg(g + 3 * (size_t)c + 2), 0.f);
        }
        const PhiloxKeys keys = philox_keys(p.seed, p.real0 + (uint32_t)rod);
        const float4 *axr = AX ? p.axis + (size_t)rod * ncell : nullptr;  // easy axes (AX)
        // carried per row: m(x-1), m(x) for the predictor; m~(x-2), m~(x-1), acc(x-1), h(x-1)
        // for the corrector one plane behind
        float3 mA[R], mB[R], tA[R], tB[R], acc[R], hth[R];
#pragma unroll
        for (int j = 0; j < R; ++j) mA[j] = mB[j] = tA[j] = tB[j] = acc[j] = hth[j] = zero3();
        __syncthreads();

        SweepOf<SHAPE> field;
        field.init(s0, p);
        float Hs = field.value();  // field at step s
        field.inc();
        float Hs1 = field.value();  // field at step s + 1
        float Hprev = Hs;           // field at step s (the end of step s - 1), for its corrector
        const long long se = p.sample_every;
        long long next_sample = (samples && se > 0) ? (s0 / se + 1) * se : -1;
        // thermal field of the next predictor, drawn one iteration ahead (before the barrier)
        float3 hpre[R];
#pragma unroll
        for (int j = 0; j < R; ++j) hpre[j] = thermal_field(keys, cbase[j], (unsigned long long)s0, p.sigma);
        // AX: the easy axis of the next predictor's cell, loaded one iteration ahead like the
        // noise, and the axis of the plane the corrector works on (the previous predictor's)
        float3 upre[R], ucor[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
            upre[j] = ucor[j] = zero3();
            if constexpr (AX) upre[j] = xyz(__ldg(axr + cbase[j]));
        }

        for (long long s = 0; s < ns; ++s) {
            const unsigned long long n = (unsigned long long)(s0 + s);
#pragma unroll
            for (int x = 0; x < NX; ++x) {
                // ---- predictor at (s, x): writes slot x & 1 ----
                const float4 *Mp = M + x * PL;
                float4 *Sw = S + (x & 1) * PL;
                float3 tnew[R], anew[R], hnew[R];
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    if (!act[j]) continue;
                    const int qq = q[j];
                    if (x == 0) {
                        mA[j] = zero3();
                        mB[j] = xyz(Mp[qq]);
                    }
                    const float3 mnext = x + 1 < NX ? xyz(Mp[qq + PL]) : zero3();
                    hnew[j] = hpre[j];
                    float3 nb = add3(mA[j], mnext);
                    nb = axpy(wm[j], xyz(Mp[qq - 1]), nb);
                    nb = axpy(wp[j], xyz(Mp[qq + 1]), nb);
                    nb = add3(nb, xyz(Mp[qq - ny]));
                    nb = add3(nb, xyz(Mp[qq + ny]));
                    const float3 H = effective_field_sel<AX>(nb, mB[j], hnew[j], p, Hs, upre[j]);
                    const float3 s0v = llg_torque(mB[j], H, p.alpha);
                    tnew[j] = normalised(axpy(p.neg_dt_g1, s0v, mB[j]));
                    anew[j] = axpy(p.neg_hdt_g1, s0v, mB[j]);
                    Sw[qq] = pad4(tnew[j]);
                    mA[j] = mB[j];
                    mB[j] = mnext;
                }
                // ---- corrector one plane behind: (s, x-1), or (s-1, NX-1) at x = 0 ----
                if (x > 0 || s > 0) {
                    const int xc = x > 0 ? x - 1 : NX - 1;
                    const float4 *Sr = S + (xc & 1) * PL;
                    float4 *Mw = M + xc * PL;
                    const float Hc = x > 0 ? Hs1 : Hprev;
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        if (!act[j]) continue;
                        const int qq = q[j];
                        const float3 tnext = x > 0 ? tnew[j] : zero3();
                        float3 nb = add3(tA[j], tnext);
                        nb = axpy(wm[j], xyz(Sr[qq - 1]), nb);
                        nb = axpy(wp[j], xyz(Sr[qq + 1]), nb);
                        nb = add3(nb, xyz(Sr[qq - ny]));
                        nb = add3(nb, xyz(Sr[qq + ny]));
                        const float3 H = effective_field_sel<AX>(nb, tB[j], hth[j], p, Hc, ucor[j]);
                        const float3 s1 = llg_torque(tB[j], H, p.alpha);
                        Mw[qq] = pad4(normalised(axpy(p.neg_hdt_g1, s1, acc[j])));
                    }
                }
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    tA[j] = x == 0 ? zero3() : tB[j];
                    tB[j] = tnew[j];
                    acc[j] = anew[j];
                    hth[j] = hnew[j];
                    // the next predictor: plane x+1 of this step, or plane 0 of the next one
                    hpre[j] = x + 1 < NX ? thermal_field(keys, cbase[j] + (uint32_t)(x + 1), n, p.sigma)
                                         : thermal_field(keys, cbase[j], n + 1, p.sigma);
                    if constexpr (AX) {
                        ucor[j] = upre[j];
                        upre[j] = xyz(__ldg(axr + cbase[j] + (uint32_t)(x + 1 < NX ? x + 1 : 0)));
                    }
                }
                __syncthreads();
                if (x == 0 && s > 0 && s0 + s == next_sample) {
                    sample(p, rod, next_sample / se, samples, status);
                    next_sample += se;
                }
            }
            Hprev = Hs1;
            Hs = Hs1;
            field.inc();
            Hs1 = field.value();
        }
        if (ns > 0) {
            // the corrector of the last plane of the last step
            const float4 *Sr = S + ((NX - 1) & 1) * PL;
            float4 *Mw = M + (NX - 1) * PL;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                if (!act[j]) continue;
                const int qq = q[j];
                float3 nb = tA[j];
                nb = axpy(wm[j], xyz(Sr[qq - 1]), nb);
                nb = axpy(wp[j], xyz(Sr[qq + 1]), nb);
                nb = add3(nb, xyz(Sr[qq - ny]));
                nb = add3(nb, xyz(Sr[qq + ny]));
                const float3 H = effective_field_sel<AX>(nb, tB[j], hth[j], p, Hprev, ucor[j]);
                const float3 s1 = llg_torque(tB[j], H, p.alpha);
                Mw[qq] = pad4(normalised(axpy(p.neg_hdt_g1, s1, acc[j])));
            }
            __syncthreads();
            if (s0 + ns == next_sample) sample(p, rod, next_sample / se, samples, status);
        }
        {
            float *g = m_glob + (size_t)rod * ncell * 3;
            for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
                const float4 v = M[(c % NX) * PL + ny + c / NX];
                g[3 * (size_t)c] = v.x;
                g[3 * (size_t)c + 1] = v.y;
                g[3 * (size_t)c + 2] = v.z;
            }
        }
        __syncthreads();
    }
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Balanced schedule of one launch (McNaughton's wrap-around rule): all n_real * N rod-steps laid
// end to end and cut into gridDim.x equal slices; a rod cut at a slice boundary runs its first
// steps at the start of the next CTA's slice and its last steps at the end of this CTA's slice,
// handed off through global memory.  Up to three segments per CTA {rod, first step offset,
// steps, kind}: kind 0 whole rod, 1 first part (release flags[rod] when done), 2 last part (wait
// for flags[rod] first).  Built on the host and passed as a kernel parameter, so the segment
// fields are uniform constant-bank values: the rod index feeds the Philox round keys, which then
// stay in uniform registers (measured on GB300: a schedule read from shared memory or walked
// on the device cost 6-9 % of the b = 1 rate).
constexpr int kMaxBalancedCtas = 256;
struct BalancedSchedule {
    int4 seg[3 * kMaxBalancedCtas];
};

struct HandoffCtl {
    unsigned long long timeout_ns;  // longest wait for a producer before giving up (status bit 1)
    int withhold;                   // test hook: producers do not release (every wait runs out)
};

// balanced == 0: one rod per CTA over [step0, step0 + n_steps); balanced == 1: the segments of
// `sched` (cooperative launch: all CTAs co-resident).  A wait for a hand-off gives up after
// hc.timeout_ns: status bit 1 is set and the CTA skips its remaining segments.
template <int R, int NX, int NY = 0, int NZ = 0, int SHAPE = -1, bool AX = false>
__global__ void __launch_bounds__(pipelined_max_threads(R), 1) rod_pipelined_nx_kernel(
    KParams p, float *__restrict__ m_glob, long long step0, int n_steps, float *__restrict__ samples,
    int *__restrict__ status, unsigned *__restrict__ flags, int balanced,
    const __grid_constant__ BalancedSchedule sched, HandoffCtl hc)
{
    static_assert(NX >= 3 && NX % 2 == 0, "merged schedule with even plane count");
    extern __shared__ float4 sm4[];
    const int PL = (p.nz + 2) * p.ny;
    for (int i = threadIdx.x; i < (NX + 2) * PL; i += blockDim.x) sm4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    PipelinedRod<R, NX, NY, NZ, SHAPE, AX> w;
    w.setup(sm4, p);
    __syncthreads();
    __shared__ int go;
    const int nseg = balanced ? 3 : 1;
    for (int i = 0; i < nseg; ++i) {
        const int4 sg = balanced ? sched.seg[3 * blockIdx.x + i] : make_int4(blockIdx.x, 0, n_steps, 0);
        if (sg.z <= 0) continue;
        if (sg.w == 2) {
            if (threadIdx.x == 0) {
                const unsigned long long t0 = globaltimer_ns();
                int ok = 1;
                while (ld_acquire_gpu(flags + sg.x) == 0u) {
                    if (globaltimer_ns() - t0 > hc.timeout_ns) {
                        ok = 0;
                        atomicOr(status, 2);
                        break;
                    }
                    __nanosleep(200);
                }
                __threadfence();
                go = ok;
            }
            __syncthreads();
            if (!go) break;
        }
        w.run(p, m_glob, sg.x, step0 + sg.y, sg.z, samples, status);
        if (sg.w == 1 && threadIdx.x == 0 && !hc.withhold) {
            __threadfence();
            st_release_gpu(flags + sg.x, 1u);
        }
    }
}

int round_warp(int n) { return (n + 31) / 32 * 32; }

// Threads of the plane-pipelined kernel for `rows` rows at up to R rows per thread (thread t owns
// rows t, t + T, t + 2T, ...).  Every plane ends in a CTA barrier, so a plane takes as long as the
// busiest of the SM's four schedulers (warp w issues on scheduler w mod 4), whose load is the sum
// of its warps' row counts.  Among the warp counts that fit the register budget (and leave no
// warp without a row), take the one with the smallest busiest-scheduler load, then the fewest row
// slots without a row (each still draws its noise, the draw being outside the row branch), then
// the most warps.  For the b = 1 rod's 1344 rows and R = 3: 15 warps with loads 11/11/11/9
// row-warps per scheduler and 3 idle row slots, instead of 14 warps at 12/12/9/9 (or 16 warps at
// 11/11/10/10 with 6 idle slots).
int pipelined_threads(int rows, int R)
{
    const int wmin = (rows + 32 * R - 1) / (32 * R);
    const int wmax = std::min(pipelined_max_threads(R) / 32, (rows + 31) / 32);
    int best_w = wmin, best_load = 1 << 30, best_idle = 1 << 30;
    for (int w = wmin; w <= wmax; ++w) {
        const int T = 32 * w;
        int load[4] = {0, 0, 0, 0}, idle = 0;
        for (int i = 0; i < w; ++i) {
            const int t = 32 * i;  // a warp's row count is its first thread's
            const int rows_w = std::min(R, (rows - t + T - 1) / T);
            load[i & 3] += rows_w;
            idle += R - rows_w;  // row slots that still draw noise without a row
        }
        const int worst = std::max(std::max(load[0], load[1]), std::max(load[2], load[3]));
        if (worst < best_load || (worst == best_load && idle <= best_idle)) {
            best_load = worst;
            best_idle = idle;
            best_w = w;
        }
    }
    return 32 * best_w;
}

}  // namespace

bool rod_plan(const KParams &p, int n_real, int dev, RodPlan *plan, int force_kind, int force_rods,
              int force_rows, int force_cpt)
{
    int smem_optin = 0, nsm = 0;
    if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return false;
    if (p.periodic != 0) return false;  // rods have free faces
    const size_t rod_pad = (size_t)(p.nx + 2) * (p.ny + 2) * (p.nz + 2);
    const size_t rod_bytes = rod_pad * 2 * sizeof(float4);
    const int rows = p.ny * p.nz;
    const size_t PL = (size_t)(p.nz + 2) * p.ny;
    const size_t pipe_bytes = ((size_t)p.nx + 2) * PL * sizeof(float4);
    const bool twophase_fits = rod_bytes <= (size_t)smem_optin && p.ncells <= 4 * kMaxThreads;
    const bool pipelined_fits = pipe_bytes <= (size_t)smem_optin && rows <= 4 * 672;
    // Default (measured on GB300): the b = 2, 4, 8 rods of the paper's ladder use the row kernel;
    // other rods of at most one CTA of threads the two-phase kernel with one rod per CTA (many
    // small CTAs per SM); larger rods the plane-pipelined kernel.
    int kind = force_kind;
    if (kind == 0)
        kind = rows_supported(p) ? 3 : ((p.ncells <= kMaxThreads && twophase_fits) ? 1 : (pipelined_fits ? 2 : 1));
    if (kind == 3) {
        if (!rows_supported(p)) return false;
        const int maxt = rows_max_threads(p);
        const size_t rbytes = rows_rod_bytes(p);
        const int by_smem = (int)std::max<size_t>(1, (size_t)smem_optin / rbytes);
        int rods = force_rods;
        if (rods == 0) {
            // one rod per CTA (measured on GB300 ahead of packing rods: 608 b = 4 rods at 9.9e10
            // cell-steps/s), unless that leaves over a quarter of the last warp idle (the b = 8
            // rod's 21 rows): then the fewest rods that leave at most a tenth of it
            rods = 1;
            if (4 * (round_warp(rows) - rows) > round_warp(rows))
                for (int r = 2; r * rows <= maxt && r <= by_smem; ++r)
                    if (10 * (round_warp(r * rows) - r * rows) <= round_warp(r * rows)) {
                        rods = r;
                        break;
                    }
        }
        if (rods < 1 || rods > by_smem || round_warp(rods * rows) > maxt) return false;
        plan->kind = 3;
        plan->rods_per_cta = rods;
        plan->cells_per_thread = p.nx;
        plan->threads = round_warp(rods * rows);
        plan->rows_per_thread = 1;
        plan->smem_bytes = rods * rbytes;
        plan->ctas = (n_real + rods - 1) / rods;
        return true;
    }
    if (kind == 1) {
        if (!twophase_fits || p.sample_every >= (1LL << 31)) return false;
        // cells per thread: forced, or the fewest that hold one rod in one CTA
        int cpt = force_cpt;
        if (cpt == 0) {
            cpt = 4;
            for (int c : {2, 1})
                if (round_warp((p.ncells + c - 1) / c) <= twophase_max_threads(p, c)) cpt = c;
        }
        if (cpt != 1 && cpt != 2 && cpt != 4) return false;
        const int maxt = twophase_max_threads(p, cpt);
        const int by_smem = (int)std::max<size_t>(1, (size_t)smem_optin / rod_bytes);
        int rods = 1;
        if (force_rods > 0) rods = force_rods;
        if (rods > by_smem || round_warp((rods * p.ncells + cpt - 1) / cpt) > maxt) return false;
        plan->kind = 1;
        plan->rods_per_cta = rods;
        plan->cells_per_thread = cpt;
        plan->threads = round_warp((rods * p.ncells + cpt - 1) / cpt);
        plan->rows_per_thread = 0;
        plan->smem_bytes = rods * rod_bytes;
        plan->ctas = (n_real + rods - 1) / rods;
        return true;
    }
    if (!pipelined_fits) return false;
    int R = force_rows;
    if (R == 0) {
        // three rows per thread for the b = 1 rod's 1344 rows (448 threads, 128 registers):
        // measured ahead of 672 x 2 rows (which spill at 80 registers) on GB300
        R = rows <= 768 ? 1 : (rows <= 1536 ? 3 : 4);
    }
    if (R < 1 || R > 4 || (rows + R - 1) / R > pipelined_max_threads(R)) return false;
    plan->kind = 2;
    plan->rows_per_thread = R;
    plan->threads = pipelined_threads(rows, R);
    plan->rods_per_cta = 1;
    plan->cells_per_thread = 0;
    plan->smem_bytes = pipe_bytes;
    plan->ctas = n_real;
    return true;
}

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// McNaughton's wrap-around schedule of n_real rods x N steps over G co-resident CTAs; false when
// some CTA's slice would need more than three segments (more than about two waves of rods),
// in which case the launch is not balanced.
static bool balanced_schedule(int n_real, int N, int G, BalancedSchedule *sc)
{
    if (G > kMaxBalancedCtas) return false;
    std::memset(sc, 0, sizeof *sc);
    const long long W = (long long)n_real * N;
    const long long C = (W + G - 1) / G;
    for (int j = 0; j < G; ++j) {
        const long long lo = std::min((long long)j * C, W), hi = std::min(lo + C, W);
        int k = 0;
        for (long long pos = lo; pos < hi;) {
            if (k == 3) return false;
            const long long rod = pos / N, off = pos - rod * N;
            const long long len = std::min(hi, (rod + 1) * N) - pos;
            int4 &g = sc->seg[3 * j + k++];
            g.x = (int)rod;
            g.z = (int)len;
            if (off != 0) {  // first len steps, then hand off
                g.y = 0;
                g.w = 1;
            } else if (len < N) {  // last len steps, after the hand-off
                g.y = (int)(N - len);
                g.w = 2;
            } else {
                g.y = 0;
                g.w = 0;
            }
            pos += len;
        }
    }
    return true;
}

// Launch of the nx-specialised kernel: balanced over a co-resident grid when the rods do not
// divide evenly into waves, else one rod per CTA.
template <int R, int NX, int NY = 0, int NZ = 0, bool AX = false>
static cudaError_t launch_nx(const KParams &p, const RodPlan &plan, float *m, int n_real, long long step0,
                             long long n_steps, float *samples, int *status, unsigned *flags,
                             cudaStream_t st)
{
    auto kern = p.shape == 1 ? rod_pipelined_nx_kernel<R, NX, NY, NZ, 1, AX> : rod_pipelined_nx_kernel<R, NX, NY, NZ, 0, AX>;
    cudaError_t e = set_smem(kern, plan.smem_bytes);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, plan.threads, plan.smem_bytes)) != cudaSuccess)
        return e;
    const int resident = nsm * per_sm;
    BalancedSchedule sched;
    int ns = (int)n_steps;
    HandoffCtl hc{plan.handoff_timeout_ns, plan.withhold_handoff ? 1 : 0};
    if (plan.balance && flags && resident > 0 && n_real > resident && n_real % resident != 0 &&
        balanced_schedule(n_real, ns, resident, &sched)) {
        if ((e = cudaMemsetAsync(flags, 0, sizeof(unsigned) * (size_t)n_real, st)) != cudaSuccess) return e;
        int balanced = 1;
        void *args[] = {(void *)&p, (void *)&m, (void *)&step0, (void *)&ns, (void *)&samples,
                        (void *)&status, (void *)&flags, (void *)&balanced, (void *)&sched, (void *)&hc};
        return cudaLaunchCooperativeKernel((const void *)kern, dim3(resident), dim3(plan.threads), args,
                                           plan.smem_bytes, st);
    }
    kern<<<n_real, plan.threads, plan.smem_bytes, st>>>(p, m, step0, ns, samples, status, flags, 0, sched, hc);
    return cudaGetLastError();
}

cudaError_t rod_advance(const KParams &p, const RodPlan &plan, float *m, int n_real,
                        long long step0, long long n_steps, float *samples, int *status,
                        unsigned *flags, cudaStream_t st)
{
    if (n_steps <= 0) return cudaSuccess;
    // the kernels count the steps of one launch in 32 bits: longer runs are split (the noise and
    // the field are functions of the absolute step index, so the split changes nothing)
    constexpr long long kMaxStepsPerLaunch = 1LL << 30;
    if (n_steps > kMaxStepsPerLaunch) {
        for (long long done = 0; done < n_steps; done += kMaxStepsPerLaunch) {
            const cudaError_t e = rod_advance(p, plan, m, n_real, step0 + done,
                                              std::min(kMaxStepsPerLaunch, n_steps - done), samples, status,
                                              flags, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    cudaError_t e = cudaSuccess;
    if (plan.kind == 1) {
        e = twophase_advance(p, plan, m, n_real, step0, (int)n_steps, samples, status, st);
        if (e != cudaSuccess) return e;
    } else if (plan.kind == 3) {
        e = rows_advance(p, plan, m, n_real, step0, (int)n_steps, samples, status, st);
        if (e != cudaSuccess) return e;
    } else if (plan.kind == 2 && p.axis && plan.rows_per_thread == 3 && p.nx == 8 && p.ny == 24 && p.nz == 56 &&
               !plan.generic) {
        // the b = 1 rod with dispersed axes: the shape-specialised kernel's axis instance
        e = launch_nx<3, 8, 24, 56, true>(p, plan, m, n_real, step0, n_steps, samples, status, flags, st);
        if (e != cudaSuccess) return e;
    } else if (plan.kind == 2) {
#define LLG_PIPELINED(R)                                                                        \
    case R:                                                                                     \
        if (p.axis) {                                                                           \
            e = set_smem(rod_pipelined_kernel<R, true>, plan.smem_bytes);                       \
            if (e != cudaSuccess) return e;                                                     \
            rod_pipelined_kernel<R, true><<<plan.ctas, plan.threads, plan.smem_bytes, st>>>(    \
                p, m, step0, n_steps, samples, status);                                         \
        } else if (p.nx == 8 && p.ny == 24 && p.nz == 56 && !plan.generic) {                    \
            e = launch_nx<R, 8, 24, 56>(p, plan, m, n_real, step0, n_steps, samples, status, flags, st); \
        } else if (p.nx == 8 && !plan.generic) {                                                \
            e = launch_nx<R, 8>(p, plan, m, n_real, step0, n_steps, samples, status, flags, st); \
        } else {                                                                                \
            e = set_smem(rod_pipelined_kernel<R, false>, plan.smem_bytes);                      \
            if (e != cudaSuccess) return e;                                                     \
            rod_pipelined_kernel<R, false><<<plan.ctas, plan.threads, plan.smem_bytes, st>>>(   \
                p, m, step0, n_steps, samples, status);                                         \
        }                                                                                       \
        break;
        switch (plan.rows_per_thread) {
            LLG_PIPELINED(1)
            LLG_PIPELINED(2)
            LLG_PIPELINED(3)
            LLG_PIPELINED(4)
            default:
                return cudaErrorInvalidValue;
        }
#undef LLG_PIPELINED
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace llg
