// k_rod_small.cu -- the resident engine's two-phase kernel, for rods whose state and predictor
// state both fit in shared memory with room for several rods per CTA (b >= 2 in the paper's
// ladder: 4x12x28, 2x6x14, 1x3x7 cells).
//
// Each rod is padded by a zero ghost layer so the 6-neighbour stencil has no branches.  Per Heun
// step: every thread takes the thermal field of its cells (drawn before the previous barrier),
// computes the predictor into the P buffer and keeps m + dt/2 f(m) in registers; barrier; the
// corrector reads P and overwrites M, then draws the next step's thermal field; barrier.  A
// thread owns CPT cells (t, t + T, t + 2T, ... of the CTA's rods), so the per-step bookkeeping
// is shared by CPT cell-updates.
//
// Instances: the b = 4 and b = 8 rods with their shape at compile time (every stencil offset an
// immediate), the sweep shape at compile time with its phase and the sample countdown in 32 bits
// (loops of fewer than 2^31 steps), and a register budget that grows with CPT (launch bound
// 768 / CPT threads); and, for any other grid, a runtime-shape instance with 64-bit sweep
// bookkeeping.  All use the neighbour order x-, x+, y-, y+, z-, z+ and the physics.cuh arithmetic
// of every other engine, so their trajectories are bitwise those of the plain engine.
#include <algorithm>

#include "llg_internal.h"
#include "physics.cuh"
#include "reduce.cuh"
#include "sweep32.cuh"

namespace llg {
namespace {

constexpr int kMaxThreads = 768;

__device__ __forceinline__ float3 zero3t() { return make_float3(0.f, 0.f, 0.f); }

// Rod extents: NXC > 0 at compile time, else from the kernel parameters.
template <int NXC, int NYC, int NZC>
struct RodDims {
    int nx_, ny_, nz_;
    __device__ __forceinline__ int nx() const { if constexpr (NXC > 0) return NXC; return nx_; }
    __device__ __forceinline__ int ny() const { if constexpr (NYC > 0) return NYC; return ny_; }
    __device__ __forceinline__ int nz() const { if constexpr (NZC > 0) return NZC; return nz_; }
    __device__ __forceinline__ int ncell() const { return nx() * ny() * nz(); }
    __device__ __forceinline__ int sy() const { return nx() + 2; }
    __device__ __forceinline__ int sz() const { return (nx() + 2) * (ny() + 2); }
    __device__ __forceinline__ int pad() const { return sz() * (nz() + 2); }
    // position of cell c (x + nx (y + ny z)) in a ghost-padded rod
    __device__ __forceinline__ int at(int c) const
    {
        const int x = c % nx(), y = (c / nx()) % ny(), z = c / (nx() * ny());
        return (x + 1) + sy() * (y + 1) + sz() * (z + 1);
    }
};

// Shared memory: M[tot] and P[tot] float4 (x, y, z, 0), tot = rods_per_cta * padded rod.
template <int CPT, bool AX, int SHAPE, int NXC, int NYC, int NZC, int MAXT>
__global__ void __launch_bounds__(MAXT) rod_twophase_kernel(KParams p, float *__restrict__ m_glob, int n_real,
                                                            int rods_per_cta, long long step0, int n_steps,
                                                            float *__restrict__ samples, int *__restrict__ status)
{
    extern __shared__ float4 sm4[];
    RodDims<NXC, NYC, NZC> D{p.nx, p.ny, p.nz};
    const int sy = D.sy(), sz = D.sz();
    const int rod_pad = D.pad();
    const int rod0 = blockIdx.x * rods_per_cta;
    const int nrod = min(rods_per_cta, n_real - rod0);
    const int tot = rods_per_cta * rod_pad;
    float4 *M = sm4, *P = sm4 + tot;
    const int T = blockDim.x;
    const int ncell = D.ncell();
    const int cta_cells = nrod * ncell;

    for (int i = threadIdx.x; i < 2 * tot; i += T) sm4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    for (int i = threadIdx.x; i < cta_cells; i += T) {
        const int rod = i / ncell, c = i - rod * ncell;
        const float *g = m_glob + ((size_t)(rod0 + rod) * ncell + c) * 3;
        M[rod * rod_pad + D.at(c)] = make_float4(g[0], g[1], g[2], 0.f);
    }

    int pidx[CPT];
    uint32_t cell[CPT], real[CPT];
    bool act[CPT];
    float3 uax[CPT];  // easy axes (dispersed-axis mode only)
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        const int i = threadIdx.x + k * T;
        act[k] = i < cta_cells;
        const int ii = act[k] ? i : 0;
        const int rod = ii / ncell, c = ii - rod * ncell;
        pidx[k] = rod * rod_pad + D.at(c);
        cell[k] = (uint32_t)c;
        real[k] = p.real0 + (uint32_t)(rod0 + rod);
        uax[k] = zero3t();
        if constexpr (AX) {
            if (act[k]) uax[k] = xyz(__ldg(p.axis + (size_t)(rod0 + rod) * ncell + c));
        }
    }
    __syncthreads();

    typename SweepSel<SHAPE>::type field;
    field.init(step0, p);
    float Hn = field.value();
    // steps to the next sample (32-bit countdown; the host keeps sample_every below 2^31)
    const long long se = p.sample_every;
    const bool sampling = samples && se > 0;
    long long k_next = sampling ? step0 / se + 1 : 0;
    int to_sample = sampling ? (int)(k_next * se - step0) : -1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = T >> 5;

    // thermal field of the next step, drawn before the barrier that ends the current one
    float3 hpre[CPT];
#pragma unroll
    for (int k = 0; k < CPT; ++k) hpre[k] = thermal_field(p.seed, real[k], cell[k], (unsigned long long)step0, p.sigma);
    unsigned long long n = (unsigned long long)step0;
    for (int s = 0; s < n_steps; ++s, ++n) {
        field.inc();
        const float Hn1 = field.value();
        float3 acc[CPT], hth[CPT];
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            if (!act[k]) continue;
            const int q = pidx[k];
            hth[k] = hpre[k];
            const float3 mi = xyz(M[q]);
            float3 nb = add3(xyz(M[q - 1]), xyz(M[q + 1]));
            nb = add3(nb, xyz(M[q - sy]));
            nb = add3(nb, xyz(M[q + sy]));
            nb = add3(nb, xyz(M[q - sz]));
            nb = add3(nb, xyz(M[q + sz]));
            const float3 H = effective_field_sel<AX>(nb, mi, hth[k], p, Hn, uax[k]);
            const float3 s0 = llg_torque(mi, H, p.alpha);
            P[q] = pad4(normalised(axpy(p.neg_dt_g1, s0, mi)));
            acc[k] = axpy(p.neg_hdt_g1, s0, mi);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            if (!act[k]) continue;
            const int q = pidx[k];
            const float3 ti = xyz(P[q]);
            float3 nb = add3(xyz(P[q - 1]), xyz(P[q + 1]));
            nb = add3(nb, xyz(P[q - sy]));
            nb = add3(nb, xyz(P[q + sy]));
            nb = add3(nb, xyz(P[q - sz]));
            nb = add3(nb, xyz(P[q + sz]));
            const float3 H = effective_field_sel<AX>(nb, ti, hth[k], p, Hn1, uax[k]);
            const float3 s1 = llg_torque(ti, H, p.alpha);
            M[q] = pad4(normalised(axpy(p.neg_hdt_g1, s1, acc[k])));
            hpre[k] = thermal_field(p.seed, real[k], cell[k], n + 1, p.sigma);
        }
        __syncthreads();
        Hn = Hn1;
        if (--to_sample == 0) {
            // M now holds the state after step n; the next phase only reads M until the
            // barrier that precedes its next write, so no extra barrier is needed here.
            to_sample = (int)se;
            const long long k = k_next++;
            if (k < p.n_samples) {
                for (int rod = warp; rod < nrod; rod += nwarps) {
                    float part = 0.f;
                    for (int c = lane; c < ncell; c += 32) part += M[rod * rod_pad + D.at(c)].z;
                    const float mean = warp_cell_mean(part, ncell);
                    if (lane == 0) {
                        samples[(size_t)(rod0 + rod) * p.n_samples + k] = mean;
                        if (!isfinite(mean)) atomicOr(status, 1);
                    }
                }
            }
        }
    }

    for (int i = threadIdx.x; i < cta_cells; i += T) {
        const int rod = i / ncell, c = i - rod * ncell;
        const float4 v = M[rod * rod_pad + D.at(c)];
        float *g = m_glob + ((size_t)(rod0 + rod) * ncell + c) * 3;
        g[0] = v.x;
        g[1] = v.y;
        g[2] = v.z;
    }
}

// ------------------------------------------------------------------------------------------
// Row kernel (the b = 2, 4, 8 rods: 4x12x28, 2x6x14, 1x3x7 cells, shapes at compile time).  A
// thread owns one x-row (fixed y, z) of NX cells and keeps the row's state, predictor, corrector
// accumulator and thermal field in registers; the x-neighbours come from registers, the y- and
// z-neighbours from shared memory.  Shared memory holds per rod, for each x, a plane of rows
// (y, z) with ghost lines at y = -1, NY and z = -1, NZ: M[x][(z + 1)(NY + 2) + y + 1] and the same
// for the predictor P, so consecutive threads (consecutive y) read consecutive float4s.  Per
// step: predictor of the row into P, barrier, corrector into M, next thermal fields, barrier --
// 8 shared loads per cell-step where the ghost-padded one-cell-per-thread layout needed 14.
// The row's cells share their rod's Philox round keys, computed once per thread.
// ------------------------------------------------------------------------------------------
template <int NX, int NY, int NZ, int SHAPE, bool AX, int MAXT>
__global__ void __launch_bounds__(MAXT) rod_rows_kernel(KParams p, float *__restrict__ m_glob, int n_real,
                                                        int rods_per_cta, long long step0, int n_steps,
                                                        float *__restrict__ samples, int *__restrict__ status)
{
    constexpr int PY = NY + 2;                   // pitch of a row plane (ghost columns in y)
    constexpr int PLANE = (NZ + 2) * PY;         // one x-plane with ghost lines
    constexpr int ROD = NX * PLANE;              // one buffer of one rod
    constexpr int ROWS = NY * NZ, NCELL = NX * ROWS;
    extern __shared__ float4 sm4[];
    const int rod0 = blockIdx.x * rods_per_cta;
    const int nrod = min(rods_per_cta, n_real - rod0);
    float4 *M = sm4, *P = sm4 + rods_per_cta * ROD;
    const int T = blockDim.x;
    for (int i = threadIdx.x; i < 2 * rods_per_cta * ROD; i += T) sm4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    // this thread's row
    const int t = threadIdx.x;
    const int rl = t / ROWS, row = t - rl * ROWS;  // rod within the CTA, row y + NY z
    const bool act = t < nrod * ROWS;
    const int y = row % NY, z = row / NY;
    const int q = rl * ROD + (z + 1) * PY + (y + 1);  // row position in plane x = 0 of its rod
    const uint32_t cbase = (uint32_t)(row * NX);      // cell index of x = 0: x + NX (y + NY z)
    const uint32_t real = p.real0 + (uint32_t)(rod0 + rl);
    float3 m[NX], u[NX];
#pragma unroll
    for (int x = 0; x < NX; ++x) {
        m[x] = u[x] = zero3t();
        if (act) {
            const float *g = m_glob + ((size_t)(rod0 + rl) * NCELL + cbase + x) * 3;
            m[x] = make_float3(g[0], g[1], g[2]);
            M[q + x * PLANE] = pad4(m[x]);
            if constexpr (AX) u[x] = xyz(__ldg(p.axis + (size_t)(rod0 + rl) * NCELL + cbase + x));
        }
    }
    const PhiloxKeys keys = philox_keys(p.seed, act ? real : p.real0);
    __syncthreads();

    typename SweepSel<SHAPE>::type field;
    field.init(step0, p);
    float Hn = field.value();
    const long long se = p.sample_every;
    const bool sampling = samples && se > 0;
    long long k_next = sampling ? step0 / se + 1 : 0;
    int to_sample = sampling ? (int)(k_next * se - step0) : -1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = T >> 5;

    // thermal field of the next step, drawn before the barrier that ends the current one
    float3 hpre[NX];
#pragma unroll
    for (int x = 0; x < NX; ++x) hpre[x] = thermal_field(keys, cbase + x, (unsigned long long)step0, p.sigma);
    unsigned long long n = (unsigned long long)step0;
    for (int s = 0; s < n_steps; ++s, ++n) {
        field.inc();
        const float Hn1 = field.value();
        float3 mt[NX], acc[NX], hth[NX];
        if (act) {
#pragma unroll
            for (int x = 0; x < NX; ++x) {
                const float4 *Mx = M + q + x * PLANE;
                hth[x] = hpre[x];
                float3 nb = add3(x > 0 ? m[x - 1] : zero3t(), x + 1 < NX ? m[x + 1] : zero3t());
                nb = add3(nb, xyz(Mx[-1]));
                nb = add3(nb, xyz(Mx[1]));
                nb = add3(nb, xyz(Mx[-PY]));
                nb = add3(nb, xyz(Mx[PY]));
                const float3 H = effective_field_sel<AX>(nb, m[x], hth[x], p, Hn, u[x]);
                const float3 s0 = llg_torque(m[x], H, p.alpha);
                mt[x] = normalised(axpy(p.neg_dt_g1, s0, m[x]));
                acc[x] = axpy(p.neg_hdt_g1, s0, m[x]);
                P[q + x * PLANE] = pad4(mt[x]);
            }
        }
        __syncthreads();
        if (act) {
#pragma unroll
            for (int x = 0; x < NX; ++x) {
                const float4 *Px = P + q + x * PLANE;
                float3 nb = add3(x > 0 ? mt[x - 1] : zero3t(), x + 1 < NX ? mt[x + 1] : zero3t());
                nb = add3(nb, xyz(Px[-1]));
                nb = add3(nb, xyz(Px[1]));
                nb = add3(nb, xyz(Px[-PY]));
                nb = add3(nb, xyz(Px[PY]));
                const float3 H = effective_field_sel<AX>(nb, mt[x], hth[x], p, Hn1, u[x]);
                const float3 s1 = llg_torque(mt[x], H, p.alpha);
                m[x] = normalised(axpy(p.neg_hdt_g1, s1, acc[x]));
                M[q + x * PLANE] = pad4(m[x]);
            }
#pragma unroll
            for (int x = 0; x < NX; ++x) hpre[x] = thermal_field(keys, cbase + x, n + 1, p.sigma);
        }
        __syncthreads();
        Hn = Hn1;
        if (--to_sample == 0) {
            // M holds the state after step n; the next phase only reads M until the barrier that
            // precedes its next write
            to_sample = (int)se;
            const long long k = k_next++;
            if (k < p.n_samples) {
                for (int r = warp; r < nrod; r += nwarps) {
                    float part = 0.f;
                    for (int c = lane; c < NCELL; c += 32) {
                        const int cx = c % NX, cr = c / NX;
                        part += M[r * ROD + cx * PLANE + (cr / NY + 1) * PY + (cr % NY + 1)].z;
                    }
                    const float mean = warp_cell_mean(part, NCELL);
                    if (lane == 0) {
                        samples[(size_t)(rod0 + r) * p.n_samples + k] = mean;
                        if (!isfinite(mean)) atomicOr(status, 1);
                    }
                }
            }
        }
    }
    if (act) {
#pragma unroll
        for (int x = 0; x < NX; ++x) {
            float *g = m_glob + ((size_t)(rod0 + rl) * NCELL + cbase + x) * 3;
            g[0] = m[x].x;
            g[1] = m[x].y;
            g[2] = m[x].z;
        }
    }
}

template <typename K>
cudaError_t launch(K kern, const KParams &p, const RodPlan &plan, float *m, int n_real, long long step0, int n_steps,
                   float *samples, int *status, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem_bytes);
    if (e != cudaSuccess) return e;
    kern<<<plan.ctas, plan.threads, plan.smem_bytes, st>>>(p, m, n_real, plan.rods_per_cta, step0, n_steps, samples,
                                                           status);
    return cudaGetLastError();
}

// the compile-time rod shape and sweep shape instance, CPT cells per thread
template <int CPT, int NX, int NY, int NZ>
cudaError_t launch_shaped(const KParams &p, const RodPlan &plan, float *m, int n_real, long long step0, int n_steps,
                          float *samples, int *status, cudaStream_t st)
{
    constexpr int MAXT = kMaxThreads / CPT;
    if (p.axis)
        return p.shape == 1 ? launch(rod_twophase_kernel<CPT, true, 1, NX, NY, NZ, MAXT>, p, plan, m, n_real, step0,
                                     n_steps, samples, status, st)
                            : launch(rod_twophase_kernel<CPT, true, 0, NX, NY, NZ, MAXT>, p, plan, m, n_real, step0,
                                     n_steps, samples, status, st);
    return p.shape == 1 ? launch(rod_twophase_kernel<CPT, false, 1, NX, NY, NZ, MAXT>, p, plan, m, n_real, step0,
                                 n_steps, samples, status, st)
                        : launch(rod_twophase_kernel<CPT, false, 0, NX, NY, NZ, MAXT>, p, plan, m, n_real, step0,
                                 n_steps, samples, status, st);
}

template <int CPT>
cudaError_t launch_generic(const KParams &p, const RodPlan &plan, float *m, int n_real, long long step0, int n_steps,
                           float *samples, int *status, cudaStream_t st)
{
    if (p.axis)
        return launch(rod_twophase_kernel<CPT, true, -1, 0, 0, 0, kMaxThreads>, p, plan, m, n_real, step0, n_steps,
                      samples, status, st);
    return launch(rod_twophase_kernel<CPT, false, -1, 0, 0, 0, kMaxThreads>, p, plan, m, n_real, step0, n_steps,
                  samples, status, st);
}

template <int NX, int NY, int NZ, int MAXT>
cudaError_t launch_rows_shaped(const KParams &p, const RodPlan &plan, float *m, int n_real, long long step0,
                               int n_steps, float *samples, int *status, cudaStream_t st)
{
    if (p.axis)
        return p.shape == 1 ? launch(rod_rows_kernel<NX, NY, NZ, 1, true, MAXT>, p, plan, m, n_real, step0, n_steps,
                                     samples, status, st)
                            : launch(rod_rows_kernel<NX, NY, NZ, 0, true, MAXT>, p, plan, m, n_real, step0, n_steps,
                                     samples, status, st);
    return p.shape == 1 ? launch(rod_rows_kernel<NX, NY, NZ, 1, false, MAXT>, p, plan, m, n_real, step0, n_steps,
                                 samples, status, st)
                        : launch(rod_rows_kernel<NX, NY, NZ, 0, false, MAXT>, p, plan, m, n_real, step0, n_steps,
                                 samples, status, st);
}

// the rows kernel's shapes: b = 2, 4, 8 rods (x-rows of 4, 2, 1 cells)
int rows_shape(const KParams &p)
{
    if (p.nx == 4 && p.ny == 12 && p.nz == 28) return 2;
    if (p.nx == 2 && p.ny == 6 && p.nz == 14) return 4;
    if (p.nx == 1 && p.ny == 3 && p.nz == 7) return 8;
    return 0;
}

}  // namespace

bool rows_supported(const KParams &p)
{
    const long long period = p.shape == 1 ? p.period : 2 * p.n_half;
    return rows_shape(p) != 0 && (p.shape == 0 || p.shape == 1) && period < (1LL << 31) &&
           p.sample_every < (1LL << 31);
}

// Largest CTA of the rows kernel: 768 threads (85 registers) for rows of 1 or 2 cells, 384 (170
// registers) for the 4-cell rows of the b = 2 rod.
int rows_max_threads(const KParams &p) { return p.nx == 4 ? 384 : kMaxThreads; }

size_t rows_rod_bytes(const KParams &p)
{
    return (size_t)2 * p.nx * (p.nz + 2) * (p.ny + 2) * sizeof(float4);
}

cudaError_t rows_advance(const KParams &p, const RodPlan &plan, float *m, int n_real, long long step0, int n_steps,
                         float *samples, int *status, cudaStream_t st)
{
    switch (rows_shape(p)) {
        case 2:
            return launch_rows_shaped<4, 12, 28, 384>(p, plan, m, n_real, step0, n_steps, samples, status, st);
        case 4:
            return launch_rows_shaped<2, 6, 14, kMaxThreads>(p, plan, m, n_real, step0, n_steps, samples, status, st);
        case 8:
            return launch_rows_shaped<1, 3, 7, kMaxThreads>(p, plan, m, n_real, step0, n_steps, samples, status, st);
        default:
            return cudaErrorInvalidValue;
    }
}

// Largest CTA of a two-phase instance: the compile-time-shape instances (b = 4 and b = 8 rods)
// give CPT cells per thread a register budget of 768 / CPT threads; the runtime-shape instance
// keeps 768 threads for every CPT.
int twophase_max_threads(const KParams &p, int cpt)
{
    return twophase_shaped(p) ? kMaxThreads / cpt : kMaxThreads;
}

bool twophase_shaped(const KParams &p)
{
    const bool b4 = p.nx == 2 && p.ny == 6 && p.nz == 14, b8 = p.nx == 1 && p.ny == 3 && p.nz == 7;
    const long long period = p.shape == 1 ? p.period : 2 * p.n_half;
    return (b4 || b8) && (p.shape == 0 || p.shape == 1) && period < (1LL << 31) && p.sample_every < (1LL << 31);
}

cudaError_t twophase_advance(const KParams &p, const RodPlan &plan, float *m, int n_real, long long step0,
                             int n_steps, float *samples, int *status, cudaStream_t st)
{
    if (twophase_shaped(p)) {
        const bool b4 = p.nx == 2;
        switch (plan.cells_per_thread) {
            case 1:
                return b4 ? launch_shaped<1, 2, 6, 14>(p, plan, m, n_real, step0, n_steps, samples, status, st)
                          : launch_shaped<1, 1, 3, 7>(p, plan, m, n_real, step0, n_steps, samples, status, st);
            case 2:
                return b4 ? launch_shaped<2, 2, 6, 14>(p, plan, m, n_real, step0, n_steps, samples, status, st)
                          : launch_shaped<2, 1, 3, 7>(p, plan, m, n_real, step0, n_steps, samples, status, st);
            case 4:
                return b4 ? launch_shaped<4, 2, 6, 14>(p, plan, m, n_real, step0, n_steps, samples, status, st)
                          : launch_shaped<4, 1, 3, 7>(p, plan, m, n_real, step0, n_steps, samples, status, st);
            default:
                return cudaErrorInvalidValue;
        }
    }
    switch (plan.cells_per_thread) {
        case 1:
            return launch_generic<1>(p, plan, m, n_real, step0, n_steps, samples, status, st);
        case 2:
            return launch_generic<2>(p, plan, m, n_real, step0, n_steps, samples, status, st);
        case 4:
            return launch_generic<4>(p, plan, m, n_real, step0, n_steps, samples, status, st);
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace llg
