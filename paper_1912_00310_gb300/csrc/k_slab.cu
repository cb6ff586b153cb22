// k_slab.cu -- the streaming engine: grids larger than shared memory (the 512x512x56 periodic
// slab) stream through shared memory once per Heun step of Eq. 1.
//
// One launch = one fused Heun step.  The state lives in HBM as float4 (x, y, z, 0) in two
// ping-pong buffers.  Each CTA owns an (x, y) tile of columns and sweeps z: at iteration z it
// computes the predictor of plane z on the tile plus a one-cell ring (the ring's predictor values
// are the lateral neighbours the corrector needs) and the corrector of plane z-1 on the tile,
// writing the new state straight to the output buffer.  State planes with a two-cell halo are
// staged by 16-byte asynchronous copies (cp.async) into a ring of three plane buffers, so the
// load of plane z+2 overlaps the arithmetic of plane z.  Three predictor planes rotate with z, so
// the corrector re-reads the predictor values of its own cell and of its z- neighbour instead of
// carrying them in registers (which spilled at four columns per thread).
// HBM traffic per cell-step: one read of the state (plus the tile halo, mostly served by L2) and
// one write.  Periodic x and y faces wrap; z faces are free.  The arithmetic, the neighbour order
// (x-, x+, y-, y+, z-, z+) and the noise keys are those of every other engine, so the trajectory
// is bitwise that of the plain engine on the same grid.
#include <algorithm>

#include "llg_internal.h"
#include "physics.cuh"

namespace llg {
namespace {

constexpr int kSlabThreads = 512;

__device__ __forceinline__ float3 zero3s() { return make_float3(0.f, 0.f, 0.f); }

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

struct SlabGeom {
    int NX, NY, NZ;
    int tiles_x, tiles_y;
    int TXmax, TYmax;  // largest tile extents (the shared-memory pitch is TXmax + 4)
};

// Wrapped (periodic) or rejected (free face) coordinate.
__device__ __forceinline__ bool wrap(int &v, int n, bool periodic)
{
    if (v >= 0 && v < n) return true;
    if (!periodic) return false;
    v %= n;  // halos reach two cells out, more than the extent of a one- or two-cell axis
    if (v < 0) v += n;
    return true;
}

template <int CPT, bool AX>
__global__ void __launch_bounds__(kSlabThreads, 1) slab_step_kernel(KParams p, SlabGeom G,
                                                                    const float4 *__restrict__ min,
                                                                    float4 *__restrict__ mout,
                                                                    unsigned long long n)
{
    extern __shared__ float4 sm4[];
    const int tx = blockIdx.x, ty = blockIdx.y, real = blockIdx.z;
    const int x0 = (int)((long long)tx * G.NX / G.tiles_x), x1 = (int)((long long)(tx + 1) * G.NX / G.tiles_x);
    const int y0 = (int)((long long)ty * G.NY / G.tiles_y), y1 = (int)((long long)(ty + 1) * G.NY / G.tiles_y);
    const int TX = x1 - x0, TY = y1 - y0;
    const int pitch = G.TXmax + 4;                 // halo-2 planes
    const int mplane = pitch * (G.TYmax + 4);
    float4 *Mb = sm4;                               // [3][mplane] state planes
    float4 *Tb = sm4 + 3 * mplane;                  // [3][mplane] predictor planes (same geometry)
                                                    // then the staging table (int2 per position)
    const bool perx = p.periodic & 1u, pery = p.periodic & 2u;
    const size_t plane_cells = (size_t)G.NX * G.NY;
    const float4 *src = min + (size_t)real * plane_cells * G.NZ;
    float4 *dst = mout + (size_t)real * plane_cells * G.NZ;
    const PhiloxKeys keys = philox_keys(p.seed, p.real0 + (uint32_t)real);
    const float4 *axr = AX ? p.axis + (size_t)real * plane_cells * G.NZ : nullptr;  // easy axes
    Sweep sw;
    sw.init((long long)n, p);
    const float Hn = sw.value();
    sw.inc();
    const float Hn1 = sw.value();

    // Staging table of this tile, built once: for every halo-2 position (smem offset in a plane,
    // offset of its cell in a global plane or -1 outside a free face).  Each plane load is then a
    // table read and a 16-byte asynchronous copy per position.
    int2 *desc = reinterpret_cast<int2 *>(Tb + 3 * mplane);
    const int w = TX + 4, h = TY + 4, npos = w * h;
    for (int i = threadIdx.x; i < npos; i += blockDim.x) {
        const int lx = i % w - 2, ly = i / w - 2;
        int gx = x0 + lx, gy = y0 + ly;
        const bool in = wrap(gx, G.NX, perx) && wrap(gy, G.NY, pery);
        desc[i] = make_int2((ly + 2) * pitch + (lx + 2), in ? gy * G.NX + gx : -1);
    }
    __syncthreads();
    auto load_plane = [&](int z, int b) {
        float4 *dstp = Mb + b * mplane;
        const float4 *srcp = src + (size_t)z * plane_cells;
        for (int i = threadIdx.x; i < npos; i += blockDim.x) {
            const int2 d = desc[i];
            if (d.y >= 0)
                cp_async16(dstp + d.x, srcp + d.y);
            else
                dstp[d.x] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        cp_async_commit();
    };

    // interior columns of this thread
    int pos[CPT];    // offset in a plane (halo-2 geometry)
    uint32_t cell[CPT];
    bool act[CPT];
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        const int c = threadIdx.x + k * blockDim.x;
        act[k] = c < TX * TY;
        const int cc = act[k] ? c : 0;
        const int lx = cc % TX, ly = cc / TX;
        pos[k] = (ly + 2) * pitch + (lx + 2);
        cell[k] = (uint32_t)((x0 + lx) + G.NX * (y0 + ly));  // + NX*NY*z per plane
    }
    // the ring cell of this thread (predictor only), counted from the last thread down: the last
    // threads own the fewest interior columns
    const int nring = 2 * (TX + 2) + 2 * TY;
    const int ridx = (int)blockDim.x - 1 - (int)threadIdx.x;
    const bool ract = ridx < nring;
    int rpos = 0;
    uint32_t rcell = 0;
    bool rin = false;
    {
        const int i = ract ? ridx : 0;
        int lx, ly;
        if (i < 2 * (TX + 2)) {
            lx = i % (TX + 2) - 1;
            ly = i < TX + 2 ? -1 : TY;
        } else {
            const int j = i - 2 * (TX + 2);
            lx = (j & 1) ? TX : -1;
            ly = j >> 1;
        }
        rpos = (ly + 2) * pitch + (lx + 2);
        int gx = x0 + lx, gy = y0 + ly;
        rin = ract && wrap(gx, G.NX, perx) && wrap(gy, G.NY, pery);
        rcell = (uint32_t)(gx + G.NX * gy);
    }

    // per column: the state at z-1 and z for the predictor, the corrector's accumulator and
    // thermal field one plane behind; the predictor values of planes z-2 and z-1 the corrector
    // needs are re-read from the three predictor slots (fewer registers than carrying them)
    float3 mA[CPT], mB[CPT], acc[CPT], hth[CPT];
#pragma unroll
    for (int k = 0; k < CPT; ++k) mA[k] = mB[k] = acc[k] = hth[k] = zero3s();
    float3 rA = zero3s(), rB = zero3s();

    load_plane(0, 0);
    if (G.NZ > 1) load_plane(1, 1);  // with one plane, plane 1 is never read (free z face)
    cp_async_wait_all();
    __syncthreads();
    // m(0) of the own columns
#pragma unroll
    for (int k = 0; k < CPT; ++k)
        if (act[k]) mB[k] = xyz(Mb[pos[k]]);
    if (rin) rB = xyz(Mb[rpos]);

    for (int z = 0; z <= G.NZ; ++z) {
        if (z > 0) {
            cp_async_wait_all();  // plane z+1, issued one iteration ago
            __syncthreads();
        }
        if (z + 2 < G.NZ) load_plane(z + 2, (z + 2) % 3);  // reuses the buffer of plane z-1
        float3 tnew[CPT], anew[CPT], hnew[CPT];
        if (z < G.NZ) {
            const float4 *Mz = Mb + (z % 3) * mplane;
            const float4 *Mn = Mb + ((z + 1) % 3) * mplane;
            float4 *Tw = Tb + (z % 3) * mplane;
            const bool has_next = z + 1 < G.NZ;
            const uint32_t zoff = (uint32_t)(plane_cells * (size_t)z);
#pragma unroll
            for (int k = 0; k < CPT; ++k) {
                if (!act[k]) continue;
                const int q = pos[k];
                const float3 mnext = has_next ? xyz(Mn[q]) : zero3s();
                hnew[k] = thermal_field(keys, cell[k] + zoff, n, p.sigma);
                float3 nb = add3(xyz(Mz[q - 1]), xyz(Mz[q + 1]));
                nb = add3(nb, xyz(Mz[q - pitch]));
                nb = add3(nb, xyz(Mz[q + pitch]));
                nb = add3(nb, mA[k]);
                nb = add3(nb, mnext);
                const float3 u = AX ? xyz(__ldg(axr + cell[k] + zoff)) : zero3s();
                const float3 H = effective_field_sel<AX>(nb, mB[k], hnew[k], p, Hn, u);
                const float3 s0 = llg_torque(mB[k], H, p.alpha);
                tnew[k] = normalised(axpy(p.neg_dt_g1, s0, mB[k]));
                anew[k] = axpy(p.neg_hdt_g1, s0, mB[k]);
                Tw[q] = pad4(tnew[k]);
                mA[k] = mB[k];
                mB[k] = mnext;
            }
            if (ract) {
                float3 rt = zero3s();
                const float3 rnext = (rin && has_next) ? xyz(Mn[rpos]) : zero3s();
                if (rin) {
                    const int q = rpos;
                    const float3 h = thermal_field(keys, rcell + zoff, n, p.sigma);
                    float3 nb = add3(xyz(Mz[q - 1]), xyz(Mz[q + 1]));
                    nb = add3(nb, xyz(Mz[q - pitch]));
                    nb = add3(nb, xyz(Mz[q + pitch]));
                    nb = add3(nb, rA);
                    nb = add3(nb, rnext);
                    const float3 u = AX ? xyz(__ldg(axr + rcell + zoff)) : zero3s();
                    const float3 H = effective_field_sel<AX>(nb, rB, h, p, Hn, u);
                    rt = normalised(axpy(p.neg_dt_g1, llg_torque(rB, H, p.alpha), rB));
                }
                Tw[rpos] = pad4(rt);
                rA = rB;
                rB = rnext;
            }
        }
        if (z > 0) {
            const int zc = z - 1;
            const float4 *Tr = Tb + (zc % 3) * mplane;
            const float4 *Tp = Tb + ((zc + 2) % 3) * mplane;  // plane zc - 1 (read only when zc > 0)
            const bool has_next = z < G.NZ;
            float4 *out = dst + plane_cells * (size_t)zc;
#pragma unroll
            for (int k = 0; k < CPT; ++k) {
                if (!act[k]) continue;
                const int t = pos[k];
                const float3 tnext = has_next ? tnew[k] : zero3s();
                const float3 tprev = zc > 0 ? xyz(Tp[t]) : zero3s();
                const float3 tself = xyz(Tr[t]);
                float3 nb = add3(xyz(Tr[t - 1]), xyz(Tr[t + 1]));
                nb = add3(nb, xyz(Tr[t - pitch]));
                nb = add3(nb, xyz(Tr[t + pitch]));
                nb = add3(nb, tprev);
                nb = add3(nb, tnext);
                const float3 u = AX ? xyz(__ldg(axr + cell[k] + plane_cells * (size_t)zc)) : zero3s();
                const float3 H = effective_field_sel<AX>(nb, tself, hth[k], p, Hn1, u);
                const float3 s1 = llg_torque(tself, H, p.alpha);
                out[cell[k]] = pad4(normalised(axpy(p.neg_hdt_g1, s1, acc[k])));
            }
        }
        if (z < G.NZ) {
#pragma unroll
            for (int k = 0; k < CPT; ++k) {
                acc[k] = anew[k];
                hth[k] = hnew[k];
            }
        }
        __syncthreads();
    }
}

// Pack the AoS float3 state into float4 and back.
__global__ void pack4_kernel(const float *__restrict__ m, float4 *__restrict__ out, long long n)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float4(m[3 * i], m[3 * i + 1], m[3 * i + 2], 0.f);
}

__global__ void unpack4_kernel(const float4 *__restrict__ in, float *__restrict__ m, long long n)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) {
        const float4 v = in[i];
        m[3 * i] = v.x;
        m[3 * i + 1] = v.y;
        m[3 * i + 2] = v.z;
    }
}

// Deterministic two-pass mean of m_z per realisation: pass 1 sums fixed contiguous chunks
// (strided per thread, then a fixed shuffle/shared-memory tree), pass 2 sums the chunk partials in
// order with one warp.
constexpr int kRedBlocks = 256, kRedThreads = 256;

__global__ void slab_partial_kernel(const float4 *__restrict__ m, long long ncells, float *__restrict__ partial)
{
    const int real = blockIdx.y;
    const float4 *mr = m + (size_t)real * ncells;
    const long long chunk = (ncells + gridDim.x - 1) / gridDim.x;
    const long long a = blockIdx.x * chunk, b = min(ncells, a + chunk);
    float s = 0.f;
    for (long long i = a + threadIdx.x; i < b; i += blockDim.x) s += mr[i].z;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    __shared__ float ws[kRedThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < kRedThreads / 32; ++w) t += ws[w];
        partial[(size_t)real * gridDim.x + blockIdx.x] = t;
    }
}

__global__ void slab_sample_kernel(const float *__restrict__ partial, int nparts, long long ncells,
                                   long long k, long long n_samples, float *__restrict__ samples,
                                   int *__restrict__ status)
{
    const int real = blockIdx.x;
    float s = 0.f;
    for (int i = threadIdx.x; i < nparts; i += 32) s += partial[(size_t)real * nparts + i];
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0) {
        const float mean = (float)((double)s / (double)ncells);
        samples[(size_t)real * n_samples + k] = mean;
        if (!isfinite(mean)) atomicOr(status, 1);
    }
}

}  // namespace

bool slab_plan(const KParams &p, int dev, SlabPlan *plan)
{
    if (p.periodic & 4u) return false;  // free z faces only
    int smem_optin = 0, nsm = 0;
    if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return false;
    const int tiles_x = (p.nx + 63) / 64;
    int tiles_y = std::max(1, std::min(p.ny, nsm / tiles_x));
    const int TXmax = (p.nx + tiles_x - 1) / tiles_x;
    int TYmax = (p.ny + tiles_y - 1) / tiles_y;
    // keep the columns per thread within the compiled variants and the shared memory within
    // the opt-in limit
    auto smem_of = [&](int ty) {
        return (size_t)6 * (TXmax + 4) * (ty + 4) * sizeof(float4) + (size_t)(TXmax + 4) * (ty + 4) * sizeof(int2);
    };
    while (TYmax > 1 && (TXmax * TYmax > 4 * kSlabThreads || smem_of(TYmax) > (size_t)smem_optin)) {
        ++tiles_y;
        TYmax = (p.ny + tiles_y - 1) / tiles_y;
    }
    if (TXmax * TYmax > 4 * kSlabThreads || smem_of(TYmax) > (size_t)smem_optin) return false;
    // All kSlabThreads threads once a tile has more columns than that (more warps at the same
    // register budget; the last threads, with one column fewer, take the predictor ring).
    const int cols = TXmax * TYmax;
    const int cpt = (cols + kSlabThreads - 1) / kSlabThreads;
    const int ring = 2 * (TXmax + 2) + 2 * TYmax;
    const int threads = std::min(kSlabThreads, std::max(32, (std::max(cols, ring) + 31) / 32 * 32));
    if (ring > threads) return false;
    plan->tiles_x = tiles_x;
    plan->tiles_y = tiles_y;
    plan->TXmax = TXmax;
    plan->TYmax = TYmax;
    plan->cols_per_thread = cpt;
    plan->threads = threads;
    plan->smem_bytes = smem_of(TYmax);
    return true;
}

cudaError_t slab_advance(const KParams &p, const SlabPlan &plan, float *m, int n_real, long long step0,
                         long long n_steps, float *samples, int *status, float4 *buf_a, float4 *buf_b,
                         float *partial, cudaStream_t st, long long *launches)
{
    const long long ncell = (long long)p.ncells;
    const long long total = ncell * n_real;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    pack4_kernel<<<blocks, 256, 0, st>>>(m, buf_a, total);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    SlabGeom G{p.nx, p.ny, p.nz, plan.tiles_x, plan.tiles_y, plan.TXmax, plan.TYmax};
    const dim3 grid(plan.tiles_x, plan.tiles_y, n_real);
    float4 *a = buf_a, *b = buf_b;
    long long count = 1;
#define LLG_SLAB(C)                                                                                   \
    case C:                                                                                           \
        if (p.axis) {                                                                                 \
            e = cudaFuncSetAttribute(slab_step_kernel<C, true>,                                       \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem_bytes); \
            if (e != cudaSuccess) return e;                                                           \
            slab_step_kernel<C, true><<<grid, plan.threads, plan.smem_bytes, st>>>(p, G, a, b, n);    \
        } else {                                                                                      \
            e = cudaFuncSetAttribute(slab_step_kernel<C, false>,                                      \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem_bytes); \
            if (e != cudaSuccess) return e;                                                           \
            slab_step_kernel<C, false><<<grid, plan.threads, plan.smem_bytes, st>>>(p, G, a, b, n);   \
        }                                                                                             \
        break;
    for (long long s = 0; s < n_steps; ++s) {
        const long long n = step0 + s;
        switch (plan.cols_per_thread) {
            LLG_SLAB(1)
            LLG_SLAB(2)
            LLG_SLAB(3)
            LLG_SLAB(4)
            default:
                return cudaErrorInvalidValue;
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ++count;
        std::swap(a, b);
        const long long done = n + 1;
        if (samples && p.sample_every > 0 && done % p.sample_every == 0 && done / p.sample_every < p.n_samples) {
            slab_partial_kernel<<<dim3(kRedBlocks, n_real), kRedThreads, 0, st>>>(a, ncell, partial);
            slab_sample_kernel<<<n_real, 32, 0, st>>>(partial, kRedBlocks, ncell, done / p.sample_every,
                                                      p.n_samples, samples, status);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            count += 2;
        }
    }
#undef LLG_SLAB
    unpack4_kernel<<<blocks, 256, 0, st>>>(a, m, total);
    ++count;
    if (launches) *launches += count;
    return cudaGetLastError();
}

size_t slab_partial_floats(int n_real) { return (size_t)kRedBlocks * n_real; }

}  // namespace llg
