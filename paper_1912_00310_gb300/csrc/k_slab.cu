// k_slab.cu -- the streaming engine: grids larger than shared memory (the 512x512x56 periodic
// slab) stream through shared memory once per Heun step of Eq. 1.
//
// One launch = one fused Heun step.  The state lives in HBM as float4 (x, y, z, 0) in two
// ping-pong buffers laid out [realisation][z][NY + 4][NX + 4]: every z-plane carries a two-cell
// frame holding the periodic images of the opposite faces (zeros on a free face).  So the
// halo-2 neighbourhood of any (x, y) tile of a plane is one dense rectangle of the padded plane,
// which the Tensor Memory Accelerator copies into shared memory with one instruction (a 5-D
// tiled box: float component, x, y, z, realisation) -- no per-thread staging, no index wrapping.
//
// Each CTA owns an (x, y) tile of columns and sweeps z.  At iteration z it computes, column by
// column, the predictor of plane z and then the corrector of plane z-1 of the same column (the
// corrector needs the predictor of its z+ neighbour, which is that column's value just
// computed), and the predictor of a one-cell ring around the tile (the lateral neighbours the
// corrector needs next iteration).  One elected thread keeps two planes of state in flight: the
// copy of plane z+2 is issued at the start of iteration z into a three-slot ring, each slot with
// an mbarrier that completes when the copy's bytes land; every thread waits on the barrier of the
// plane it reads (with a time limit: a wait that runs out sets a status bit and the CTA stops).
// Three predictor slots rotate with z, so the corrector reads its own and its z- neighbour's
// predictor values from shared memory.  One CTA barrier per plane orders the predictor writes
// before the next plane's corrector reads and frees a state slot before it is refilled.  The
// corrector writes the new state straight to the output buffer, and the cells within two of a
// periodic face also to their images in the frame, so the next step's copies see a complete
// frame.  The z loop is unrolled by three (the three state planes rotate), so the register
// rotation and the slot offsets are compile-time; for the slab's 64 x 27 tiles the plane pitch is
// compile-time too.
//
// The arithmetic, the neighbour order (x-, x+, y-, y+, z-, z+) and the noise keys are those of
// every other engine, so the trajectory is bitwise that of the plain engine on the same grid.
#include <cuda.h>  // CUtensorMap and its enums; the encoder is fetched from the driver at run time

#include <algorithm>
#include <cstring>

#include "llg_internal.h"
#include "physics.cuh"

namespace llg {
namespace {

constexpr int kSlabThreads = 512;
constexpr unsigned long long kStageWaitNs = 2000000000ull;  // longest wait for a staged plane

__device__ __forceinline__ float3 zero3s() { return make_float3(0.f, 0.f, 0.f); }

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `parity` to complete, giving up after kStageWaitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = gtimer_ns();
    while (!mbar_try_wait(bar, parity))
        if (gtimer_ns() - t0 > kStageWaitNs) return false;
    return true;
}

// One box of the padded state: coordinates (float component, x, y, z, realisation).
__device__ __forceinline__ void tma_load_plane(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z,
                                               int r)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)map), "r"(0), "r"(x), "r"(y), "r"(z), "r"(r), "r"(smem_u32(bar))
        : "memory");
}

struct SlabGeom {
    int NX, NY, NZ;
    int NXp, NYp;        // padded extents NX + 4, NY + 4
    int tiles_x, tiles_y;
    int TXmax, TYmax;
    int pitch, rows;     // copied box: (TXmax + 4) x (TYmax + 4) float4
    int slot;            // float4 entries per state slot (box rounded up to 128 bytes)
    int tslot;           // float4 entries per predictor slot (two rows fewer)
    unsigned box_bytes;  // bytes of one copied box
};

__host__ __device__ constexpr int slot_of(int pitch, int rows) { return (pitch * rows + 7) / 8 * 8; }

// Per-CTA state of the z sweep.  PITCH, ROWS > 0: the box geometry at compile time.  NXC > 0:
// the slab's x extent at compile time, with tiles of exactly PITCH - 4 = 64 columns and blockDim.x
// a multiple of 64 -- then the columns of a thread share their x and lie blockDim.x / 64 rows
// apart, so their positions are compile-time strides from the first column's (kept in
// registers for one column only).
template <int CPT, int PITCH, int ROWS, bool AX, int NXC = 0>
struct SlabSweep {
    static constexpr bool kFixed = NXC > 0;
    float4 *Mb, *Tb;     // [3][slot] state planes; [3][tslot] predictor planes (Tb one row early)
    uint64_t *bar;       // [3] one mbarrier per state slot
    int pitch_rt, slot_rt, NZ;
    bool lead;           // the thread that issues the copies
    int tile_x, tile_y, real;
    const CUtensorMap *tin;
    float4 *dst;         // this realisation's output state
    int plane_p;         // float4 entries per padded plane
    uint32_t plane_c;    // cells per interior plane
    PhiloxKeys keys;
    const float4 *axr;
    float Hn, Hn1;
    unsigned long long n;
    int *status;
    // columns of this thread (kFixed: only [0] is kept; column k is [0] plus k row strides)
    int q_[kFixed ? 1 : CPT];          // position in a staged plane
    uint32_t cell_[kFixed ? 1 : CPT];  // interior cell index in plane 0 (+ plane_c per plane)
    int gofs_[kFixed ? 1 : CPT];       // padded position in a plane
    unsigned actm;       // bit k: column k lies in the tile
    unsigned ghost;      // bit k: column k lies within two cells of a periodic face
    __device__ __forceinline__ int q(int k) const
    {
        if constexpr (kFixed) return q_[0] + k * (kSlabThreads / 64) * PITCH;  // rows between columns: 512 / 64
        return q_[k];
    }
    __device__ __forceinline__ uint32_t cell(int k) const
    {
        if constexpr (kFixed) return cell_[0] + (uint32_t)(k * (kSlabThreads / 64) * NXC);
        return cell_[k];
    }
    __device__ __forceinline__ int gofs(int k) const
    {
        if constexpr (kFixed) return gofs_[0] + k * (kSlabThreads / 64) * (NXC + 4);
        return gofs_[k];
    }
    __device__ __forceinline__ bool act(int k) const { return (actm >> k) & 1u; }
    // ring cell of this thread (predictor only)
    int rpos;
    uint32_t rcell;
    bool ract, rin;
    int NX, NY, NXp;
    bool perx, pery;
    // registers carried along z: the own state of plane z-1 (its slot is refilled before the
    // predictor of plane z reads it; the own state of plane z is re-read from its slot) and the
    // corrector's accumulator m + dt/2 f of the last predictor; the thermal field the corrector
    // reuses waits in shared memory (Hs), which keeps the four-column instance in registers
    float3 Sp[CPT], A[CPT];  // own state of the previous plane, accumulator of the last predictor
    float3 rSp;              // the ring cell's state of the previous plane
    float4 *Hs;          // [CPT][blockDim.x] thermal field of the own columns' last predictor

    __device__ __forceinline__ int pitch() const
    {
        if constexpr (PITCH > 0) return PITCH;
        return pitch_rt;
    }
    __device__ __forceinline__ int slot() const
    {
        if constexpr (PITCH > 0) return slot_of(PITCH, ROWS);
        return slot_rt;
    }
    // predictor slots hold only the tile and its one-cell ring: two rows fewer than a state slot,
    // addressed with the state slots' positions through a base one row back (Tb = start - pitch)
    __device__ __forceinline__ int tslot() const
    {
        if constexpr (PITCH > 0) return slot_of(PITCH, ROWS - 2);
        return tslot_rt;
    }
    int tslot_rt;

    unsigned box_bytes;
    int last_issued;  // lead thread: the last plane whose copy was issued

    __device__ __forceinline__ void issue(int z, int s)
    {
        mbar_expect_tx(bar + s, box_bytes);
        tma_load_plane(Mb + s * slot(), tin, bar + s, tile_x, tile_y, z, real);
        last_issued = z;
    }

    // After a staging wait gave up: let the copies still in flight land before the CTA's shared
    // memory is released (each wait bounded).  Plane z used its slot for the (z / 3)-th time.
    __device__ void drain()
    {
        for (int z = max(0, last_issued - 2); z <= last_issued; ++z) mbar_wait(bar + z % 3, (unsigned)((z / 3) & 1));
    }

    // A column's new state goes to its padded position and, near a periodic face, to the images
    // of that position in the frame (x image, y image, corner image).
    __device__ __forceinline__ void store(int k, int zc, float4 v)
    {
        float4 *o = dst + (size_t)zc * plane_p;
        o[gofs(k)] = v;
        if ((ghost >> k) & 1u) {
            const int X = (int)(cell(k) % (uint32_t)NX), Y = (int)(cell(k) / (uint32_t)NX);
            const int gx = (perx && X < 2) ? X + NX + 2 : ((perx && X >= NX - 2) ? X - NX + 2 : -1);
            const int gy = (pery && Y < 2) ? Y + NY + 2 : ((pery && Y >= NY - 2) ? Y - NY + 2 : -1);
            if (gx >= 0) o[(Y + 2) * NXp + gx] = v;
            if (gy >= 0) o[gy * NXp + X + 2] = v;
            if (gx >= 0 && gy >= 0) o[gy * NXp + gx] = v;
        }
    }

    // Iteration z of the sweep, z = 3 j + U: predictor of plane z (z < NZ) and corrector of
    // plane z - 1 (z >= 1).  Ends in a CTA barrier; returns true (in every thread) when some
    // thread's staging wait gave up.
    template <int U>
    __device__ __forceinline__ bool iteration(const KParams &p, int z)
    {
        constexpr int s0 = U % 3, sm1 = (U + 2) % 3, sp1 = (U + 1) % 3;  // slots of planes z, z-1, z+1 (and z-2 = sp1)
        // plane z+1 is the ((z + 1) / 3)-th use of its slot
        const unsigned par_next = (unsigned)(((z + 1) / 3) & 1);
        const int P = pitch();
        const bool pred = z < NZ, corr = z >= 1;
        const bool has_next = z + 1 < NZ;
        int fail = 0;
        // plane z+1, issued an iteration ago
        if (pred && has_next && !mbar_wait(bar + sp1, par_next)) {
            atomicOr(status, 4);
            fail = 1;
        }
        // plane z+2 into the slot plane z-1 left (freed by the previous iteration's barrier)
        if (lead && z + 2 < NZ) issue(z + 2, sm1);
        const float4 *Mz = Mb + s0 * slot(), *Mn = Mb + sp1 * slot();
        float4 *Tw = Tb + s0 * tslot();
        const float4 *Tr = Tb + sm1 * tslot(), *Tp = Tb + sp1 * tslot();
        const uint32_t zoff = plane_c * (uint32_t)z, zcoff = plane_c * (uint32_t)(z - 1);
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
            if (!act(k)) continue;
            const int c = q(k);
            float3 tnew = zero3s(), h = zero3s(), anew = zero3s();
            float4 *hs = Hs + k * blockDim.x + threadIdx.x;
            if (pred) {
                const float3 mcur = xyz(Mz[c]);
                const float3 mnext = has_next ? xyz(Mn[c]) : zero3s();
                h = thermal_field(keys, cell(k) + zoff, n, p.sigma);
                float3 nb = add3(xyz(Mz[c - 1]), xyz(Mz[c + 1]));
                nb = add3(nb, xyz(Mz[c - P]));
                nb = add3(nb, xyz(Mz[c + P]));
                nb = add3(nb, Sp[k]);
                nb = add3(nb, mnext);
                Sp[k] = mcur;
                const float3 u = AX ? xyz(__ldg(axr + cell(k) + zoff)) : zero3s();
                const float3 H = effective_field_sel<AX>(nb, mcur, h, p, Hn, u);
                const float3 sv = llg_torque(mcur, H, p.alpha);
                tnew = normalised(axpy(p.neg_dt_g1, sv, mcur));
                anew = axpy(p.neg_hdt_g1, sv, mcur);
                Tw[c] = pad4(tnew);
            }
            if (corr) {
                const float3 tself = xyz(Tr[c]);
                const float3 tprev = z >= 2 ? xyz(Tp[c]) : zero3s();
                float3 nb = add3(xyz(Tr[c - 1]), xyz(Tr[c + 1]));
                nb = add3(nb, xyz(Tr[c - P]));
                nb = add3(nb, xyz(Tr[c + P]));
                nb = add3(nb, tprev);
                nb = add3(nb, pred ? tnew : zero3s());
                const float3 u = AX ? xyz(__ldg(axr + cell(k) + zcoff)) : zero3s();
                const float3 H = effective_field_sel<AX>(nb, tself, xyz(*hs), p, Hn1, u);
                const float3 s1 = llg_torque(tself, H, p.alpha);
                store(k, z - 1, pad4(normalised(axpy(p.neg_hdt_g1, s1, A[k]))));
            }
            if (pred) {
                *hs = pad4(h);  // after the corrector read the previous plane's
                A[k] = anew;
            }
        }
        if (pred && ract) {
            float3 rt = zero3s();
            if (rin) {
                const float3 rcur = xyz(Mz[rpos]);
                const float3 rnext = has_next ? xyz(Mn[rpos]) : zero3s();
                const float3 h = thermal_field(keys, rcell + zoff, n, p.sigma);
                float3 nb = add3(xyz(Mz[rpos - 1]), xyz(Mz[rpos + 1]));
                nb = add3(nb, xyz(Mz[rpos - P]));
                nb = add3(nb, xyz(Mz[rpos + P]));
                nb = add3(nb, rSp);
                nb = add3(nb, rnext);
                const float3 u = AX ? xyz(__ldg(axr + rcell + zoff)) : zero3s();
                const float3 H = effective_field_sel<AX>(nb, rcur, h, p, Hn, u);
                rt = normalised(axpy(p.neg_dt_g1, llg_torque(rcur, H, p.alpha), rcur));
                rSp = rcur;
            }
            Tw[rpos] = pad4(rt);
        }
        return __syncthreads_or(fail) != 0;
    }
};

template <int CPT, int PITCH, int ROWS, bool AX, int NXC = 0>
__global__ void __launch_bounds__(kSlabThreads, 1) slab_step_kernel(KParams p, SlabGeom G,
                                                                    const __grid_constant__ CUtensorMap tin,
                                                                    float4 *__restrict__ mout, unsigned long long n,
                                                                    int *__restrict__ status)
{
    extern __shared__ __align__(128) float4 sm4[];
    // the copies need a 128-byte aligned destination; refuse (status bit) rather than fault
    if (smem_u32(sm4) & 127u) {
        if (threadIdx.x == 0) atomicOr(status, 4);
        return;
    }
    SlabSweep<CPT, PITCH, ROWS, AX, NXC> w;
    w.pitch_rt = G.pitch;
    w.slot_rt = G.slot;
    w.tslot_rt = G.tslot;
    const int slot = w.slot(), tslot = w.tslot();
    w.Mb = sm4;
    w.Tb = sm4 + 3 * slot - w.pitch();  // row 0 of a predictor slot is row 1 of the box
    w.Hs = sm4 + 3 * slot + 3 * tslot;
    w.bar = reinterpret_cast<uint64_t *>(w.Hs + CPT * blockDim.x);
    w.NZ = G.NZ;
    w.NX = G.NX;
    w.NY = G.NY;
    w.NXp = G.NXp;
    w.perx = p.periodic & 1u;
    w.pery = p.periodic & 2u;
    w.lead = threadIdx.x == 0;
    w.tin = &tin;
    w.box_bytes = G.box_bytes;
    w.n = n;
    w.status = status;
    const int tx = blockIdx.x, ty = blockIdx.y, real = blockIdx.z;
    const int x0 = (int)((long long)tx * G.NX / G.tiles_x), x1 = (int)((long long)(tx + 1) * G.NX / G.tiles_x);
    const int y0 = (int)((long long)ty * G.NY / G.tiles_y), y1 = (int)((long long)(ty + 1) * G.NY / G.tiles_y);
    const int TX = x1 - x0, TY = y1 - y0;
    // the box starts two cells before the tile: padded coordinates (x0, y0)
    w.tile_x = x0;
    w.tile_y = y0;
    w.real = real;
    w.plane_p = G.NXp * G.NYp;
    w.plane_c = (uint32_t)G.NX * (uint32_t)G.NY;
    w.dst = mout + (size_t)real * (size_t)w.plane_p * G.NZ;
    w.keys = philox_keys(p.seed, p.real0 + (uint32_t)real);
    w.axr = AX ? p.axis + (size_t)real * w.plane_c * G.NZ : nullptr;
    {
        Sweep sw;
        sw.init((long long)n, p);
        w.Hn = sw.value();
        sw.inc();
        w.Hn1 = sw.value();
    }
    const int P = w.pitch();
    w.ghost = 0u;
    w.actm = 0u;
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        const int c = threadIdx.x + k * blockDim.x;
        const bool a = c < TX * TY;
        const int cc = a ? c : (int)threadIdx.x;  // an idle slot keeps the first column's position
        const int lx = cc % TX, ly = cc / TX;
        const int X = x0 + lx, Y = y0 + ly;
        if (k == 0 || !w.kFixed) {
            w.q_[w.kFixed ? 0 : k] = (ly + 2) * P + (lx + 2);
            w.cell_[w.kFixed ? 0 : k] = (uint32_t)(X + G.NX * Y);
            w.gofs_[w.kFixed ? 0 : k] = (Y + 2) * G.NXp + (X + 2);
        }
        const bool near = (w.perx && (X < 2 || X >= G.NX - 2)) || (w.pery && (Y < 2 || Y >= G.NY - 2));
        if (a) w.actm |= 1u << k;
        if (a && near) w.ghost |= 1u << k;
    }
    // ring cell (predictor only), counted from the last thread down: the last threads own the
    // fewest interior columns.  Order: the y- row, the y+ row, then x- / x+ pairs by row.
    {
        const int nring = 2 * TX + 2 * TY;
        const int ridx = (int)blockDim.x - 1 - (int)threadIdx.x;
        w.ract = ridx < nring;
        const int i = w.ract ? ridx : 0;
        int lx, ly;
        if (i < 2 * TX) {
            lx = i % TX;
            ly = i < TX ? -1 : TY;
        } else {
            const int j = i - 2 * TX;
            lx = (j & 1) ? TX : -1;
            ly = j >> 1;
        }
        w.rpos = (ly + 2) * P + (lx + 2);
        int gx = x0 + lx, gy = y0 + ly;
        bool in = true;
        if (gx < 0 || gx >= G.NX) {
            in = in && w.perx;
            gx = (gx % G.NX + G.NX) % G.NX;
        }
        if (gy < 0 || gy >= G.NY) {
            in = in && w.pery;
            gy = (gy % G.NY + G.NY) % G.NY;
        }
        w.rin = w.ract && in;
        w.rcell = (uint32_t)(gx + G.NX * gy);
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < 3; ++s) mbar_init(w.bar + s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    w.last_issued = -1;
    if (w.lead) {
        w.issue(0, 0);
        if (G.NZ > 1) w.issue(1, 1);
    }
    // plane 0 before the sweep starts
    int fail = 0;
    if (!mbar_wait(w.bar, 0u)) {
        atomicOr(status, 4);
        fail = 1;
    }
#pragma unroll
    for (int k = 0; k < CPT; ++k) w.Sp[k] = w.A[k] = zero3s();  // plane -1: the free z face
    w.rSp = zero3s();
    bool aborted = __syncthreads_or(fail) != 0;
    for (int zz = 0; zz <= G.NZ && !aborted; zz += 3) {
        aborted = w.template iteration<0>(p, zz);
        if (!aborted && zz + 1 <= G.NZ) aborted = w.template iteration<1>(p, zz + 1);
        if (!aborted && zz + 2 <= G.NZ) aborted = w.template iteration<2>(p, zz + 2);
    }
    if (aborted && w.lead) w.drain();
}

// Pack the AoS float3 state into the padded float4 layout (frame = periodic images or zeros),
// and back.
__global__ void pack_padded_kernel(const float *__restrict__ m, float4 *__restrict__ out, int NX, int NY, int NZ,
                                   unsigned periodic, long long total)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int NXp = NX + 4, NYp = NY + 4;
    const int xp = (int)(i % NXp);
    const long long t = i / NXp;
    const int yp = (int)(t % NYp);
    const long long t2 = t / NYp;
    const int z = (int)(t2 % NZ);
    const long long r = t2 / NZ;
    int x = xp - 2, y = yp - 2;
    bool in = true;
    if (x < 0 || x >= NX) {
        in = in && (periodic & 1u);
        x = (x % NX + NX) % NX;
    }
    if (y < 0 || y >= NY) {
        in = in && (periodic & 2u);
        y = (y % NY + NY) % NY;
    }
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (in) {
        const float *src = m + 3 * ((size_t)r * NX * NY * NZ + (size_t)x + (size_t)NX * (y + (size_t)NY * z));
        v = make_float4(src[0], src[1], src[2], 0.f);
    }
    out[i] = v;
}

__global__ void unpack_padded_kernel(const float4 *__restrict__ in, float *__restrict__ m, int NX, int NY, int NZ,
                                     long long total)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const long long ncell = (long long)NX * NY * NZ;
    const long long r = i / ncell, c = i - r * ncell;
    const int x = (int)(c % NX), y = (int)((c / NX) % NY), z = (int)(c / ((long long)NX * NY));
    const float4 v = in[(size_t)r * (NX + 4) * (NY + 4) * NZ + ((size_t)z * (NY + 4) + (y + 2)) * (NX + 4) + (x + 2)];
    m[3 * i] = v.x;
    m[3 * i + 1] = v.y;
    m[3 * i + 2] = v.z;
}

// Deterministic two-pass mean of m_z per realisation: pass 1 sums fixed contiguous chunks of the
// interior cell index (strided per thread, then a fixed shuffle/shared-memory tree), pass 2 sums
// the chunk partials in order with one warp.
constexpr int kRedBlocks = 256, kRedThreads = 256;

__global__ void slab_partial_kernel(const float4 *__restrict__ m, int NX, int NY, int NZ, float *__restrict__ partial)
{
    const int real = blockIdx.y;
    const long long ncells = (long long)NX * NY * NZ;
    const float4 *mr = m + (size_t)real * (NX + 4) * (NY + 4) * NZ;
    const long long chunk = (ncells + gridDim.x - 1) / gridDim.x;
    const long long a = blockIdx.x * chunk, b = min(ncells, a + chunk);
    float s = 0.f;
    for (long long i = a + threadIdx.x; i < b; i += blockDim.x) {
        const int x = (int)(i % NX), y = (int)((i / NX) % NY), z = (int)(i / ((long long)NX * NY));
        s += mr[((size_t)z * (NY + 4) + (y + 2)) * (NX + 4) + (x + 2)].z;
    }
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

// cuTensorMapEncodeTiled from the driver (no link-time dependency on libcuda).
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder()
{
    static EncodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// Tensor map of a padded state buffer: dims (4 floats, NX + 4, NY + 4, NZ, n_real), box
// (4, pitch, rows, 1, 1); out-of-range elements (past the last tile's box) read as zero.
bool encode_state_map(CUtensorMap *map, float4 *base, const SlabGeom &G, int n_real)
{
    EncodeTiled fn = encoder();
    if (!fn) return false;
    const cuuint64_t dims[5] = {4, (cuuint64_t)G.NXp, (cuuint64_t)G.NYp, (cuuint64_t)G.NZ, (cuuint64_t)n_real};
    const cuuint64_t strides[4] = {16, 16ull * G.NXp, 16ull * G.NXp * G.NYp, 16ull * G.NXp * G.NYp * G.NZ};
    const cuuint32_t box[5] = {4, (cuuint32_t)G.pitch, (cuuint32_t)G.rows, 1, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Compile-time box of the 512 x 512 slab's 64 x 27 tiles.
constexpr int kSpecPitch = 68, kSpecRows = 31, kSpecNX = 512;

template <int C, bool AX>
cudaError_t launch_step(const KParams &p, const SlabGeom &G, const SlabPlan &plan, const CUtensorMap &map,
                        float4 *out, int n_real, unsigned long long n, int *status, cudaStream_t st)
{
    const dim3 grid(G.tiles_x, G.tiles_y, n_real);
    auto go = [&](auto kern) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem_bytes);
        if (e != cudaSuccess) return e;
        kern<<<grid, plan.threads, plan.smem_bytes, st>>>(p, G, map, out, n, status);
        return cudaGetLastError();
    };
    if constexpr (C == 4) {
        // the 512-wide slab in 64 x 27 tiles of 512 threads: every thread's four columns share x
        if (G.pitch == kSpecPitch && G.rows == kSpecRows && G.NX == kSpecNX && G.NX % 64 == 0 &&
            G.tiles_x * 64 == G.NX && plan.threads == kSlabThreads)
            return go(slab_step_kernel<4, kSpecPitch, kSpecRows, AX, kSpecNX>);
        if (G.pitch == kSpecPitch && G.rows == kSpecRows)
            return go(slab_step_kernel<4, kSpecPitch, kSpecRows, AX>);
    }
    return go(slab_step_kernel<C, 0, 0, AX>);
}

}  // namespace

bool slab_plan(const KParams &p, int dev, SlabPlan *plan)
{
    if (p.periodic & 4u) return false;  // free z faces only
    // a periodic axis needs at least four cells, so that each cell has at most one image per axis
    // in the two-cell frame
    if (((p.periodic & 1u) && p.nx < 4) || ((p.periodic & 2u) && p.ny < 4)) return false;
    if (!encoder()) return false;
    int smem_optin = 0, nsm = 0;
    if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return false;
    const int tiles_x = (p.nx + 63) / 64;
    int tiles_y = std::max(1, std::min(p.ny, nsm / tiles_x));
    const int TXmax = (p.nx + tiles_x - 1) / tiles_x;
    int TYmax = (p.ny + tiles_y - 1) / tiles_y;
    // three state slots, three predictor slots, the thermal-field store of every column slot of the
    // CTA, three mbarriers
    auto smem_of = [&](int ty) {
        const int cols = TXmax * ty;
        const int thr = std::min(kSlabThreads, std::max(32, (std::max(cols, 2 * TXmax + 2 * ty) + 31) / 32 * 32));
        const int cpt = (cols + kSlabThreads - 1) / kSlabThreads;
        return (size_t)3 * (slot_of(TXmax + 4, ty + 4) + slot_of(TXmax + 4, ty + 2)) * sizeof(float4) +
               (size_t)cpt * thr * sizeof(float4) + 3 * sizeof(uint64_t);
    };
    while (TYmax > 1 && (TXmax * TYmax > 4 * kSlabThreads || smem_of(TYmax) > (size_t)smem_optin ||
                         TYmax + 4 > 256)) {
        ++tiles_y;
        TYmax = (p.ny + tiles_y - 1) / tiles_y;
    }
    if (TXmax * TYmax > 4 * kSlabThreads || smem_of(TYmax) > (size_t)smem_optin || TXmax + 4 > 256 || TYmax + 4 > 256)
        return false;
    const int cols = TXmax * TYmax;
    const int cpt = (cols + kSlabThreads - 1) / kSlabThreads;
    const int ring = 2 * TXmax + 2 * TYmax;
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

size_t slab_state_float4s(const KParams &p, int n_real)
{
    return (size_t)n_real * (size_t)(p.nx + 4) * (size_t)(p.ny + 4) * (size_t)p.nz;
}

cudaError_t slab_advance(const KParams &p, const SlabPlan &plan, float *m, int n_real, long long step0,
                         long long n_steps, float *samples, int *status, float4 *buf_a, float4 *buf_b,
                         float *partial, cudaStream_t st, long long *launches)
{
    SlabGeom G{};
    G.NX = p.nx;
    G.NY = p.ny;
    G.NZ = p.nz;
    G.NXp = p.nx + 4;
    G.NYp = p.ny + 4;
    G.tiles_x = plan.tiles_x;
    G.tiles_y = plan.tiles_y;
    G.TXmax = plan.TXmax;
    G.TYmax = plan.TYmax;
    G.pitch = plan.TXmax + 4;
    G.rows = plan.TYmax + 4;
    G.slot = slot_of(G.pitch, G.rows);
    G.tslot = slot_of(G.pitch, G.rows - 2);
    G.box_bytes = (unsigned)(G.pitch * G.rows * sizeof(float4));
    CUtensorMap map_a, map_b;
    if (!encode_state_map(&map_a, buf_a, G, n_real) || !encode_state_map(&map_b, buf_b, G, n_real))
        return cudaErrorInvalidValue;
    const long long padded = (long long)slab_state_float4s(p, n_real);
    const long long total = (long long)p.ncells * n_real;
    pack_padded_kernel<<<(unsigned)((padded + 255) / 256), 256, 0, st>>>(m, buf_a, p.nx, p.ny, p.nz, p.periodic,
                                                                         padded);
    // the output buffer's frame: its periodic images are rewritten every step, and a free face's
    // zeros must be there from the start
    pack_padded_kernel<<<(unsigned)((padded + 255) / 256), 256, 0, st>>>(m, buf_b, p.nx, p.ny, p.nz, p.periodic,
                                                                         padded);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    float4 *a = buf_a, *b = buf_b;
    const CUtensorMap *ma = &map_a, *mb = &map_b;
    long long count = 2;
    for (long long s = 0; s < n_steps; ++s) {
        const unsigned long long n = (unsigned long long)(step0 + s);
        switch (plan.cols_per_thread) {
            case 1:
                e = p.axis ? launch_step<1, true>(p, G, plan, *ma, b, n_real, n, status, st)
                           : launch_step<1, false>(p, G, plan, *ma, b, n_real, n, status, st);
                break;
            case 2:
                e = p.axis ? launch_step<2, true>(p, G, plan, *ma, b, n_real, n, status, st)
                           : launch_step<2, false>(p, G, plan, *ma, b, n_real, n, status, st);
                break;
            case 3:
                e = p.axis ? launch_step<3, true>(p, G, plan, *ma, b, n_real, n, status, st)
                           : launch_step<3, false>(p, G, plan, *ma, b, n_real, n, status, st);
                break;
            case 4:
                e = p.axis ? launch_step<4, true>(p, G, plan, *ma, b, n_real, n, status, st)
                           : launch_step<4, false>(p, G, plan, *ma, b, n_real, n, status, st);
                break;
            default:
                return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
        ++count;
        std::swap(a, b);
        std::swap(ma, mb);
        const long long done = (long long)n + 1;
        if (samples && p.sample_every > 0 && done % p.sample_every == 0 && done / p.sample_every < p.n_samples) {
            slab_partial_kernel<<<dim3(kRedBlocks, n_real), kRedThreads, 0, st>>>(a, p.nx, p.ny, p.nz, partial);
            slab_sample_kernel<<<n_real, 32, 0, st>>>(partial, kRedBlocks, p.ncells, done / p.sample_every,
                                                      p.n_samples, samples, status);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            count += 2;
        }
    }
    unpack_padded_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(a, m, p.nx, p.ny, p.nz, total);
    ++count;
    if (launches) *launches += count;
    return cudaGetLastError();
}

size_t slab_partial_floats(int n_real) { return (size_t)kRedBlocks * n_real; }

}  // namespace llg
