// k_plain.cu -- the plain engine: the ensemble state lives in global memory and every Heun step
// of Eq. 1 is one predictor launch and one corrector launch over all (realisation, cell) pairs.
// It is the straightforward form of the method, kept as the per-step baseline against which the
// resident engine is measured, and the engine for periodic grids that do not fit on chip.
//
// Layout: m, mt (predictor), acc (m + dt/2 f(m)), hth (thermal field) are [n_real][ncells][3].
#include "llg_internal.h"
#include "physics.cuh"
#include "reduce.cuh"

namespace llg {
namespace {

__device__ __forceinline__ float3 ld3(const float *p) { return make_float3(p[0], p[1], p[2]); }
__device__ __forceinline__ void st3(float *p, float3 v)
{
    p[0] = v.x;
    p[1] = v.y;
    p[2] = v.z;
}

// sum_j m_j over the six face neighbours, added in the fixed order x-, x+, y-, y+, z-, z+ (the
// order every engine uses); a missing neighbour at a free face contributes an exact zero.
__device__ __forceinline__ float3 neighbour_sum(const float *s, int x, int y, int z, const KParams &p)
{
    const int d[3] = {p.nx, p.ny, p.nz};
    const int stride[3] = {1, p.nx, p.nx * p.ny};
    const int c[3] = {x, y, z};
    const int self = x + p.nx * (y + p.ny * z);
    float3 v[6];
#pragma unroll
    for (int axis = 0; axis < 3; ++axis) {
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int dir = side ? 1 : -1;
            const int q = c[axis] + dir;
            int j = self + dir * stride[axis];
            bool ok = q >= 0 && q < d[axis];
            if (!ok && (p.periodic >> axis & 1u)) {
                ok = true;
                j += (q < 0 ? d[axis] : -d[axis]) * stride[axis];
            }
            v[2 * axis + side] = ok ? ld3(s + 3 * (size_t)j) : make_float3(0.f, 0.f, 0.f);
        }
    }
    return add3(add3(add3(add3(add3(v[0], v[1]), v[2]), v[3]), v[4]), v[5]);
}

__device__ __forceinline__ float field_at(const KParams &p, unsigned long long n)
{
    Sweep sw;
    sw.init((long long)n, p);
    return sw.value();
}

__global__ void plain_pred_kernel(KParams p, const float *__restrict__ m, float *__restrict__ mt,
                                  float *__restrict__ acc, float *__restrict__ hth, int n_real,
                                  unsigned long long n)
{
    const float Hz = field_at(p, n);
    const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gid >= (long long)n_real * p.ncells) return;
    const int r = (int)(gid / p.ncells);
    const int i = (int)(gid - (long long)r * p.ncells);
    const int x = i % p.nx, y = (i / p.nx) % p.ny, z = i / (p.nx * p.ny);
    const float *mr = m + (size_t)r * p.ncells * 3;
    const float3 mi = ld3(mr + 3 * (size_t)i);
    const float3 nb = neighbour_sum(mr, x, y, z, p);
    const float3 h = thermal_field(p.seed, p.real0 + (uint32_t)r, (uint32_t)i, n, p.sigma);
    const float3 H = p.axis ? effective_field_axis(nb, mi, h, p.c_ex, p.c_an, Hz, xyz(__ldg(p.axis + gid)))
                            : effective_field(nb, mi, h, p.c_ex, p.c_an, Hz);
    const float3 s0 = llg_torque(mi, H, p.alpha);
    st3(mt + 3 * gid, normalised(axpy(p.neg_dt_g1, s0, mi)));
    st3(acc + 3 * gid, axpy(p.neg_hdt_g1, s0, mi));
    st3(hth + 3 * gid, h);
}

__global__ void plain_corr_kernel(KParams p, float *__restrict__ m, const float *__restrict__ mt,
                                  const float *__restrict__ acc, const float *__restrict__ hth,
                                  int n_real, unsigned long long n)
{
    const float Hz1 = field_at(p, n + 1);
    const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gid >= (long long)n_real * p.ncells) return;
    const int r = (int)(gid / p.ncells);
    const int i = (int)(gid - (long long)r * p.ncells);
    const int x = i % p.nx, y = (i / p.nx) % p.ny, z = i / (p.nx * p.ny);
    const float *tr = mt + (size_t)r * p.ncells * 3;
    const float3 ti = ld3(tr + 3 * (size_t)i);
    const float3 nb = neighbour_sum(tr, x, y, z, p);
    const float3 h = ld3(hth + 3 * gid);
    const float3 H = p.axis ? effective_field_axis(nb, ti, h, p.c_ex, p.c_an, Hz1, xyz(__ldg(p.axis + gid)))
                            : effective_field(nb, ti, h, p.c_ex, p.c_an, Hz1);
    const float3 s1 = llg_torque(ti, H, p.alpha);
    st3(m + 3 * gid, normalised(axpy(p.neg_hdt_g1, s1, ld3(acc + 3 * gid))));
}

// One warp per realisation: the canonical cell-average of m_z (see reduce.cuh).
__global__ void plain_sample_kernel(KParams p, const float *__restrict__ m, int n_real, long long k,
                                    float *__restrict__ samples, int *__restrict__ status)
{
    const int r = blockIdx.x;
    const float *mr = m + (size_t)r * p.ncells * 3;
    float part = 0.f;
    for (int c = threadIdx.x; c < p.ncells; c += 32) part += mr[3 * (size_t)c + 2];
    const float mean = warp_cell_mean(part, p.ncells);
    if (threadIdx.x == 0) {
        samples[(size_t)r * p.n_samples + k] = mean;
        if (!isfinite(mean)) atomicOr(status, 1);
    }
}

__global__ void axis_fill_kernel(float4 *__restrict__ ax, int n_real, int ncells, uint32_t seed,
                                 uint32_t real0, float w_max)
{
    const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (gid >= (long long)n_real * ncells) return;
    const int r = (int)(gid / ncells);
    const int c = (int)(gid - (long long)r * ncells);
    ax[gid] = pad4(easy_axis(seed, real0 + (uint32_t)r, (uint32_t)c, w_max));
}

__global__ void fill_column_kernel(float *a, int rows, long long ld, long long col, float v)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < rows) a[(size_t)r * ld + col] = v;
}

constexpr int kThreads = 256;

unsigned blocks_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

cudaError_t plain_predictor(const KParams &p, const float *m, float *mt, float *acc, float *hth,
                            int n_real, long long n, cudaStream_t st)
{
    plain_pred_kernel<<<blocks_for((long long)n_real * p.ncells), kThreads, 0, st>>>(
        p, m, mt, acc, hth, n_real, (unsigned long long)n);
    return cudaGetLastError();
}

cudaError_t plain_corrector(const KParams &p, float *m, const float *mt, const float *acc,
                            const float *hth, int n_real, long long n, cudaStream_t st)
{
    plain_corr_kernel<<<blocks_for((long long)n_real * p.ncells), kThreads, 0, st>>>(
        p, m, mt, acc, hth, n_real, (unsigned long long)n);
    return cudaGetLastError();
}

cudaError_t plain_sample(const KParams &p, const float *m, int n_real, long long k, float *samples,
                         int *status, cudaStream_t st)
{
    plain_sample_kernel<<<n_real, 32, 0, st>>>(p, m, n_real, k, samples, status);
    return cudaGetLastError();
}

cudaError_t fill_column(float *a, int rows, long long ld, long long col, float v, cudaStream_t st)
{
    if (rows <= 0) return cudaSuccess;
    fill_column_kernel<<<(rows + 255) / 256, 256, 0, st>>>(a, rows, ld, col, v);
    return cudaGetLastError();
}

cudaError_t axis_fill(float4 *ax, int n_real, int ncells, uint32_t seed, uint32_t real0, float w_max,
                      cudaStream_t st)
{
    const long long n = (long long)n_real * ncells;
    if (n <= 0) return cudaSuccess;
    axis_fill_kernel<<<blocks_for(n), kThreads, 0, st>>>(ax, n_real, ncells, seed, real0, w_max);
    return cudaGetLastError();
}

cudaError_t plain_advance(const KParams &p, float *m, float *mt, float *acc, float *hth, int n_real,
                          long long step0, long long n_steps, float *samples, int *status,
                          cudaStream_t st, long long *launches)
{
    long long count = 0;
    for (long long s = 0; s < n_steps; ++s) {
        const long long n = step0 + s;
        cudaError_t e = plain_predictor(p, m, mt, acc, hth, n_real, n, st);
        if (e != cudaSuccess) return e;
        e = plain_corrector(p, m, mt, acc, hth, n_real, n, st);
        if (e != cudaSuccess) return e;
        count += 2;
        const long long done = n + 1;
        if (samples && p.sample_every > 0 && done % p.sample_every == 0 &&
            done / p.sample_every < p.n_samples) {
            e = plain_sample(p, m, n_real, done / p.sample_every, samples, status, st);
            if (e != cudaSuccess) return e;
            ++count;
        }
    }
    if (launches) *launches += count;
    return cudaSuccess;
}

}  // namespace llg
