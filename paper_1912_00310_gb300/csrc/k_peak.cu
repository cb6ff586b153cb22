// k_peak.cu -- issue-rate microbenchmarks of the SM's 32-bit lanes, the denominator of the
// resident and streaming kernels' ALU roofline (those kernels are bound by the issue of 32-bit
// integer and floating-point lane operations, not by memory).
//
//   ffma kernel: every thread runs eight independent FP32 fused multiply-add chains, so the
//                FMA pipe is never waiting on a dependency; lane-ops = threads x 8 x unroll x iters.
//   int kernel:  the integer mix of the thermal-noise generator (Philox4x32-10 rounds: a 32x32->64
//                product counted as two lane operations, 3-input xors, key bumps), in four
//                independent streams per thread; counted with the same rule as the algorithmic
//                lane-op count of a cell-step.
//
// Each CTA also reads the SM clock counter and the global timer at its start and end, so the
// effective SM clock during the measurement is reported beside the rate (read, never set).
#include <algorithm>
#include <cstdio>
#include <vector>

#include "../../include/llg.h"
#include "llg_internal.h"

namespace llg {
namespace {

constexpr int kPeakThreads = 1024;
constexpr int kUnroll = 16;

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(kPeakThreads) ffma_kernel(float *out, int iters, unsigned long long *clk)
{
    const unsigned long long c0 = clock64(), t0 = gtimer();
    float a[8];
    const float x = 0.9999f, y = 1e-4f * (float)(threadIdx.x & 7);
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = (float)(threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int j = 0; j < 8; ++j) a[j] = fmaf(a[j], x, y);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    if (s == 12345.678f) out[threadIdx.x] = s;  // keeps the chains live
    if (threadIdx.x == 0) {
        clk[2 * blockIdx.x] = clock64() - c0;
        clk[2 * blockIdx.x + 1] = gtimer() - t0;
    }
}

// One Philox-style round on four independent counters: per counter two 32x32->64 products (four
// lane-ops) and two 3-input xors (four lane-ops), and the key bump (two lane-ops per round, shared by
// the four counters) -- the counting rule of the algorithmic lane-op count of a cell-step.
__global__ void __launch_bounds__(kPeakThreads) int_kernel(unsigned *out, int iters, unsigned long long *clk)
{
    const unsigned long long c0 = clock64(), t0 = gtimer();
    unsigned c[4][4];
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int j = 0; j < 4; ++j) c[s][j] = threadIdx.x * 2654435761u + (unsigned)(s * 4 + j);
    unsigned k0 = blockIdx.x, k1 = ~blockIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const unsigned long long p0 = (unsigned long long)0xD2511F53u * c[s][0];
                const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c[s][2];
                const unsigned n0 = (unsigned)(p1 >> 32) ^ c[s][1] ^ k0;
                const unsigned n2 = (unsigned)(p0 >> 32) ^ c[s][3] ^ k1;
                c[s][0] = n0;
                c[s][1] = (unsigned)p1;
                c[s][2] = n2;
                c[s][3] = (unsigned)p0;
            }
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
    }
    unsigned r = 0;
#pragma unroll
    for (int s = 0; s < 4; ++s) r ^= c[s][0] ^ c[s][1] ^ c[s][2] ^ c[s][3];
    if (r == 0x12345678u) out[threadIdx.x] = r;
    if (threadIdx.x == 0) {
        clk[2 * blockIdx.x] = clock64() - c0;
        clk[2 * blockIdx.x + 1] = gtimer() - t0;
    }
}

}  // namespace
}  // namespace llg

extern "C" llg_status llg_measure_alu_peak(int device, double out[4])
{
    if (!out) {
        llg::set_last_error("out is NULL");
        return LLG_EINVAL;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        llg::set_last_error("invalid device");
        return LLG_EINVAL;
    }
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    const int blocks = 2 * nsm;  // two CTAs of 1024 threads per SM: 64 warps, 16 per scheduler
    void *buf = nullptr;
    unsigned long long *clk = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    llg_status status = LLG_OK;
    char msg[160] = "";
    auto ck = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && status == LLG_OK) {
            std::snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString(e));
            status = LLG_ECUDA;
        }
        return status == LLG_OK;
    };
    ck(cudaMalloc(&buf, sizeof(float) * llg::kPeakThreads), "cudaMalloc");
    ck(cudaMalloc(&clk, sizeof(unsigned long long) * 2 * (size_t)blocks), "cudaMalloc");
    ck(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream");
    ck(cudaEventCreate(&e0), "event");
    ck(cudaEventCreate(&e1), "event");
    std::vector<unsigned long long> hc(2 * (size_t)blocks);
    // best of five timed launches of each kernel after a warm-up, ~tens of ms each
    auto measure = [&](int which, int iters, double ops_per_iter, double *rate, double *mhz) {
        double best = 0.0, best_mhz = 0.0;
        for (int rep = 0; rep < 6 && status == LLG_OK; ++rep) {
            ck(cudaEventRecord(e0, st), "record");
            if (which == 0)
                llg::ffma_kernel<<<blocks, llg::kPeakThreads, 0, st>>>(static_cast<float *>(buf), iters, clk);
            else
                llg::int_kernel<<<blocks, llg::kPeakThreads, 0, st>>>(static_cast<unsigned *>(buf), iters, clk);
            ck(cudaGetLastError(), "launch");
            ck(cudaEventRecord(e1, st), "record");
            if (!ck(cudaEventSynchronize(e1), "sync")) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ck(cudaMemcpy(hc.data(), clk, sizeof(unsigned long long) * hc.size(), cudaMemcpyDeviceToHost), "copy");
            if (rep == 0) continue;  // warm-up
            const double r = ops_per_iter * iters * (double)blocks * llg::kPeakThreads / (ms * 1e-3);
            std::vector<double> f;
            for (int b = 0; b < blocks; ++b)
                if (hc[2 * (size_t)b + 1] > 0) f.push_back((double)hc[2 * (size_t)b] / (double)hc[2 * (size_t)b + 1] * 1e3);
            std::sort(f.begin(), f.end());
            if (r > best) {
                best = r;
                best_mhz = f.empty() ? 0.0 : f[f.size() / 2];
            }
        }
        *rate = best;
        *mhz = best_mhz;
    };
    double ffma = 0, ffma_mhz = 0, integer = 0, int_mhz = 0;
    // FFMA: 8 chains x 16 per iteration; integer: 4 rounds x (4 counters x 8 lane-ops + 2 key bumps)
    measure(0, 32768, 8.0 * llg::kUnroll, &ffma, &ffma_mhz);
    measure(1, 16384, 4.0 * (4.0 * 8.0 + 2.0), &integer, &int_mhz);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(buf);
    cudaFree(clk);
    if (prev >= 0) cudaSetDevice(prev);
    if (status != LLG_OK) {
        llg::set_last_error(msg);
        return status;
    }
    out[0] = ffma;
    out[1] = ffma_mhz;
    out[2] = integer;
    out[3] = int_mhz;
    return LLG_OK;
}
