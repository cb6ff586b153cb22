// k_noalloc.cu -- allocation-free entry point of the plain engine.
//
// Some callers cannot call cudaMalloc: code that runs while a stream is being captured into a
// CUDA graph (allocation is not a capturable operation), hosts whose device memory is owned by
// another allocator that must see every allocation, and real-time loops that cannot afford the
// device-wide synchronisation an allocation may cause.  For them this file keeps the plain
// engine's scratch (the predictor state, the m + dt/2 f(m) accumulator and the thermal field of
// every cell, plus a status word) in one fixed array in device global memory that is part of the
// library image: every GPU that loads the library holds it until the process exits, and no call
// here allocates anything.  The caller passes the state and the sample buffer.
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/llg.h"
#include "llg_internal.h"

namespace {

// Scratch of the allocation-free entry point: 9 floats per (realisation, cell) for the
// predictor state, the accumulator and the thermal field, after a 256-byte header whose first
// word is the status flag.
constexpr size_t kHeaderFloats = 64;
constexpr size_t kScratchFloats = kHeaderFloats + 9 * (size_t)LLG_NOALLOC_MAX_CELL_REALISATIONS;
static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
float *g_scratch_addr[kMaxDevices] = {};

llg_status error(llg_status st, const char *fmt, ...)
{
    char msg[256];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    llg::set_last_error(msg);
    return st;
}

// Device address of the scratch array on `device` (the current device), looked up once.
cudaError_t scratch_address(int device, float **out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = static_cast<float *>(p);
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

// True when p is device memory of `device` (or managed memory): host pointers and other
// devices' memory are refused before anything is enqueued.
bool on_device(const void *p, int device)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

}  // namespace

extern "C" llg_status llg_plain_advance_noalloc(const llg_ctx *ctx, float *m, int n_real, uint32_t seed,
                                                uint32_t real_offset, int64_t step0, int64_t n_steps,
                                                float *m_samples, void *cuda_stream, int *status_out)
{
    if (!ctx || !m || n_real < 1 || step0 < 0 || n_steps < 0)
        return error(LLG_EINVAL, "need a context, a state, n_real >= 1, step0 >= 0, n_steps >= 0");
    // host-side parameter setup from the context (no device work, no allocation)
    llg::KParams kp;
    const llg_status s = llg::kparams_from_ctx(ctx, &kp);
    if (s != LLG_OK) return s;
    const long long ncells = llg_num_cells(ctx);
    if ((long long)n_real * ncells > (long long)LLG_NOALLOC_MAX_CELL_REALISATIONS)
        return error(LLG_EINVAL,
                     "%d realisations x %lld cells exceed the allocation-free scratch of %d cell-realisations",
                     n_real, ncells, LLG_NOALLOC_MAX_CELL_REALISATIONS);
    // The work runs on the current device, which must be the context's; the state and the
    // sample buffer must be that device's memory (another GPU's pointer would be dereferenced
    // without peer access).
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return error(LLG_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (device != llg::ctx_device(ctx))
        return error(LLG_EINVAL, "the current device (%d) is not the context's device (%d)", device,
                     llg::ctx_device(ctx));
    if (!on_device(m, device) || (m_samples && !on_device(m_samples, device)))
        return error(LLG_EINVAL, "m and m_samples must be device memory of device %d", device);
    const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // status_out needs a device-to-host read and a stream synchronisation, which a stream that is
    // being captured cannot take
    if (status_out) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
            cudaGetLastError();
            return error(LLG_EINVAL, "status_out must be NULL while the stream is being captured");
        }
    }
    if (device < 0 || device >= kMaxDevices) return error(LLG_EINVAL, "device ordinal %d too large", device);
    float *base = nullptr;
    e = scratch_address(device, &base);
    if (e != cudaSuccess) return error(LLG_ECUDA, "scratch set-up: %s", cudaGetErrorString(e));
    kp.seed = seed;
    kp.real0 = real_offset;
    int *status = reinterpret_cast<int *>(base);
    float *work = base + kHeaderFloats;
    const size_t per = (size_t)n_real * (size_t)ncells * 3;
    // the status word must start at zero; the other scratch is written before it is read
    e = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (e == cudaSuccess)
        e = llg::plain_advance(kp, m, work, work + per, work + 2 * per, n_real, step0, n_steps, m_samples,
                               status, st, nullptr);
    if (e == cudaSuccess && status_out) {
        e = cudaMemcpyAsync(status_out, status, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) return error(LLG_ECUDA, "plain engine: %s", cudaGetErrorString(e));
    return LLG_OK;
}
