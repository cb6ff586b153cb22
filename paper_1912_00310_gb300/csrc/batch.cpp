// batch.cpp -- the batching layer and the autotuner of the resident engine.
//
// llg_run_batch: uneven jobs (rods of different size b, sweep rates and damping, each job a
// context with its own ensemble) advance together in ONE launch: a CUDA graph with one kernel
// node per job on independent branches, so the hardware runs the jobs' CTAs side by side and the
// small-rod CTAs fill the wave tails of the large ones.  Jobs are ordered longest first (the
// block scheduler starts branches roughly in capture order).  Each call captures the graph of
// its launches (cheap) and refreshes a cached instantiation of the same job set with
// cudaGraphExecUpdate (an instantiation costs hundreds of microseconds); a request of more steps
// than the jobs' steps per launch (LLG_TUNE_CHUNK_STEPS, chosen by the autotuner) runs as several
// graph launches.  Within a batch, b = 1 rods run one rod per CTA: the balanced wrap-around
// schedule needs all CTAs of its launch co-resident (a cooperative launch), which inside a batch
// would hold the whole GPU and serialise the other jobs, whose CTAs fill the tails instead.
//
// llg_autotune: times the resident engine's launch shapes (rows per thread of the
// plane-pipelined kernel, rods per CTA and cells per thread of the two-phase kernel) on a scratch
// copy of a context's ensemble and keeps the fastest, cached per (device, grid, realisation
// count); it also sets the steps per launch so that the launch overhead, measured as the time of
// a one-step launch less one step, stays near 1% of a launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/llg.h"
#include "llg_internal.h"

namespace {

// Autotuned launch shapes, keyed by what selects the kernel instances: the device, the grid, the
// ensemble size, the sweep shape, whether the sweep and sample bookkeeping fit 32 bits, dispersed
// axes and the periodic faces.
struct TuneKey {
    std::string device;
    int nx, ny, nz, n_real, shape, fits32, axes, periodic;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(device, nx, ny, nz, n_real, shape, fits32, axes, periodic) <
               std::tie(o.device, o.nx, o.ny, o.nz, o.n_real, o.shape, o.fits32, o.axes, o.periodic);
    }
};
struct TuneValue {
    int kind, rods, rows, cpt;
    long long chunk;
    double rate;
};
std::mutex g_tune_mutex;
std::map<TuneKey, TuneValue> g_tune_cache;

// Instantiated batch graphs, keyed by the device and the ordered list of job contexts with
// steps to run (least recently used dropped beyond kGraphCache entries).
constexpr size_t kGraphCache = 8;
struct GraphEntry {
    std::vector<const void *> key;
    cudaGraphExec_t exec;
    unsigned long long used;
};
std::mutex g_graph_mutex;
std::vector<GraphEntry> g_graphs;
unsigned long long g_graph_clock = 0;

// An executable graph for `graph` under `key`: the cached one updated in place, or a new
// instantiation (replacing the cached one, or the least recently used entry).
cudaError_t graph_exec_for(const std::vector<const void *> &key, cudaGraph_t graph, cudaGraphExec_t *out)
{
    std::lock_guard<std::mutex> lock(g_graph_mutex);
    ++g_graph_clock;
    for (GraphEntry &e : g_graphs) {
        if (e.key != key) continue;
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(e.exec, graph, &info) == cudaSuccess) {
            e.used = g_graph_clock;
            *out = e.exec;
            return cudaSuccess;
        }
        cudaGetLastError();
        cudaGraphExecDestroy(e.exec);
        const cudaError_t r = cudaGraphInstantiate(&e.exec, graph, 0);
        if (r != cudaSuccess) {
            e.exec = nullptr;
            e.key.clear();
            return r;
        }
        e.used = g_graph_clock;
        *out = e.exec;
        return cudaSuccess;
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t r = cudaGraphInstantiate(&ex, graph, 0);
    if (r != cudaSuccess) return r;
    if (g_graphs.size() >= kGraphCache) {
        auto lru = std::min_element(g_graphs.begin(), g_graphs.end(),
                                    [](const GraphEntry &a, const GraphEntry &b) { return a.used < b.used; });
        if (lru->exec) cudaGraphExecDestroy(lru->exec);
        *lru = GraphEntry{key, ex, g_graph_clock};
    } else {
        g_graphs.push_back(GraphEntry{key, ex, g_graph_clock});
    }
    *out = ex;
    return cudaSuccess;
}

}  // namespace

extern "C" llg_status llg_autotune(llg_ctx *ctx, int64_t trial_steps, double *best_rate)
{
    llg::NvtxRange nvtx("llg_autotune");
    if (!ctx || trial_steps < 1) {
        llg::set_last_error("need a context and trial_steps >= 1");
        return LLG_EINVAL;
    }
    llg::CtxView v;
    llg_status s = llg::ctx_view(ctx, &v);
    if (s != LLG_OK) return s;
    if (v.n_real < 1 || !v.d_m) {
        llg::set_last_error("autotune needs an ensemble (llg_reset first)");
        return LLG_EINVAL;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, v.device) != cudaSuccess) {
        llg::set_last_error("cudaGetDeviceProperties failed");
        return LLG_ECUDA;
    }
    const long long period = v.kp.shape == 1 ? v.kp.period : 2 * v.kp.n_half;
    const int fits32 = period < (1LL << 31) && v.kp.sample_every < (1LL << 31);
    const TuneKey key{prop.name, v.kp.nx, v.kp.ny, v.kp.nz, v.n_real, v.kp.shape, fits32,
                      v.kp.axis != nullptr, (int)v.kp.periodic};
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        llg::RodPlan check{};
        // a cached shape is taken only while it still plans for this context
        if (it != g_tune_cache.end() &&
            (it->second.kind == 0 || llg::rod_plan(v.kp, v.n_real, v.device, &check, it->second.kind,
                                                   it->second.rods, it->second.rows, it->second.cpt))) {
            llg_set_tuning(ctx, LLG_TUNE_ROD_KIND, it->second.kind);
            llg_set_tuning(ctx, LLG_TUNE_RODS_PER_CTA, it->second.rods);
            llg_set_tuning(ctx, LLG_TUNE_ROWS_PER_THREAD, it->second.rows);
            llg_set_tuning(ctx, LLG_TUNE_CELLS_PER_THREAD, it->second.cpt);
            llg_set_tuning(ctx, LLG_TUNE_CHUNK_STEPS, it->second.chunk);
            if (best_rate) *best_rate = it->second.rate;
            return LLG_OK;
        }
    }
    // candidates: (kind, rods per CTA, rows per thread, cells per thread); 0 = automatic
    std::vector<std::tuple<int, int, int, int>> cand;
    for (int rows : {0, 1, 2, 3, 4}) cand.emplace_back(2, 0, rows, 0);
    for (int cpt : {0, 1, 2, 4})
        for (int rods : {0, 1, 2, 3, 4, 6, 8, 12, 16, 24, 32}) cand.emplace_back(1, rods, 0, cpt);
    for (int rods : {0, 1, 2, 4, 8, 16, 32}) cand.emplace_back(3, rods, 0, 0);
    const size_t bytes = (size_t)v.n_real * (size_t)v.kp.ncells * 3 * sizeof(float);
    float *scratch = nullptr;
    if (cudaMalloc(&scratch, bytes) != cudaSuccess) {
        cudaGetLastError();
        llg::set_last_error("autotune scratch allocation failed");
        return LLG_ENOMEM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = -1.0;
    TuneValue bestv{0, 0, 0, 0, 0, 0.0};
    llg::RodPlan best_plan{};
    double best_ms = 0.0;
    for (auto [kind, rods, rows, cpt] : cand) {
        llg::RodPlan plan{};
        if (!llg::rod_plan(v.kp, v.n_real, v.device, &plan, kind, rods, rows, cpt)) continue;
        if (kind == 2 && rows == 0 && plan.kind != 2) continue;
        plan.balance = true;
        double t_best = 1e30;
        bool ok = true;
        for (int rep = 0; rep < 2 && ok; ++rep) {
            cudaMemcpyAsync(scratch, v.d_m, bytes, cudaMemcpyDeviceToDevice, v.stream);
            cudaEventRecord(e0, v.stream);
            ok = llg::rod_advance(v.kp, plan, scratch, v.n_real, v.step, trial_steps, nullptr, v.d_status,
                                  v.d_flags, v.stream) == cudaSuccess;
            cudaEventRecord(e1, v.stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            t_best = std::min(t_best, (double)ms);
        }
        cudaGetLastError();
        if (!ok) continue;
        const double rate = (double)v.n_real * v.kp.ncells * trial_steps / (t_best * 1e-3);
        if (rate > best) {
            best = rate;
            bestv = TuneValue{kind, rods, rows, cpt, 0, rate};
            best_plan = plan;
            best_ms = t_best;
        }
    }
    // steps per launch: time a one-step launch of the best shape; what it costs beyond one step
    // of the trial rate is the per-launch overhead, which a launch of `chunk` steps should keep
    // near 1% (between 2^10 and 2^20 steps, a power of two)
    if (best > 0.0) {
        double t1 = 1e30;
        for (int rep = 0; rep < 3; ++rep) {
            cudaMemcpyAsync(scratch, v.d_m, bytes, cudaMemcpyDeviceToDevice, v.stream);
            cudaEventRecord(e0, v.stream);
            const bool ok = llg::rod_advance(v.kp, best_plan, scratch, v.n_real, v.step, 1, nullptr, v.d_status,
                                             v.d_flags, v.stream) == cudaSuccess;
            cudaEventRecord(e1, v.stream);
            float ms = 0.f;
            if (ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
                t1 = std::min(t1, (double)ms);
        }
        cudaGetLastError();
        const double per_step = best_ms / (double)trial_steps;
        const double overhead = std::max(0.0, t1 - per_step);
        long long chunk = 1LL << 10;
        while (chunk < (1LL << 20) && (double)chunk * per_step < 100.0 * overhead) chunk <<= 1;
        bestv.chunk = chunk;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(scratch);
    if (best <= 0.0) {
        llg::set_last_error("no resident launch shape can hold this grid");
        return LLG_EUNSUPPORTED;
    }
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = bestv;
    }
    llg_set_tuning(ctx, LLG_TUNE_ROD_KIND, bestv.kind);
    llg_set_tuning(ctx, LLG_TUNE_RODS_PER_CTA, bestv.rods);
    llg_set_tuning(ctx, LLG_TUNE_ROWS_PER_THREAD, bestv.rows);
    llg_set_tuning(ctx, LLG_TUNE_CELLS_PER_THREAD, bestv.cpt);
    llg_set_tuning(ctx, LLG_TUNE_CHUNK_STEPS, bestv.chunk);
    if (best_rate) *best_rate = best;
    return LLG_OK;
}

extern "C" llg_status llg_run_batch(llg_ctx *const *jobs, int n_jobs, int64_t max_steps,
                                    float *const *m_samples, int64_t *steps_done)
{
    llg::NvtxRange nvtx("llg_run_batch");
    if (!jobs || n_jobs < 1 || max_steps < 0) {
        llg::set_last_error("need jobs, n_jobs >= 1, max_steps >= 0");
        return LLG_EINVAL;
    }
    std::vector<llg::CtxView> views((size_t)n_jobs);
    std::vector<long long> steps((size_t)n_jobs);
    std::vector<llg::RodPlan> plans((size_t)n_jobs);
    for (int j = 0; j < n_jobs; ++j) {
        llg_status s = llg::ctx_view(jobs[j], &views[(size_t)j]);
        if (s != LLG_OK) return s;
        const llg::CtxView &v = views[(size_t)j];
        if (v.n_real < 1 || !v.d_m) {
            llg::set_last_error("every batch job needs an ensemble (llg_reset first)");
            return LLG_EINVAL;
        }
        if (v.device != views[0].device) {
            llg::set_last_error("all batch jobs must be on one device");
            return LLG_EINVAL;
        }
        // steps left in the job's loop (a constant field runs max_steps)
        const long long left = v.steps_per_loop > 0 ? std::max(0LL, v.steps_per_loop - v.step) : max_steps;
        steps[(size_t)j] = std::min<long long>(left, max_steps);
        if (!llg::rod_plan(v.kp, v.n_real, v.device, &plans[(size_t)j], v.tune_kind, v.tune_rods, v.tune_rows,
                           v.tune_cpt)) {
            char msg[128];
            std::snprintf(msg, sizeof msg, "batch job %d: the resident engine cannot hold its grid", j);
            llg::set_last_error(msg);
            return LLG_EUNSUPPORTED;
        }
        plans[(size_t)j].balance = false;  // jobs share the GPU; no co-resident grid per job
        plans[(size_t)j].generic = v.tune_generic;
    }
    // steps per graph launch: the smallest of the jobs' steps per launch
    long long chunk = 1LL << 30;
    for (int j = 0; j < n_jobs; ++j)
        if (steps[(size_t)j] > 0) chunk = std::min(chunk, std::max(1LL, views[(size_t)j].chunk_steps));
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(views[0].device);
    const cudaStream_t origin = views[0].stream;
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> br((size_t)n_jobs, nullptr);
    std::vector<cudaEvent_t> ev((size_t)n_jobs + 1, nullptr);
    llg_status status = LLG_OK;
    auto check = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && status == LLG_OK) {
            char msg[256];
            std::snprintf(msg, sizeof msg, "batch %s: %s", what, cudaGetErrorString(e));
            llg::set_last_error(msg);
            status = LLG_ECUDA;
        }
        return e == cudaSuccess;
    };
    check(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "stream");
    for (int j = 0; j < n_jobs && status == LLG_OK; ++j) check(cudaStreamCreateWithFlags(&br[(size_t)j], cudaStreamNonBlocking), "stream");
    for (auto &e : ev)
        if (status == LLG_OK) check(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    // the graphs run after the work already queued on the jobs' streams
    for (int j = 0; j < n_jobs && status == LLG_OK; ++j) {
        check(cudaEventRecord(ev[(size_t)j + 1], views[(size_t)j].stream), "order");
        check(cudaStreamWaitEvent(origin, ev[(size_t)j + 1], 0), "order");
    }
    std::vector<long long> done((size_t)n_jobs, 0), now((size_t)n_jobs, 0);
    for (;;) {
        bool any = false;
        for (int j = 0; j < n_jobs; ++j) {
            now[(size_t)j] = std::min(chunk, steps[(size_t)j] - done[(size_t)j]);
            any = any || now[(size_t)j] > 0;
        }
        if (!any || status != LLG_OK) break;
        // longest first: cell-steps of the job in this launch
        std::vector<int> order;
        for (int j = 0; j < n_jobs; ++j)
            if (now[(size_t)j] > 0) order.push_back(j);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            const double wa = (double)views[(size_t)a].n_real * views[(size_t)a].kp.ncells * now[(size_t)a];
            const double wb = (double)views[(size_t)b].n_real * views[(size_t)b].kp.ncells * now[(size_t)b];
            return wa > wb;
        });
        std::vector<const void *> key{reinterpret_cast<const void *>((uintptr_t)views[0].device)};
        cudaGraph_t graph = nullptr;
        if (check(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "capture")) {
            check(cudaEventRecord(ev[0], cap), "record");
            for (int j : order) {
                const llg::CtxView &v = views[(size_t)j];
                cudaStream_t st = br[(size_t)j];
                key.push_back(jobs[j]);
                check(cudaStreamWaitEvent(st, ev[0], 0), "fork");
                check(llg::rod_advance(v.kp, plans[(size_t)j], v.d_m, v.n_real, v.step + done[(size_t)j], now[(size_t)j],
                                       m_samples ? m_samples[j] : nullptr, v.d_status, v.d_flags, st),
                      "launch");
                check(cudaEventRecord(ev[(size_t)j + 1], st), "record");
                check(cudaStreamWaitEvent(cap, ev[(size_t)j + 1], 0), "join");
            }
            const cudaError_t e = cudaStreamEndCapture(cap, &graph);
            check(e, "end capture");
        }
        cudaGraphExec_t exec = nullptr;
        if (status == LLG_OK && check(graph_exec_for(key, graph, &exec), "instantiate"))
            check(cudaGraphLaunch(exec, origin), "graph launch");
        if (graph) cudaGraphDestroy(graph);
        for (int j = 0; j < n_jobs; ++j) done[(size_t)j] += now[(size_t)j];
    }
    if (status == LLG_OK) {
        check(cudaEventRecord(ev[0], origin), "order");
        for (int j = 0; j < n_jobs && status == LLG_OK; ++j)
            check(cudaStreamWaitEvent(views[(size_t)j].stream, ev[0], 0), "order");
    }
    for (auto e : ev)
        if (e) cudaEventDestroy(e);
    for (auto st : br)
        if (st) cudaStreamDestroy(st);
    if (cap) cudaStreamDestroy(cap);
    if (prev >= 0) cudaSetDevice(prev);
    if (status != LLG_OK) return status;
    for (int j = 0; j < n_jobs; ++j) {
        llg::ctx_add_steps(jobs[j], steps[(size_t)j]);
        if (steps_done) steps_done[j] = steps[(size_t)j];
    }
    return LLG_OK;
}
