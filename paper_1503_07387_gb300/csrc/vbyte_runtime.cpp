// Host runtime on top of the decode kernels: reusable batched plans (launch
// parameters picked by timing, the launch sequence replayed from a CUDA
// graph) and the one-call-per-list form that batched decoding replaces.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "vbyte.h"
#include "vbyte_internal.h"

struct vbyte_plan {
    int dev = 0;
    vbk::BatchArgs a{};
    vbk::LaunchCfg cfg{};
    uint8_t *ws = nullptr;
    cudaGraphExec_t exec = nullptr;
    float tuned_ms = 0.f;
    int tuned = 0;   // 0: defaults, 1: timed now, 2: taken from the per-class cache
};

namespace {

// Length class of a batch: delta mode, log2 of the mean bytes per list and
// log2 of the total bytes.  Tuned launch parameters are cached per class.
using ClassKey = std::tuple<int, int, int, int>;   // device, delta, log2 mean, log2 total
std::mutex g_tune_mu;
std::map<ClassKey, std::pair<vbk::LaunchCfg, float>> g_tuned;

int ilog2(double x) { return x < 1.0 ? 0 : static_cast<int>(std::floor(std::log2(x))); }

ClassKey class_of(int dev, const vbk::BatchArgs &a)
{
    const double mean = a.L ? static_cast<double>(a.nbytes) / static_cast<double>(a.L) : 0.0;
    return ClassKey(dev, a.delta ? 1 : 0, ilog2(mean), ilog2(static_cast<double>(a.nbytes)));
}

// Median time of `reps` runs of cfg on s (after one untimed run).
int time_cfg(const vbk::BatchArgs &a, uint8_t *ws, const vbk::LaunchCfg &cfg, cudaStream_t s, int reps,
             float *ms)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return VBYTE_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return VBYTE_ECUDA;
    }
    int rc = vbk::enqueue_sbatched(a, ws, cfg, s);
    std::vector<float> t;
    for (int r = 0; r < reps && rc == VBYTE_OK; ++r) {
        cudaEventRecord(e0, s);
        rc = vbk::enqueue_sbatched(a, ws, cfg, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = VBYTE_ECUDA;
        float x = 0.f;
        cudaEventElapsedTime(&x, e0, e1);
        t.push_back(x);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != VBYTE_OK) return rc;
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return VBYTE_OK;
}

}  // namespace

extern "C" {

int vbyte_plan_create(vbyte_plan **plan_out, const uint8_t *d_in, size_t nbytes, const uint64_t *d_byte_off,
                      uint32_t *d_out, size_t n, const uint64_t *d_val_off, size_t num_lists, const uint32_t *d_prev,
                      int delta, int autotune, void *stream)
{
    if (!plan_out) return VBYTE_EINVAL;
    *plan_out = nullptr;
    const vbk::BatchArgs a{d_in, nbytes, d_byte_off, d_out, n, d_val_off, num_lists, delta ? d_prev : nullptr,
                           delta != 0};
    int rc = vbk::check_batch(a);
    if (rc != VBYTE_OK) return rc;
    if (num_lists == 0) return VBYTE_EINVAL;
    vbyte_plan *P = new vbyte_plan();
    P->a = a;
    cudaGetDevice(&P->dev);
    cudaStream_t s = nullptr;
    cudaGraph_t graph = nullptr;
    auto fail = [&](int code) {
        cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        if (s) cudaStreamDestroy(s);
        if (P->exec) cudaGraphExecDestroy(P->exec);
        if (P->ws) cudaFree(P->ws);
        delete P;
        return code;
    };
    // inputs may still be in flight on the caller's stream
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return fail(VBYTE_ECUDA);
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return fail(VBYTE_ECUDA);
    if (cudaMalloc(&P->ws, vbk::sbatched_workspace_bytes(a)) != cudaSuccess) return fail(VBYTE_ENOMEM);
    if (cudaMemsetAsync(P->ws, 0, sizeof(uint32_t), s) != cudaSuccess) return fail(VBYTE_ECUDA);

    if (autotune) {
        const ClassKey key = class_of(P->dev, a);
        bool cached = false;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tuned.find(key);
            if (it != g_tuned.end()) {
                P->cfg = it->second.first;
                P->tuned_ms = it->second.second;
                P->tuned = 2;
                cached = true;
            }
        }
        if (!cached) {
            const int occ = vbk::sbatched_max_ctas(a.delta);
            const uint64_t slacks[] = {3584, 4608, 5632};
            float best = 0.f;
            for (int c = 1; c <= occ; ++c) {
                for (uint64_t sl : slacks) {
                    vbk::LaunchCfg cfg;
                    cfg.ctas_per_sm = c;
                    cfg.lead_slack = sl;
                    float ms = 0.f;
                    rc = time_cfg(a, P->ws, cfg, s, 3, &ms);
                    if (rc != VBYTE_OK) return fail(rc);
                    if (P->tuned == 0 || ms < best) {
                        best = ms;
                        P->cfg = cfg;
                        P->tuned = 1;
                    }
                }
            }
            P->tuned_ms = best;
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tuned[key] = {P->cfg, best};
        }
        // the tuning runs' data errors belong to no caller launch
        if (cudaMemsetAsync(P->ws, 0, sizeof(uint32_t), s) != cudaSuccess) return fail(VBYTE_ECUDA);
    }

    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return fail(VBYTE_ECUDA);
    rc = vbk::enqueue_sbatched(a, P->ws, P->cfg, s);
    const cudaError_t ce = cudaStreamEndCapture(s, &graph);
    if (rc != VBYTE_OK) return fail(rc);
    if (ce != cudaSuccess) return fail(VBYTE_ECUDA);
    if (cudaGraphInstantiate(&P->exec, graph, 0) != cudaSuccess) return fail(VBYTE_ECUDA);
    cudaGraphDestroy(graph);
    graph = nullptr;
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(VBYTE_ECUDA);
    cudaStreamDestroy(s);
    *plan_out = P;
    return VBYTE_OK;
}

int vbyte_plan_launch(vbyte_plan *plan, void *stream)
{
    if (!plan || !plan->exec) return VBYTE_EINVAL;
    return cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
}

int vbyte_plan_get_status(vbyte_plan *plan, void *stream, uint32_t *status_out)
{
    if (!plan || !status_out) return VBYTE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t v = 0;
    if (cudaMemcpyAsync(&v, plan->ws, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess) return VBYTE_ECUDA;
    if (cudaMemsetAsync(plan->ws, 0, sizeof(uint32_t), s) != cudaSuccess) return VBYTE_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return VBYTE_ECUDA;
    *status_out = v;
    return VBYTE_OK;
}

int vbyte_plan_describe(const vbyte_plan *plan, int *ctas_per_sm, uint64_t *lead_slack, float *tuned_ms,
                        int *tuned)
{
    if (!plan) return VBYTE_EINVAL;
    if (ctas_per_sm) *ctas_per_sm = plan->cfg.ctas_per_sm;
    if (lead_slack) *lead_slack = plan->cfg.lead_slack;
    if (tuned_ms) *tuned_ms = plan->tuned_ms;
    if (tuned) *tuned = plan->tuned;
    return VBYTE_OK;
}

void vbyte_plan_destroy(vbyte_plan *plan)
{
    if (!plan) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(plan->dev);
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->ws) cudaFree(plan->ws);
    cudaSetDevice(cur);
    delete plan;
}

int vbyte_decode_each(const uint8_t *d_in, const uint64_t *h_byte_off, uint32_t *d_out, const uint64_t *h_val_off,
                      size_t num_lists, int delta, const uint32_t *h_prev, void *stream)
{
    if (num_lists && (!h_byte_off || !h_val_off)) return VBYTE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (size_t j = 0; j < num_lists; ++j) {
        const uint64_t b0 = h_byte_off[j], b1 = h_byte_off[j + 1];
        const uint64_t v0 = h_val_off[j], v1 = h_val_off[j + 1];
        if (b1 < b0 || v1 < v0) return VBYTE_EINVAL;
        const int rc = vbk::launch_decode(d_in + b0, b1 - b0, d_out + v0, v1 - v0, delta != 0,
                                          (delta && h_prev) ? h_prev[j] : 0u, s);
        if (rc != VBYTE_OK) return rc;
    }
    return VBYTE_OK;
}

}  // extern "C"
