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
    int kernel = 0;              // 0: segmented stream kernel, 1: list items
    vbk::LaunchCfg cfg{};        // kernel 0: CTAs per SM and count-ahead slack
    uint64_t chunk = 0;          // kernel 1: lists of up to `chunk` bytes decoded whole, longer ones in chunks
    int warps = 8;               // kernel 1: warps per CTA of the decode launch
    bool table = false;          // kernel 1: units decoded by the table-driven steps of Sec. 4
    uint8_t *ws = nullptr;       // status word, and kernel 0's workspace
    void *lp_mem = nullptr;      // kernel 1's device arrays
    vbk::ListPlan lp{};
    cudaGraphExec_t exec = nullptr;
    float tuned_ms = 0.f;
    int tuned = 0;               // 0: defaults, 1: timed now, 2: taken from the per-class cache
    // length classes by bytes per list: class k holds lists of 2^k .. 2^(k+1) - 1 bytes (class 0 also the empty ones)
    uint64_t cls_lists[64] = {};
    uint64_t cls_values[64] = {};
};

namespace {

// Length class of a batch: delta mode, log2 of the mean bytes per list and
// log2 of the total bytes.  Tuned choices are cached per class.
struct Choice {
    int kernel;
    vbk::LaunchCfg cfg;
    uint64_t chunk;
    int warps;
    bool table;
    float ms;
};
using ClassKey = std::tuple<int, int, int, int>;   // device, delta, log2 mean, log2 total
std::mutex g_tune_mu;
std::map<ClassKey, Choice> g_tuned;

int ilog2(double x) { return x < 1.0 ? 0 : static_cast<int>(std::floor(std::log2(x))); }

ClassKey class_of(int dev, const vbk::BatchArgs &a)
{
    const double mean = a.L ? static_cast<double>(a.nbytes) / static_cast<double>(a.L) : 0.0;
    return ClassKey(dev, a.delta ? 1 : 0, ilog2(mean), ilog2(static_cast<double>(a.nbytes)));
}

// The offset arrays' contract, checked on the host copies.
bool offsets_ok(const std::vector<uint64_t> &bo, const std::vector<uint64_t> &vo, const vbk::BatchArgs &a)
{
    if (bo.front() != 0 || vo.front() != 0 || bo.back() != a.nbytes || vo.back() != a.n) return false;
    for (size_t j = 0; j < a.L; ++j)
        if (bo[j] > bo[j + 1] || vo[j] > vo[j + 1]) return false;
    return true;
}

// Items for chunk size C: lists of at most C bytes whole, longer lists cut
// at 16-byte boundaries of the input every C bytes; decode order longest
// first; the chunked lists' items in chunk order.
struct HostItems {
    std::vector<vbk::ListItem> items;
    std::vector<uint32_t> citem, cfirst;
};

HostItems build_items(const std::vector<uint64_t> &bo, uintptr_t in, uint64_t C)
{
    HostItems h;
    std::vector<vbk::ListItem> raw;
    std::vector<std::pair<size_t, size_t>> chunked;   // (first raw item, items)
    const size_t L = bo.size() - 1;
    raw.reserve(L + bo.back() / C + 1);
    for (size_t j = 0; j < L; ++j) {
        const uint64_t b0 = bo[j], b1 = bo[j + 1];
        if (b1 - b0 <= C) {
            raw.push_back({b0, b1, static_cast<uint32_t>(j), vbk::kItemOnly | vbk::kItemLast});
            continue;
        }
        const size_t first = raw.size();
        const uint64_t a = ((in + b0) & ~static_cast<uint64_t>(15)) - in;   // the list's first 16-byte boundary (at or before b0)
        uint64_t st = b0;
        for (uint64_t k = 1;; ++k) {
            const uint64_t e = a + k * C;
            if (e >= b1) {
                raw.push_back({st, b1, static_cast<uint32_t>(j), vbk::kItemLast});
                break;
            }
            raw.push_back({st, e, static_cast<uint32_t>(j), 0u});
            st = e;
        }
        chunked.emplace_back(first, raw.size() - first);
    }
    std::vector<uint32_t> order(raw.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = static_cast<uint32_t>(i);
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
        return raw[x].b1 - raw[x].b0 > raw[y].b1 - raw[y].b0;
    });
    std::vector<uint32_t> pos(raw.size());
    h.items.resize(raw.size());
    for (size_t i = 0; i < order.size(); ++i) {
        h.items[i] = raw[order[i]];
        pos[order[i]] = static_cast<uint32_t>(i);
    }
    for (const auto &c : chunked) {
        h.cfirst.push_back(static_cast<uint32_t>(h.citem.size()));
        for (size_t r = c.first; r < c.first + c.second; ++r) h.citem.push_back(pos[r]);
    }
    h.cfirst.push_back(static_cast<uint32_t>(h.citem.size()));
    return h;
}

// Upload an item set into one device allocation (`rel` zeroed).
int upload_items(const HostItems &h, void **mem, vbk::ListPlan *lp, cudaStream_t s)
{
    const size_t ni = h.items.size(), nc = h.citem.size(), nf = h.cfirst.size();
    auto up16 = [](size_t x) { return (x + 15) / 16 * 16; };
    const size_t o_items = 0, o_citem = up16(o_items + ni * sizeof(vbk::ListItem));
    const size_t o_cfirst = up16(o_citem + nc * 4), o_cs = up16(o_cfirst + nf * 4);
    const size_t o_rel = up16(o_cs + ni * 8), o_q = up16(o_rel + ni * 8), total = o_q + 16;
    uint8_t *m = nullptr;
    if (cudaMalloc(reinterpret_cast<void **>(&m), total) != cudaSuccess) {
        cudaGetLastError();
        return VBYTE_ENOMEM;
    }
    *mem = m;
    lp->items = reinterpret_cast<vbk::ListItem *>(m + o_items);
    lp->nitems = static_cast<uint32_t>(ni);
    lp->citem = reinterpret_cast<uint32_t *>(m + o_citem);
    lp->cfirst = reinterpret_cast<uint32_t *>(m + o_cfirst);
    lp->ncl = static_cast<uint32_t>(nf - 1);
    lp->cs = reinterpret_cast<uint2 *>(m + o_cs);
    lp->rel = reinterpret_cast<uint2 *>(m + o_rel);
    lp->queue = reinterpret_cast<unsigned int *>(m + o_q);
    if (ni && cudaMemcpyAsync(lp->items, h.items.data(), ni * sizeof(vbk::ListItem), cudaMemcpyHostToDevice, s) !=
                  cudaSuccess)
        return VBYTE_ECUDA;
    if (nc && cudaMemcpyAsync(lp->citem, h.citem.data(), nc * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return VBYTE_ECUDA;
    if (cudaMemcpyAsync(lp->cfirst, h.cfirst.data(), nf * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return VBYTE_ECUDA;
    if (cudaMemsetAsync(lp->rel, 0, ni * 8, s) != cudaSuccess) return VBYTE_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
}

int enqueue_plan(const vbyte_plan &P, cudaStream_t s)
{
    if (P.kernel == 1)
        return vbk::enqueue_list_plan(P.a, P.lp, P.warps, reinterpret_cast<uint32_t *>(P.ws), s, P.table);
    return vbk::enqueue_sbatched(P.a, P.ws, P.cfg, s);
}

// Median time of `reps` runs of the plan's current choice on s (after one
// untimed run).
int time_plan(const vbyte_plan &P, cudaStream_t s, int reps, float *ms)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return VBYTE_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return VBYTE_ECUDA;
    }
    int rc = enqueue_plan(P, s);
    std::vector<float> t;
    for (int r = 0; r < reps && rc == VBYTE_OK; ++r) {
        cudaEventRecord(e0, s);
        rc = enqueue_plan(P, s);
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

void free_items(vbyte_plan *P)
{
    if (P->lp_mem) cudaFree(P->lp_mem);
    P->lp_mem = nullptr;
    P->lp = vbk::ListPlan{};
}

// Make the plan's kernel 1 arrays those of chunk size C.
int set_items(vbyte_plan *P, const std::vector<uint64_t> &bo, uint64_t C, cudaStream_t s)
{
    free_items(P);
    const HostItems h = build_items(bo, reinterpret_cast<uintptr_t>(P->a.in), C);
    return upload_items(h, &P->lp_mem, &P->lp, s);
}

constexpr uint64_t kChunks[] = {8u << 10, 16u << 10, 32u << 10, 64u << 10};
constexpr int kWarpChoices[] = {4, 8};

// vbyte_debug_force_plan
std::mutex g_force_mu;
int g_force_kernel = -1;
uint64_t g_force_chunk = 0;
int g_force_warps = 8;
bool g_force_table = false;

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
        free_items(P);
        delete P;
        return code;
    };
    // inputs may still be in flight on the caller's stream
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return fail(VBYTE_ECUDA);
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return fail(VBYTE_ECUDA);
    if (cudaMalloc(&P->ws, vbk::sbatched_workspace_bytes(a)) != cudaSuccess) return fail(VBYTE_ENOMEM);
    if (cudaMemsetAsync(P->ws, 0, sizeof(uint32_t), s) != cudaSuccess) return fail(VBYTE_ECUDA);
    // the offsets on the host: length classes and list items
    std::vector<uint64_t> bo(num_lists + 1), vo(num_lists + 1);
    if (cudaMemcpy(bo.data(), d_byte_off, bo.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(vo.data(), d_val_off, vo.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(VBYTE_ECUDA);
    const bool items_ok = offsets_ok(bo, vo, a);
    if (items_ok) {
        for (size_t j = 0; j < num_lists; ++j) {
            const uint64_t nb = bo[j + 1] - bo[j];
            const int k = nb ? 63 - __builtin_clzll(nb) : 0;
            P->cls_lists[k] += 1;
            P->cls_values[k] += vo[j + 1] - vo[j];
        }
    }
    // defaults: list items of 32 KiB chunks, 8 warps per CTA (the segmented
    // stream kernel when the offsets break their contract: it reports that)
    P->kernel = items_ok ? 1 : 0;
    P->chunk = 32u << 10;
    P->warps = 8;
    int forced = -1;
    {
        std::lock_guard<std::mutex> lk(g_force_mu);
        if (g_force_kernel == 0 || (g_force_kernel == 1 && items_ok)) {
            forced = g_force_kernel;
            P->kernel = g_force_kernel;
            P->chunk = g_force_chunk;
            P->warps = g_force_warps;
            P->table = g_force_table;
        }
    }

    if (autotune && forced < 0) {
        const ClassKey key = class_of(P->dev, a);
        bool cached = false;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tuned.find(key);
            if (it != g_tuned.end() && (items_ok || it->second.kernel == 0)) {
                P->kernel = it->second.kernel;
                P->cfg = it->second.cfg;
                P->chunk = it->second.chunk;
                P->warps = it->second.warps;
                P->table = it->second.table;
                P->tuned_ms = it->second.ms;
                P->tuned = 2;
                cached = true;
            }
        }
        if (!cached) {
            Choice best{0, vbk::LaunchCfg(), 0, 8, false, 0.f};
            bool have = false;
            auto consider = [&](const Choice &c, float ms) {
                if (!have || ms < best.ms) {
                    best = c;
                    best.ms = ms;
                    have = true;
                }
            };
            // the segmented stream kernel
            const int occ = vbk::sbatched_max_ctas(a.delta);
            for (uint64_t sl : {uint64_t(3584), uint64_t(4608)}) {
                P->kernel = 0;
                P->cfg.ctas_per_sm = occ;
                P->cfg.lead_slack = sl;
                float ms = 0.f;
                if ((rc = time_plan(*P, s, 3, &ms)) != VBYTE_OK) return fail(rc);
                consider(Choice{0, P->cfg, 0, 8, false, 0.f}, ms);
            }
            // list items: chunk size (which length classes are decoded whole
            // in one pass and which by count-then-decode) x warps per CTA
            if (items_ok) {
                for (uint64_t C : kChunks) {
                    if ((rc = set_items(P, bo, C, s)) != VBYTE_OK) return fail(rc);
                    for (int w : kWarpChoices) {
                        // units by per-terminator assembly, and (256 threads)
                        // by the table-driven steps of Sec. 4
                        for (int tb = 0; tb < (w == 8 ? 2 : 1); ++tb) {
                            P->kernel = 1;
                            P->chunk = C;
                            P->warps = w;
                            P->table = tb != 0;
                            float ms = 0.f;
                            if ((rc = time_plan(*P, s, 3, &ms)) != VBYTE_OK) return fail(rc);
                            consider(Choice{1, vbk::LaunchCfg(), C, w, tb != 0, 0.f}, ms);
                        }
                    }
                }
            }
            P->kernel = best.kernel;
            P->cfg = best.cfg;
            P->chunk = best.chunk;
            P->warps = best.warps;
            P->table = best.table;
            P->tuned_ms = best.ms;
            P->tuned = 1;
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tuned[key] = best;
        }
        // the tuning runs' data errors belong to no caller launch
        if (cudaMemsetAsync(P->ws, 0, sizeof(uint32_t), s) != cudaSuccess) return fail(VBYTE_ECUDA);
    }
    if (P->kernel == 1) {
        if ((rc = set_items(P, bo, P->chunk, s)) != VBYTE_OK) return fail(rc);
    } else {
        free_items(P);
    }

    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return fail(VBYTE_ECUDA);
    rc = enqueue_plan(*P, s);
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

int vbyte_debug_force_plan(int kernel, uint64_t chunk_bytes, int threads_per_block)
{
    if (kernel < -1 || kernel > 2) return VBYTE_EINVAL;
    if (kernel >= 1 && (chunk_bytes < 4096 || chunk_bytes % 16 || (threads_per_block != 128 && threads_per_block != 256)))
        return VBYTE_EINVAL;
    std::lock_guard<std::mutex> lk(g_force_mu);
    g_force_table = kernel == 2;
    g_force_kernel = kernel == 2 ? 1 : kernel;
    g_force_chunk = chunk_bytes;
    g_force_warps = threads_per_block / 32;
    return VBYTE_OK;
}

int vbyte_plan_choice(const vbyte_plan *plan, int *kernel, uint64_t *chunk_bytes, int *threads_per_block)
{
    if (!plan) return VBYTE_EINVAL;
    if (kernel) *kernel = plan->kernel == 1 && plan->table ? 2 : plan->kernel;
    if (chunk_bytes) *chunk_bytes = plan->kernel == 1 ? plan->chunk : 0;
    if (threads_per_block) *threads_per_block = plan->kernel == 1 ? plan->warps * 32 : 256;
    return VBYTE_OK;
}

int vbyte_plan_class(const vbyte_plan *plan, int k, uint64_t *lists, uint64_t *values, int *mode)
{
    if (!plan || k < 0 || k > 63) return VBYTE_EINVAL;
    if (lists) *lists = plan->cls_lists[k];
    if (values) *values = plan->cls_values[k];
    if (mode) {
        int m = 0;
        if (plan->cls_lists[k]) {
            if (plan->kernel == 0)
                m = 3;
            else
                m = ((uint64_t(2) << k) - 1 <= plan->chunk) ? 1 : 2;   // the whole class fits one item
        }
        *mode = m;
    }
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
    free_items(plan);
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
