// Serving loop: a pool of compressed posting lists stays resident in device
// memory; queries (each naming several lists) arrive at any time; a
// scheduler thread admits them in arrival order, as far as the device arena
// has room for their decoded output, into batches that run on several
// streams at once (continuous batching), and records each query's
// completion time.  A batch is decoded in place: its lists become work items
// (a whole list, or a chunk of a long one) that warps decode straight from
// the pool into the query's arena space (the list-item kernels of batched
// plans).  Comparison forms: every list with its own single-stream call, and
// the lists gathered end to end into a staging buffer and decoded with one
// segmented batched launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "vbyte.h"
#include "vbyte_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

constexpr uint64_t kArenaUnit = 256;                 // arena allocation granule (bytes)
constexpr uint32_t kPieceBytes = 64u << 10;          // gather piece size
constexpr uint64_t kItemBytes = 32u << 10;           // in-place form: lists of more bytes are cut into chunks
constexpr int kItemWarps = 8;                        // in-place form: warps per CTA of the decode launch

struct Query {
    std::vector<uint32_t> lists;
    uint64_t n = 0;         // values
    uint64_t bytes = 0;     // compressed bytes
    double t_arrival = 0.0;
    double t_done = 0.0;
    int state = 0;          // 0 queued, 1 on the GPU, 2 done, 3 released
    bool auto_release = false;
    uint64_t batch = 0;
    uint32_t batch_queries = 0;
    uint64_t block = 0;     // arena block
    uint64_t out_off = 0;   // first value within the arena
    uint32_t status = 0;
};

struct Block {
    uint64_t off = 0, size = 0;   // arena units
    uint32_t refs = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    uint8_t *d_staging = nullptr;
    uint8_t *d_desc = nullptr;     // bo | vo | prev | pieces
    uint8_t *h_desc = nullptr;     // pinned mirror
    uint32_t *h_status = nullptr;  // pinned
    size_t desc_bytes = 0;
    bool busy = false;
    std::vector<uint64_t> queries;   // the batch's queries
    std::vector<uint32_t> lists;     // their lists, in output order (copied under the lock)
    uint64_t batch = 0;
};

}  // namespace

struct vbyte_server {
    int dev = 0;
    const uint8_t *d_pool = nullptr;
    size_t pool_bytes = 0;
    std::vector<uint64_t> bo, vo;
    std::vector<uint32_t> prev;
    size_t L = 0;
    bool delta = false;
    vbyte_server_config cfg{};
    uint32_t *d_arena = nullptr;
    uint64_t arena_units = 0;
    std::map<uint64_t, uint64_t> free_units;   // offset -> size
    std::map<uint64_t, Block> blocks;
    uint64_t next_block = 1;
    std::vector<Slot> slots;
    std::vector<Query> queries;
    std::deque<uint64_t> pending;
    std::mutex mu;
    std::condition_variable cv;
    std::condition_variable cv_work;   // the scheduler, idle: a query arrived, memory was released, or stop
    std::thread worker;
    std::atomic<bool> stop{false};
    int error = VBYTE_OK;
    uint64_t n_batches = 0, n_queries = 0, n_values = 0, n_lists = 0;

    // ---- arena (first fit, coalescing) -- caller holds mu
    bool arena_alloc(uint64_t units, uint64_t *off)
    {
        for (auto it = free_units.begin(); it != free_units.end(); ++it) {
            if (it->second >= units) {
                *off = it->first;
                const uint64_t rest = it->second - units;
                const uint64_t o = it->first + units;
                free_units.erase(it);
                if (rest) free_units[o] = rest;
                return true;
            }
        }
        return false;
    }

    void arena_free(uint64_t off, uint64_t units)
    {
        auto it = free_units.emplace(off, units).first;
        auto nx = std::next(it);
        if (nx != free_units.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_units.erase(nx);
        }
        if (it != free_units.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_units.erase(it);
            }
        }
    }

    void release_locked(Query &q)
    {
        if (q.state != 2) return;
        q.state = 3;
        auto it = blocks.find(q.block);
        if (it != blocks.end() && --it->second.refs == 0) {
            arena_free(it->second.off, it->second.size);
            blocks.erase(it);
            cv_work.notify_one();   // admission may have been waiting for this memory
        }
    }

    // ---- in place: the batch's lists as work items over the pool.  Virtual
    // list v (its batch position) has entries 2v and 2v + 1 in the batch's
    // offset arrays: its pool bytes, its output ranks within the batch's
    // arena block, and x_0 -- the layout the list-item kernels read.
    int launch_items(Slot &sl, uint32_t *out)
    {
        const size_t nl = sl.lists.size();
        std::vector<vbk::ListItem> raw;
        std::vector<std::pair<size_t, size_t>> chunked;
        raw.reserve(2 * nl);
        const uintptr_t in = reinterpret_cast<uintptr_t>(d_pool);
        for (size_t v = 0; v < nl; ++v) {
            const uint32_t j = sl.lists[v];
            const uint64_t b0 = bo[j], b1 = bo[j + 1];
            const uint32_t lv = static_cast<uint32_t>(2 * v);
            if (b1 - b0 <= kItemBytes) {
                raw.push_back({b0, b1, lv, vbk::kItemOnly | vbk::kItemLast});
                continue;
            }
            const size_t first = raw.size();
            const uint64_t a = ((in + b0) & ~static_cast<uint64_t>(15)) - in;
            uint64_t st = b0;
            for (uint64_t k = 1;; ++k) {
                const uint64_t e = a + k * kItemBytes;
                if (e >= b1) {
                    raw.push_back({st, b1, lv, vbk::kItemLast});
                    break;
                }
                raw.push_back({st, e, lv, 0u});
                st = e;
            }
            chunked.emplace_back(first, raw.size() - first);
        }
        // decode order: longest first
        std::vector<uint32_t> order(raw.size()), pos(raw.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = static_cast<uint32_t>(i);
        std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
            return raw[x].b1 - raw[x].b0 > raw[y].b1 - raw[y].b0;
        });
        const size_t ni = raw.size();
        size_t nci = 0;
        for (const auto &c : chunked) nci += c.second;
        const size_t ncl = chunked.size();
        auto up16 = [](size_t x) { return (x + 15) / 16 * 16; };
        const size_t o_items = 0, o_citem = up16(ni * sizeof(vbk::ListItem)), o_cfirst = up16(o_citem + nci * 4);
        const size_t o_bo = up16(o_cfirst + (ncl + 1) * 4), o_vo = o_bo + 16 * nl, o_pv = o_vo + 16 * nl;
        const size_t o_rel = up16(o_pv + 8 * nl), upload = o_rel + 8 * ni;
        const size_t o_cs = up16(upload), o_q = up16(o_cs + 8 * ni), total = o_q + 16;
        if (total > sl.desc_bytes) return VBYTE_EINVAL;
        vbk::ListItem *hi = reinterpret_cast<vbk::ListItem *>(sl.h_desc + o_items);
        for (size_t i = 0; i < ni; ++i) {
            hi[i] = raw[order[i]];
            pos[order[i]] = static_cast<uint32_t>(i);
        }
        uint32_t *hci = reinterpret_cast<uint32_t *>(sl.h_desc + o_citem);
        uint32_t *hcf = reinterpret_cast<uint32_t *>(sl.h_desc + o_cfirst);
        size_t e = 0;
        for (size_t c = 0; c < ncl; ++c) {
            hcf[c] = static_cast<uint32_t>(e);
            for (size_t r = chunked[c].first; r < chunked[c].first + chunked[c].second; ++r) hci[e++] = pos[r];
        }
        hcf[ncl] = static_cast<uint32_t>(e);
        uint64_t *hbo = reinterpret_cast<uint64_t *>(sl.h_desc + o_bo);
        uint64_t *hvo = reinterpret_cast<uint64_t *>(sl.h_desc + o_vo);
        uint32_t *hpv = reinterpret_cast<uint32_t *>(sl.h_desc + o_pv);
        uint64_t o = 0;
        for (size_t v = 0; v < nl; ++v) {
            const uint32_t j = sl.lists[v];
            hbo[2 * v] = bo[j];
            hbo[2 * v + 1] = bo[j + 1];
            hvo[2 * v] = o;
            o += vo[j + 1] - vo[j];
            hvo[2 * v + 1] = o;
            hpv[2 * v] = delta ? prev[j] : 0u;
            hpv[2 * v + 1] = 0u;
        }
        std::memset(sl.h_desc + o_rel, 0, 8 * ni);
        if (cudaMemcpyAsync(sl.d_desc, sl.h_desc, upload, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
            return VBYTE_ECUDA;
        vbk::ListPlan lp{};
        lp.items = reinterpret_cast<vbk::ListItem *>(sl.d_desc + o_items);
        lp.nitems = static_cast<uint32_t>(ni);
        lp.citem = reinterpret_cast<uint32_t *>(sl.d_desc + o_citem);
        lp.cfirst = reinterpret_cast<uint32_t *>(sl.d_desc + o_cfirst);
        lp.ncl = static_cast<uint32_t>(ncl);
        lp.cs = reinterpret_cast<uint2 *>(sl.d_desc + o_cs);
        lp.rel = reinterpret_cast<uint2 *>(sl.d_desc + o_rel);
        lp.queue = reinterpret_cast<unsigned int *>(sl.d_desc + o_q);
        const vbk::BatchArgs a{d_pool, pool_bytes, reinterpret_cast<const uint64_t *>(sl.d_desc + o_bo), out, o,
                               reinterpret_cast<const uint64_t *>(sl.d_desc + o_vo), 2 * nl,
                               delta ? reinterpret_cast<const uint32_t *>(sl.d_desc + o_pv) : nullptr, delta};
        uint32_t *d_status = nullptr;
        if (vbk::status_word(sl.stream, &d_status) != VBYTE_OK) return VBYTE_ECUDA;
        return vbk::enqueue_list_plan(a, lp, kItemWarps, d_status, sl.stream);
    }

    // descriptor bytes a slot needs for the in-place form
    static size_t items_desc_bytes(const vbyte_server_config &c)
    {
        const size_t nl = static_cast<size_t>(c.max_batch_lists);
        const size_t ni = 2 * nl + c.staging_bytes / kItemBytes + 1;
        return ni * (sizeof(vbk::ListItem) + 4 + 16) + (nl + 2) * 4 + nl * 40 + 256;
    }

    // ---- one batch on slot sl (queries already marked on the GPU)
    int launch(Slot &sl, uint64_t block_units_off)
    {
        cudaGetLastError();   // clear non-sticky results of earlier queries
        uint32_t *out = d_arena + block_units_off * (kArenaUnit / 4);
        if (cfg.per_list == 0) {
            const int rc = launch_items(sl, out);
            if (rc != VBYTE_OK) return rc;
        } else if (cfg.per_list == 1) {
            uint64_t o = 0;
            for (uint32_t j : sl.lists) {
                const uint64_t nb = bo[j + 1] - bo[j], nv = vo[j + 1] - vo[j];
                const int rc = vbk::launch_decode(d_pool + bo[j], nb, out + o, nv, delta, delta ? prev[j] : 0u,
                                                  sl.stream);
                if (rc != VBYTE_OK) return rc;
                o += nv;
            }
        } else {
            // descriptors: lists end to end in staging order
            size_t nl = 0, np = 0;
            for (uint32_t j : sl.lists) {
                ++nl;
                np += (bo[j + 1] - bo[j] + kPieceBytes - 1) / kPieceBytes;
            }
            const size_t o_bo = 0, o_vo = (nl + 1) * 8, o_prev = o_vo + (nl + 1) * 8;
            const size_t o_pc = (o_prev + nl * 4 + 15) / 16 * 16;
            const size_t total = o_pc + np * sizeof(vbk::GatherPiece);
            if (total > sl.desc_bytes) return VBYTE_EINVAL;
            uint64_t *hbo = reinterpret_cast<uint64_t *>(sl.h_desc + o_bo);
            uint64_t *hvo = reinterpret_cast<uint64_t *>(sl.h_desc + o_vo);
            uint32_t *hpv = reinterpret_cast<uint32_t *>(sl.h_desc + o_prev);
            vbk::GatherPiece *hpc = reinterpret_cast<vbk::GatherPiece *>(sl.h_desc + o_pc);
            uint64_t b = 0, v = 0;
            size_t li = 0, pi = 0;
            for (uint32_t j : sl.lists) {
                const uint64_t nb = bo[j + 1] - bo[j];
                hbo[li] = b;
                hvo[li] = v;
                hpv[li] = delta ? prev[j] : 0u;
                for (uint64_t x = 0; x < nb; x += kPieceBytes) {
                    hpc[pi].src = bo[j] + x;
                    hpc[pi].dst = b + x;
                    hpc[pi].len = static_cast<uint32_t>(std::min<uint64_t>(kPieceBytes, nb - x));
                    hpc[pi].pad = 0;
                    ++pi;
                }
                b += nb;
                v += vo[j + 1] - vo[j];
                ++li;
            }
            hbo[li] = b;
            hvo[li] = v;
            if (cudaMemcpyAsync(sl.d_desc, sl.h_desc, total, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
                return VBYTE_ECUDA;
            int rc = vbk::enqueue_gather(d_pool, sl.d_staging,
                                         reinterpret_cast<const vbk::GatherPiece *>(sl.d_desc + o_pc), np, sl.stream);
            if (rc != VBYTE_OK) return rc;
            const vbk::BatchArgs a{sl.d_staging, b, reinterpret_cast<const uint64_t *>(sl.d_desc + o_bo), out, v,
                                   reinterpret_cast<const uint64_t *>(sl.d_desc + o_vo), nl,
                                   delta ? reinterpret_cast<const uint32_t *>(sl.d_desc + o_prev) : nullptr, delta};
            rc = vbk::launch_decode_batched(a, sl.stream);
            if (rc != VBYTE_OK) return rc;
        }
        uint32_t *d_status = nullptr;
        if (vbk::status_word(sl.stream, &d_status) != VBYTE_OK) return VBYTE_ECUDA;
        if (cudaMemcpyAsync(sl.h_status, d_status, 4, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess)
            return VBYTE_ECUDA;
        if (cudaMemsetAsync(d_status, 0, 4, sl.stream) != cudaSuccess) return VBYTE_ECUDA;
        return cudaEventRecord(sl.done, sl.stream) == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
    }

    // ---- the scheduler thread
    void run()
    {
        cudaSetDevice(dev);
        while (!stop.load(std::memory_order_relaxed)) {
            bool progress = false;
            // completions
            for (Slot &sl : slots) {
                if (!sl.busy || cudaEventQuery(sl.done) != cudaSuccess) continue;
                const double t = now_s();
                std::lock_guard<std::mutex> lk(mu);
                for (uint64_t qi : sl.queries) {
                    Query &q = queries[qi];
                    q.t_done = t;
                    q.state = 2;
                    q.status = *sl.h_status;
                    if (q.auto_release) release_locked(q);
                }
                sl.busy = false;
                sl.queries.clear();
                progress = true;
                cv.notify_all();
            }
            // admissions: the longest arrival-order prefix that fits one batch
            Slot *free_slot = nullptr;
            for (Slot &sl : slots)
                if (!sl.busy) {
                    free_slot = &sl;
                    break;
                }
            if (free_slot) {
                std::unique_lock<std::mutex> lk(mu);
                std::vector<uint64_t> take;
                uint64_t bytes = 0, vals = 0;
                size_t lists = 0;
                for (uint64_t qi : pending) {
                    const Query &q = queries[qi];
                    if (!take.empty() &&
                        (take.size() >= static_cast<size_t>(cfg.max_batch_queries) ||
                         bytes + q.bytes > cfg.staging_bytes ||
                         lists + q.lists.size() > static_cast<size_t>(cfg.max_batch_lists)))
                        break;
                    take.push_back(qi);
                    bytes += q.bytes;
                    vals += q.n;
                    lists += q.lists.size();
                }
                uint64_t off = 0;
                while (!take.empty()) {   // admission by free output memory
                    const uint64_t units = std::max<uint64_t>(1, (vals * 4 + kArenaUnit - 1) / kArenaUnit);
                    if (arena_alloc(units, &off)) {
                        const uint64_t bid = next_block++;
                        blocks[bid] = Block{off, units, static_cast<uint32_t>(take.size())};
                        uint64_t o = 0;
                        const uint64_t batch = ++n_batches;
                        for (uint64_t qi : take) {
                            Query &q = queries[qi];
                            q.state = 1;
                            q.block = bid;
                            q.out_off = off * (kArenaUnit / 4) + o;
                            q.batch = batch;
                            q.batch_queries = static_cast<uint32_t>(take.size());
                            o += q.n;
                            n_values += q.n;
                            n_lists += q.lists.size();
                        }
                        n_queries += take.size();
                        pending.erase(pending.begin(), pending.begin() + take.size());
                        free_slot->lists.clear();
                        for (uint64_t qi : take)
                            free_slot->lists.insert(free_slot->lists.end(), queries[qi].lists.begin(),
                                                    queries[qi].lists.end());
                        free_slot->queries = take;
                        free_slot->batch = batch;
                        free_slot->busy = true;
                        break;
                    }
                    const Query &last = queries[take.back()];
                    vals -= last.n;
                    take.pop_back();
                }
                lk.unlock();
                if (free_slot->busy) {
                    const int rc = launch(*free_slot, off);
                    if (rc != VBYTE_OK) {
                        std::lock_guard<std::mutex> lk2(mu);
                        error = rc;
                        stop = true;
                        cv.notify_all();
                    }
                    progress = true;
                }
            }
            if (!progress) {
                bool busy = false;
                for (const Slot &sl : slots) busy = busy || sl.busy;
                if (busy) {
                    std::this_thread::yield();   // a batch in flight: poll its event again soon
                } else {
                    // nothing in flight: sleep until a query arrives or memory is
                    // released (bounded, in case admission waits on something else)
                    std::unique_lock<std::mutex> lk(mu);
                    cv_work.wait_for(lk, std::chrono::milliseconds(1), [&] {
                        return stop.load(std::memory_order_relaxed) || !pending.empty();
                    });
                }
            }
        }
    }

    int submit_at(const uint32_t *lists, size_t k, double t_arrival, bool auto_release, uint64_t *qid)
    {
        Query q;
        q.lists.assign(lists, lists + k);
        for (uint32_t j : q.lists) {
            if (j >= L) return VBYTE_EINVAL;
            q.n += vo[j + 1] - vo[j];
            q.bytes += bo[j + 1] - bo[j];
        }
        if (k == 0 || k > static_cast<size_t>(cfg.max_batch_lists) || q.bytes > cfg.staging_bytes ||
            (q.n * 4 + kArenaUnit - 1) / kArenaUnit > arena_units)
            return VBYTE_EINVAL;
        q.t_arrival = t_arrival;
        q.auto_release = auto_release;
        std::lock_guard<std::mutex> lk(mu);
        if (error != VBYTE_OK) return error;
        *qid = queries.size();
        queries.push_back(std::move(q));
        pending.push_back(*qid);
        cv_work.notify_one();
        return VBYTE_OK;
    }
};

extern "C" {

int vbyte_server_create(vbyte_server **out, const uint8_t *d_pool, size_t pool_bytes, const uint64_t *h_byte_off,
                        const uint64_t *h_val_off, size_t num_lists, int delta, const uint32_t *h_prev,
                        const vbyte_server_config *cfg)
{
    if (!out || !cfg || !h_byte_off || !h_val_off || num_lists == 0 || (pool_bytes && !d_pool)) return VBYTE_EINVAL;
    if (cfg->arena_bytes < kArenaUnit || cfg->staging_bytes == 0 || cfg->max_inflight < 1 ||
        cfg->max_batch_queries < 1 || cfg->max_batch_lists < 1 || cfg->per_list < 0 || cfg->per_list > 2)
        return VBYTE_EINVAL;
    *out = nullptr;
    if (h_byte_off[0] != 0 || h_byte_off[num_lists] != pool_bytes || h_val_off[0] != 0) return VBYTE_EINVAL;
    for (size_t j = 0; j < num_lists; ++j)
        if (h_byte_off[j + 1] < h_byte_off[j] || h_val_off[j + 1] < h_val_off[j]) return VBYTE_EINVAL;
    vbyte_server *S = new vbyte_server();
    cudaGetDevice(&S->dev);
    S->d_pool = d_pool;
    S->pool_bytes = pool_bytes;
    S->bo.assign(h_byte_off, h_byte_off + num_lists + 1);
    S->vo.assign(h_val_off, h_val_off + num_lists + 1);
    S->prev.assign(num_lists, 0u);
    if (delta && h_prev) S->prev.assign(h_prev, h_prev + num_lists);
    S->L = num_lists;
    S->delta = delta != 0;
    S->cfg = *cfg;
    S->arena_units = cfg->arena_bytes / kArenaUnit;
    auto fail = [&](int rc) {
        for (Slot &sl : S->slots) {
            if (sl.stream) {
                cudaStreamSynchronize(sl.stream);
                vbk::release_workspace(sl.stream);
                cudaStreamDestroy(sl.stream);
                sl.stream = nullptr;
            }
            if (sl.done) cudaEventDestroy(sl.done);
            if (sl.d_staging) cudaFree(sl.d_staging);
            if (sl.d_desc) cudaFree(sl.d_desc);
            if (sl.h_desc) cudaFreeHost(sl.h_desc);
            if (sl.h_status) cudaFreeHost(sl.h_status);
        }
        if (S->d_arena) cudaFree(S->d_arena);
        cudaGetLastError();
        delete S;
        return rc;
    };
    if (cudaMalloc(&S->d_arena, S->arena_units * kArenaUnit) != cudaSuccess) return fail(VBYTE_ENOMEM);
    S->free_units[0] = S->arena_units;
    uint64_t max_list = 0;
    for (size_t j = 0; j < num_lists; ++j) max_list = std::max(max_list, h_byte_off[j + 1] - h_byte_off[j]);
    const size_t nl = static_cast<size_t>(cfg->max_batch_lists);
    const size_t np = cfg->staging_bytes / kPieceBytes + nl + 1;
    const size_t desc = std::max((nl + 1) * 16 + nl * 4 + 16 + np * sizeof(vbk::GatherPiece),
                                 vbyte_server::items_desc_bytes(*cfg));
    S->slots.resize(static_cast<size_t>(cfg->max_inflight));
    for (Slot &sl : S->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) return fail(VBYTE_ECUDA);
        if (cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) return fail(VBYTE_ECUDA);
        if (cfg->per_list == 2 && cudaMalloc(&sl.d_staging, cfg->staging_bytes) != cudaSuccess)
            return fail(VBYTE_ENOMEM);
        if (cudaMalloc(&sl.d_desc, desc) != cudaSuccess) return fail(VBYTE_ENOMEM);
        if (cudaMallocHost(&sl.h_desc, desc) != cudaSuccess) return fail(VBYTE_ENOMEM);
        if (cudaMallocHost(&sl.h_status, 4) != cudaSuccess) return fail(VBYTE_ENOMEM);
        sl.desc_bytes = desc;
        // every workspace the loop will use is allocated now
        if (vbk::reserve_workspace(sl.stream, cfg->per_list == 1 ? max_list : cfg->staging_bytes) != VBYTE_OK)
            return fail(VBYTE_ENOMEM);
        uint32_t *d_status = nullptr;
        if (vbk::status_word(sl.stream, &d_status) != VBYTE_OK) return fail(VBYTE_ECUDA);
        cudaMemsetAsync(d_status, 0, 4, sl.stream);
        if (cudaStreamSynchronize(sl.stream) != cudaSuccess) return fail(VBYTE_ECUDA);
    }
    // kernel code is loaded now, not at the first query
    if (vbk::load_kernels() != VBYTE_OK || vbk::load_gather_kernel() != VBYTE_OK) return fail(VBYTE_ECUDA);
    S->worker = std::thread([S] { S->run(); });
    *out = S;
    return VBYTE_OK;
}

int vbyte_server_submit(vbyte_server *srv, const uint32_t *h_lists, size_t k, uint64_t *query_id)
{
    if (!srv || !h_lists || !query_id) return VBYTE_EINVAL;
    return srv->submit_at(h_lists, k, now_s(), false, query_id);
}

int vbyte_server_wait(vbyte_server *srv, uint64_t query_id, double *latency_s, uint32_t *status)
{
    if (!srv) return VBYTE_EINVAL;
    std::unique_lock<std::mutex> lk(srv->mu);
    if (query_id >= srv->queries.size()) return VBYTE_EINVAL;
    srv->cv.wait(lk, [&] { return srv->queries[query_id].state >= 2 || srv->error != VBYTE_OK; });
    if (srv->queries[query_id].state < 2) return srv->error;
    const Query &q = srv->queries[query_id];
    if (latency_s) *latency_s = q.t_done - q.t_arrival;
    if (status) *status = q.status;
    return VBYTE_OK;
}

int vbyte_server_result(vbyte_server *srv, uint64_t query_id, uint32_t **d_values, size_t *n,
                        uint32_t *batch_queries)
{
    if (!srv || !d_values || !n) return VBYTE_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (query_id >= srv->queries.size() || srv->queries[query_id].state != 2) return VBYTE_EINVAL;
    const Query &q = srv->queries[query_id];
    *d_values = srv->d_arena + q.out_off;
    *n = q.n;
    if (batch_queries) *batch_queries = q.batch_queries;
    return VBYTE_OK;
}

int vbyte_server_release(vbyte_server *srv, uint64_t query_id)
{
    if (!srv) return VBYTE_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (query_id >= srv->queries.size() || srv->queries[query_id].state != 2) return VBYTE_EINVAL;
    srv->release_locked(srv->queries[query_id]);
    return VBYTE_OK;
}

int vbyte_server_replay(vbyte_server *srv, const uint64_t *h_query_off, const uint32_t *h_query_lists,
                        size_t num_queries, const double *h_arrival_s, double *h_latency_s, uint32_t *h_status)
{
    if (!srv || (num_queries && (!h_query_off || !h_query_lists || !h_arrival_s || !h_latency_s)))
        return VBYTE_EINVAL;
    std::vector<uint64_t> ids(num_queries);
    const double t0 = now_s();
    for (size_t i = 0; i < num_queries; ++i) {
        const double target = t0 + h_arrival_s[i];
        for (;;) {   // open loop: wait for the query's arrival time
            const double dt = target - now_s();
            if (dt <= 0) break;
            if (dt > 200e-6) std::this_thread::sleep_for(std::chrono::duration<double>(dt - 100e-6));
        }
        const int rc = srv->submit_at(h_query_lists + h_query_off[i], h_query_off[i + 1] - h_query_off[i], target,
                                      true, &ids[i]);
        if (rc != VBYTE_OK) return rc;
    }
    for (size_t i = 0; i < num_queries; ++i) {
        uint32_t st = 0;
        const int rc = vbyte_server_wait(srv, ids[i], &h_latency_s[i], &st);
        if (rc != VBYTE_OK) return rc;
        if (h_status) h_status[i] = st;
    }
    return VBYTE_OK;
}

int vbyte_server_stats(vbyte_server *srv, uint64_t *batches, uint64_t *queries, uint64_t *values, uint64_t *lists)
{
    if (!srv) return VBYTE_EINVAL;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (batches) *batches = srv->n_batches;
    if (queries) *queries = srv->n_queries;
    if (values) *values = srv->n_values;
    if (lists) *lists = srv->n_lists;
    return srv->error;
}

void vbyte_server_destroy(vbyte_server *srv)
{
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        srv->cv_work.notify_all();
    }
    if (srv->worker.joinable()) srv->worker.join();
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(srv->dev);
    for (Slot &sl : srv->slots) {
        cudaStreamSynchronize(sl.stream);
        vbk::release_workspace(sl.stream);
        cudaStreamDestroy(sl.stream);
        cudaEventDestroy(sl.done);
        if (sl.d_staging) cudaFree(sl.d_staging);
        cudaFree(sl.d_desc);
        cudaFreeHost(sl.h_desc);
        cudaFreeHost(sl.h_status);
    }
    cudaFree(srv->d_arena);
    cudaSetDevice(cur);
    delete srv;
}

}  // extern "C"
