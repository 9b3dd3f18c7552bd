// libvbyte host side: per-stream workspaces, the list-head ranges of batched
// calls, the fixed scratch of vbyte_decode_noalloc, and the C entry points.
// The decoding kernels are in vbyte_stream.cu.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <utility>

#include "vbyte.h"
#include "vbyte_debug.h"
#include "vbyte_device.cuh"
#include "vbyte_internal.h"

namespace vbk {

constexpr int kTile = kHeadTile;   // the decoders' 4 KiB tiles

// ---- list-head ranges of batched calls

struct HeadRangeParams {
    const uint8_t *in;
    uint64_t nbytes;
    uint64_t n;
    uint64_t ntiles;
    uintptr_t base;            // 16-byte aligned address of tile 0
    const uint64_t *bo;
    const uint64_t *vo;
    uint64_t L;
    uint64_t *hr;
    uint32_t *status;
};

// For every tile, the range [first, end) of list indices whose byte offset
// lies in [tile start - kHeadBack, tile end) (binary searches over bo), and
// the offset arrays' contract: bo and vo non-decreasing from 0 to nbytes and
// n; a list that starts at the end of the bytes holds no values.
__device__ __forceinline__ uint64_t lower_bound_bo(const uint64_t *bo, uint64_t L, long long x)
{
    if (x <= 0) return 0;
    uint64_t lo = 0, hi = L + 1;
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (static_cast<long long>(bo[mid]) < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(256) head_range_kernel(const HeadRangeParams p)
{
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    const uint64_t i0 = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const long long in0 = static_cast<long long>(reinterpret_cast<uintptr_t>(p.in));
    uint64_t *hr = p.hr;
    for (uint64_t t = i0; t < p.ntiles; t += stride) {
        const long long trel = static_cast<long long>(p.base + t * kTile) - in0;
        uint64_t a = lower_bound_bo(p.bo, p.L, trel - kHeadBack);
        uint64_t e = lower_bound_bo(p.bo, p.L, trel + kTile);
        if (e > p.L) e = p.L;
        if (a > e) a = e;
        *reinterpret_cast<ulonglong2 *>(hr + 2 * t) = make_ulonglong2(a, e);
    }
    uint32_t bad = 0;
    for (uint64_t j = i0; j < p.L; j += stride) {
        if (p.bo[j] > p.bo[j + 1] || p.vo[j] > p.vo[j + 1]) bad |= VBYTE_ERR_BAD_OFFSETS;
        if (p.bo[j] == p.nbytes && p.vo[j] != p.n) bad |= VBYTE_ERR_COUNT_MISMATCH;
    }
    if (i0 == 0 && (p.bo[0] != 0 || p.vo[0] != 0 || p.bo[p.L] != p.nbytes || p.vo[p.L] != p.n))
        bad |= VBYTE_ERR_BAD_OFFSETS;
    if (bad) atomicOr(p.status, bad);
}

int enqueue_head_ranges(const uint8_t *in, size_t nbytes, const uint64_t *bo, const uint64_t *vo, size_t L,
                        size_t n, uint64_t *hr, uint32_t *status, int sms, cudaStream_t s)
{
    HeadRangeParams p = {};
    p.in = in;
    p.nbytes = nbytes;
    p.n = n;
    const uintptr_t a = reinterpret_cast<uintptr_t>(in);
    p.ntiles = nbytes ? ((a & 15u) + nbytes + kTile - 1) / kTile : 0;
    p.base = a & ~static_cast<uintptr_t>(15);
    p.bo = bo;
    p.vo = vo;
    p.L = L;
    p.hr = hr;
    p.status = status;
    const uint64_t work = std::max<uint64_t>(p.ntiles, L);
    const unsigned grid = static_cast<unsigned>(std::min<uint64_t>((work + 255) / 256, static_cast<uint64_t>(sms) * 8));
    head_range_kernel<<<std::max(grid, 1u), 256, 0, s>>>(p);
    return cudaGetLastError() == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
}

__global__ void set_status_kernel(uint32_t *status, uint32_t bits) { atomicOr(status, bits); }

// ---- fault injection (vbyte_debug.h)

std::atomic<uint64_t> g_skip_tile{~0ull};
std::atomic<uint64_t> g_wait_ns{kWaitLimitNs};

FaultCfg fault_cfg() { return FaultCfg{g_skip_tile.load(), g_wait_ns.load()}; }

std::atomic<int> g_passes{0};
int forced_passes() { return g_passes.load(); }

// The kernel for a single stream, by the mean code length nbytes / n (a
// length class) and the size, from measurements on GB300 (2^26..2^28
// values): small inputs take the single pass (fewest launches), one-byte
// codes count-then-decode in one launch (the input read once), the rest the
// split launches.
int choose_passes(size_t nbytes, size_t n, bool delta)
{
    const int f = forced_passes();
    if (f) return f;
    if (nbytes < (size_t(16) << 20) || n == 0) return 1;
    const double mean = static_cast<double>(nbytes) / static_cast<double>(n);
    if (mean < 1.1) return 2;
    return 3;
}

// ---- per-stream workspaces

// One workspace per (device, stream), grown on demand with cudaMallocAsync
// on that stream: [0, 4) the stream's status word, then the decoders'
// layouts (vbyte_stream.cu).  Host-call staging buffers are kept the same way.
constexpr size_t kWsHead = 256;

struct Workspace {
    uint8_t *ptr = nullptr;
    size_t cap = 0;
    bool caller = false;   // the caller's buffer (vbyte_set_workspace): never grown or freed here
};

struct HostBuffers {
    uint8_t *d_in = nullptr;
    size_t cap_in = 0;
    uint32_t *d_out = nullptr;
    size_t cap_out = 0;
};

std::mutex g_mu;
std::map<std::pair<int, uintptr_t>, Workspace> g_ws;
std::map<std::pair<int, uintptr_t>, HostBuffers> g_hb;

bool capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return false;
    return cs != cudaStreamCaptureStatusNone;
}

// Returns the workspace of (current device, s) with at least `need` bytes.
int get_workspace(cudaStream_t s, size_t need, Workspace **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VBYTE_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    Workspace &w = g_ws[{dev, reinterpret_cast<uintptr_t>(s)}];
    if (w.cap < need) {
        if (w.caller || capturing(s)) return VBYTE_ENOMEM;
        size_t cap = std::max<size_t>(need, std::max<size_t>(2 * w.cap, size_t(1) << 20));
        void *np = nullptr;
        if (cudaMallocAsync(&np, cap, s) != cudaSuccess) {
            cudaGetLastError();
            return VBYTE_ENOMEM;
        }
        if (w.ptr) {
            cudaMemcpyAsync(np, w.ptr, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
            cudaFreeAsync(w.ptr, s);
        } else {
            cudaMemsetAsync(np, 0, sizeof(uint32_t), s);
        }
        w.ptr = static_cast<uint8_t *>(np);
        w.cap = cap;
    }
    *out = &w;
    return VBYTE_OK;
}

int stream_workspace(cudaStream_t s, size_t need, uint8_t **ptr)
{
    Workspace *w = nullptr;
    const int rc = get_workspace(s, need, &w);
    if (rc == VBYTE_OK) *ptr = w->ptr;
    return rc;
}

int set_status_async(uint32_t *status, uint32_t bits, cudaStream_t s)
{
    set_status_kernel<<<1, 1, 0, s>>>(status, bits);
    return cudaGetLastError() == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
}

// Batched decoding: lists j in [0, L) are bytes [bo[j], bo[j+1]) of in and
// values [vo[j], vo[j+1]) of out; the concatenation is decoded as one stream
// whose running value (delta) restarts at prevs[j] at each list head.
int check_batch(const BatchArgs &a)
{
    if ((a.nbytes && !a.in) || (a.n && !a.out) || !a.bo || !a.vo) return VBYTE_EINVAL;
    if (reinterpret_cast<uintptr_t>(a.out) & 3u) return VBYTE_EINVAL;
    if ((reinterpret_cast<uintptr_t>(a.bo) | reinterpret_cast<uintptr_t>(a.vo)) & 7u) return VBYTE_EINVAL;
    if (a.prevs && (reinterpret_cast<uintptr_t>(a.prevs) & 3u)) return VBYTE_EINVAL;
    if (a.L == 0 && (a.nbytes || a.n)) return VBYTE_EINVAL;
    return VBYTE_OK;
}

int status_word(cudaStream_t s, uint32_t **word)
{
    Workspace *w = nullptr;
    const int rc = get_workspace(s, kWsHead, &w);
    if (rc == VBYTE_OK) *word = reinterpret_cast<uint32_t *>(w->ptr);
    return rc;
}

void release_workspace(cudaStream_t s)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_ws.find({dev, reinterpret_cast<uintptr_t>(s)});
    if (it != g_ws.end()) {
        if (it->second.ptr && !it->second.caller) cudaFreeAsync(it->second.ptr, s);
        g_ws.erase(it);
    }
    auto ih = g_hb.find({dev, reinterpret_cast<uintptr_t>(s)});
    if (ih != g_hb.end()) {
        if (ih->second.d_in) cudaFreeAsync(ih->second.d_in, s);
        if (ih->second.d_out) cudaFreeAsync(ih->second.d_out, s);
        g_hb.erase(ih);
    }
}

int launch_decode_batched(const BatchArgs &a, cudaStream_t s)
{
    int rc = check_batch(a);
    if (rc != VBYTE_OK || a.L == 0) return rc;
    Workspace *w = nullptr;
    rc = get_workspace(s, sbatched_workspace_bytes(a), &w);
    if (rc != VBYTE_OK) return rc;
    return enqueue_sbatched(a, w->ptr, LaunchCfg(), s);
}

// ---- scratch for vbyte_decode_noalloc
// A file-scope device array replaces the per-stream workspace for callers
// that cannot allocate device memory.  It holds the single-stream layout of
// an input of up to VBYTE_NOALLOC_MAX_BYTES bytes (about 513 KiB); every call
// on a device shares it.
constexpr size_t kStaticScratchBytes = size_t(576) << 10;
static __device__ __align__(256) uint8_t g_scratch[kStaticScratchBytes];

constexpr int kMaxStaticDevices = 64;
std::mutex g_static_mu;
uint8_t *g_static_ptr[kMaxStaticDevices] = {};

// Set-up, once per device, with that device current: the address of
// g_scratch on it.  No allocation.
int static_scratch(uint8_t **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VBYTE_ECUDA;
    if (dev < 0 || dev >= kMaxStaticDevices) return VBYTE_EINVAL;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            return VBYTE_ECUDA;
        }
        g_static_ptr[dev] = static_cast<uint8_t *>(ptr);
    }
    *out = g_static_ptr[dev];
    return VBYTE_OK;
}

int launch_decode_noalloc(const uint8_t *in, size_t nbytes, uint32_t *out, size_t n, bool delta, uint32_t prev,
                          uint32_t *status, cudaStream_t s)
{
    if (nbytes > VBYTE_NOALLOC_MAX_BYTES) return VBYTE_ETOOBIG;
    if ((nbytes && !in) || (n && !out)) return VBYTE_EINVAL;
    if (reinterpret_cast<uintptr_t>(out) & 3u) return VBYTE_EINVAL;
    if (reinterpret_cast<uintptr_t>(status) & 3u) return VBYTE_EINVAL;
    uint8_t *scratch = nullptr;
    int rc = static_scratch(&scratch);
    if (rc != VBYTE_OK) return rc;
    if (nbytes == 0 && n == 0) return VBYTE_OK;
    if (stream_workspace_bytes(in, nbytes) > kStaticScratchBytes) return VBYTE_ETOOBIG;
    // without a caller status word, data errors go to the array's own head
    if (status == nullptr) status = reinterpret_cast<uint32_t *>(scratch);
    if (nbytes == 0) return set_status_async(status, VBYTE_ERR_COUNT_MISMATCH, s);   // n > 0 from no bytes
    return enqueue_stream(in, nbytes, out, n, delta, prev, scratch, status, s);
}

// Make ptr (caller-owned, bytes long) the workspace of (current device, s),
// or with ptr == nullptr hand the stream back to library allocations; the
// status word carries over either way.
int set_workspace(cudaStream_t s, uint8_t *ptr, size_t bytes)
{
    if (ptr && ((reinterpret_cast<uintptr_t>(ptr) & 255u) || bytes < workspace_bound(0))) return VBYTE_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VBYTE_ECUDA;
    if (capturing(s)) return VBYTE_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    Workspace &w = g_ws[{dev, reinterpret_cast<uintptr_t>(s)}];
    if (!ptr) {
        if (!w.caller) return VBYTE_OK;   // already the library's
        const size_t cap = size_t(1) << 20;
        void *np = nullptr;
        if (cudaMallocAsync(&np, cap, s) != cudaSuccess) {
            cudaGetLastError();
            return VBYTE_ENOMEM;
        }
        if (cudaMemcpyAsync(np, w.ptr, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return VBYTE_ECUDA;
        w.ptr = static_cast<uint8_t *>(np);
        w.cap = cap;
        w.caller = false;
        return VBYTE_OK;
    }
    if (ptr == w.ptr) {
        w.cap = bytes;   // the same buffer again, perhaps with a new length
        w.caller = true;
        return VBYTE_OK;
    }
    if (w.ptr) {
        if (cudaMemcpyAsync(ptr, w.ptr, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return VBYTE_ECUDA;
        if (!w.caller) cudaFreeAsync(w.ptr, s);
    } else if (cudaMemsetAsync(ptr, 0, sizeof(uint32_t), s) != cudaSuccess) {
        return VBYTE_ECUDA;
    }
    w.ptr = ptr;
    w.cap = bytes;
    w.caller = true;
    return VBYTE_OK;
}

int reserve_workspace(cudaStream_t s, size_t nbytes)
{
    Workspace *w = nullptr;
    return get_workspace(s, workspace_bound(nbytes), &w);
}

}  // namespace vbk

extern "C" {

int vbyte_decode(const uint8_t *d_in, size_t nbytes, uint32_t *d_out, size_t n, void *stream)
{
    return vbk::launch_decode(d_in, nbytes, d_out, n, false, 0u, static_cast<cudaStream_t>(stream));
}

int vbyte_decode_delta(const uint8_t *d_in, size_t nbytes, uint32_t *d_out, size_t n, uint32_t prev,
                       void *stream)
{
    return vbk::launch_decode(d_in, nbytes, d_out, n, true, prev, static_cast<cudaStream_t>(stream));
}

int vbyte_decode_delta_m1(const uint8_t *d_in, size_t nbytes, uint32_t *d_out, size_t n, uint32_t prev,
                          void *stream)
{
    return vbk::launch_decode(d_in, nbytes, d_out, n, true, prev, static_cast<cudaStream_t>(stream), true);
}

int vbyte_decode_delta4(const uint8_t *d_in, size_t nbytes, uint32_t *d_out, size_t n, const uint32_t *h_prev4,
                        void *stream)
{
    if (nbytes == 0 && n == 0) return VBYTE_OK;
    if ((nbytes && !d_in) || (n && !d_out)) return VBYTE_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_out) & 3u) return VBYTE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t *ws = nullptr;
    const int rc = vbk::stream_workspace(s, vbk::stream_workspace_bytes_any(d_in, nbytes), &ws);
    if (rc != VBYTE_OK) return rc;
    uint32_t *status = reinterpret_cast<uint32_t *>(ws);
    if (nbytes == 0) return vbk::set_status_async(status, VBYTE_ERR_COUNT_MISMATCH, s);   // n > 0 from no bytes
    const uint32_t zeros[4] = {0u, 0u, 0u, 0u};
    return vbk::enqueue_split(d_in, nbytes, d_out, n, false, 0u, ws, status, s, false, h_prev4 ? h_prev4 : zeros);
}

int vbyte_decode_batched(const uint8_t *d_in, size_t nbytes, const uint64_t *d_byte_off, uint32_t *d_out,
                         size_t n, const uint64_t *d_val_off, size_t num_lists, void *stream)
{
    const vbk::BatchArgs a{d_in, nbytes, d_byte_off, d_out, n, d_val_off, num_lists, nullptr, false};
    return vbk::launch_decode_batched(a, static_cast<cudaStream_t>(stream));
}

int vbyte_decode_delta_batched(const uint8_t *d_in, size_t nbytes, const uint64_t *d_byte_off, uint32_t *d_out,
                               size_t n, const uint64_t *d_val_off, size_t num_lists, const uint32_t *d_prev,
                               void *stream)
{
    const vbk::BatchArgs a{d_in, nbytes, d_byte_off, d_out, n, d_val_off, num_lists, d_prev, true};
    return vbk::launch_decode_batched(a, static_cast<cudaStream_t>(stream));
}

int vbyte_decode_host(const uint8_t *h_in, size_t nbytes, uint32_t *h_out, size_t n, int delta,
                      uint32_t prev, void *stream)
{
    if ((nbytes && !h_in) || (n && !h_out)) return VBYTE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VBYTE_ECUDA;
    vbk::HostBuffers *hb;
    {
        std::lock_guard<std::mutex> lk(vbk::g_mu);
        hb = &vbk::g_hb[{dev, reinterpret_cast<uintptr_t>(s)}];
        if (hb->cap_in < nbytes) {
            if (hb->d_in) cudaFreeAsync(hb->d_in, s);
            hb->d_in = nullptr;
            hb->cap_in = 0;
            void *p = nullptr;
            if (cudaMallocAsync(&p, nbytes, s) != cudaSuccess) return VBYTE_ENOMEM;
            hb->d_in = static_cast<uint8_t *>(p);
            hb->cap_in = nbytes;
        }
        if (hb->cap_out < n) {
            if (hb->d_out) cudaFreeAsync(hb->d_out, s);
            hb->d_out = nullptr;
            hb->cap_out = 0;
            void *p = nullptr;
            if (cudaMallocAsync(&p, n * sizeof(uint32_t), s) != cudaSuccess) return VBYTE_ENOMEM;
            hb->d_out = static_cast<uint32_t *>(p);
            hb->cap_out = n;
        }
    }
    // large inputs: pieces copied in, decoded and copied back with the copies
    // in both directions and the kernels overlapping
    if (nbytes >= 2 * vbk::kPipePiece && n) {
        uint8_t *ws = nullptr;
        int rc = vbk::stream_workspace(s, vbk::pipe_workspace_bytes(nbytes), &ws);
        if (rc != VBYTE_OK) return rc;
        return vbk::decode_host_pipelined(h_in, nbytes, h_out, n, delta != 0, prev, hb->d_in, hb->d_out, ws,
                                          reinterpret_cast<uint32_t *>(ws), s, vbk::kPipePiece);
    }
    if (nbytes && cudaMemcpyAsync(hb->d_in, h_in, nbytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return VBYTE_ECUDA;
    int rc = vbk::launch_decode(hb->d_in, nbytes, hb->d_out, n, delta != 0, prev, s);
    if (rc != VBYTE_OK) return rc;
    if (n && cudaMemcpyAsync(h_out, hb->d_out, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return VBYTE_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
}

int vbyte_decode_noalloc(const uint8_t *d_in, size_t nbytes, uint32_t *d_out, size_t n, int delta,
                         uint32_t prev, uint32_t *d_status, void *stream)
{
    return vbk::launch_decode_noalloc(d_in, nbytes, d_out, n, delta != 0, prev, d_status,
                                      static_cast<cudaStream_t>(stream));
}

int vbyte_get_status(void *stream, uint32_t *status_out)
{
    if (!status_out) return VBYTE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    vbk::Workspace *w = nullptr;
    int rc = vbk::get_workspace(s, vbk::kWsHead, &w);
    if (rc != VBYTE_OK) return rc;
    uint32_t v = 0;
    if (cudaMemcpyAsync(&v, w->ptr, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess) return VBYTE_ECUDA;
    if (cudaMemsetAsync(w->ptr, 0, sizeof(uint32_t), s) != cudaSuccess) return VBYTE_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return VBYTE_ECUDA;
    *status_out = v;
    return VBYTE_OK;
}

const char *vbyte_strerror(int code)
{
    switch (code) {
    case VBYTE_OK: return "ok";
    case VBYTE_EINVAL: return "invalid argument (null pointer with nonzero size or misaligned output)";
    case VBYTE_ECUDA: return "CUDA runtime error or kernel launch failure";
    case VBYTE_ENOMEM: return "workspace allocation failed (or needed during stream capture)";
    case VBYTE_ETOOBIG: return "input larger than VBYTE_NOALLOC_MAX_BYTES (vbyte_decode_noalloc)";
    default: return "unknown vbyte error code";
    }
}

size_t vbyte_workspace_size(size_t nbytes) { return vbk::workspace_bound(nbytes); }

int vbyte_debug_force_passes(int passes)
{
    if (passes < 0 || passes > 4) return VBYTE_EINVAL;
    vbk::g_passes.store(passes);
    return VBYTE_OK;
}

int vbyte_debug_passes_for(size_t nbytes, size_t n, int delta)
{
    return vbk::choose_passes(nbytes, n, delta != 0);
}

int vbyte_debug_inject(long long skip_tile, uint64_t wait_limit_ns)
{
    if (wait_limit_ns > vbk::kWaitLimitNs) return VBYTE_EINVAL;
    vbk::g_skip_tile.store(skip_tile < 0 ? ~0ull : static_cast<uint64_t>(skip_tile));
    vbk::g_wait_ns.store(wait_limit_ns ? wait_limit_ns : vbk::kWaitLimitNs);
    return VBYTE_OK;
}

int vbyte_set_workspace(void *stream, void *d_ws, size_t bytes)
{
    return vbk::set_workspace(static_cast<cudaStream_t>(stream), static_cast<uint8_t *>(d_ws), bytes);
}

int vbyte_release_stream(void *stream)
{
    vbk::release_workspace(static_cast<cudaStream_t>(stream));
    return VBYTE_OK;
}

}  // extern "C"
