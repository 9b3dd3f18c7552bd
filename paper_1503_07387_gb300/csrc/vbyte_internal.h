// Internal interface between the decode kernels (vbyte_stream.cu), the host
// side of the library (vbyte_api.cu: workspaces, entry points) and the
// runtime built on them (vbyte_runtime.cpp: batched plans and the
// one-call-per-list form; vbyte_server.cpp: the serving loop).  Not
// installed; not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace vbk {

constexpr uint64_t kDefaultLeadSlack = 4608;

// One batched decode: list j is bytes [bo[j], bo[j+1]) of in and values
// [vo[j], vo[j+1]) of out (bo, vo, prevs in device memory).
struct BatchArgs {
    const uint8_t *in;
    size_t nbytes;
    const uint64_t *bo;
    uint32_t *out;
    size_t n;
    const uint64_t *vo;
    size_t L;
    const uint32_t *prevs;
    bool delta;
};

// Launch parameters of the batched kernel (the plan autotuner's choices).
struct LaunchCfg {
    int ctas_per_sm = 0;                        // 0: the occupancy limit
    uint64_t lead_slack = kDefaultLeadSlack;    // tickets between a chunk's last count and first decode
};

int check_batch(const BatchArgs &a);
// Fault injection for tests of the bounded waits (vbyte_debug.h): the tile
// whose count descriptor later decode launches leave unpublished (~0: none)
// and the bound of every wait in them (ns).
struct FaultCfg {
    uint64_t skip_tile;
    uint64_t wait_ns;
};
FaultCfg fault_cfg();
// 0: the library's choice of kernel; 1, 2 or 3: that kernel (tests).
int forced_passes();
// The per-stream workspace of s (current device) with at least need bytes;
// its first 4 bytes are the stream's status word.
int stream_workspace(cudaStream_t s, size_t need, uint8_t **ptr);
// OR bits into a device status word, on s.
int set_status_async(uint32_t *status, uint32_t bits, cudaStream_t s);
// Workspace bytes of the single-stream decoder for an input at `in`.
size_t stream_workspace_bytes(const uint8_t *in, size_t nbytes);
// Enough workspace for any single-stream or batched call on nbytes.
size_t workspace_bound(size_t nbytes);
// Queue a checked single-stream decode (nbytes > 0) with its scratch in ws
// (stream_workspace_bytes) and data errors OR-ed into *status.  rank (delta
// only): the gaps-minus-one variant, every value plus its rank.
// passes: 2 = count-then-decode (the workspace layout of
// stream_workspace_bytes), 1 = single pass with a decoupled look-back, 3 = the
// split count / scan / decode launches, 4 = the split launches decoding by the
// table-driven steps of Sec. 4 (1, 3 and 4 need stream_workspace_bytes_any).
int enqueue_stream(const uint8_t *in, size_t nbytes, uint32_t *out, size_t n, bool delta, uint32_t prev,
                   uint8_t *ws, uint32_t *status, cudaStream_t s, bool rank = false, int passes = 2);
// Workspace bytes for a single-stream call with any of the kernels.
size_t stream_workspace_bytes_any(const uint8_t *in, size_t nbytes);
// The split decoder (vbyte_split.cu): count, scan and decode launches with no
// wait between CTAs; its workspace for an input at `in`, and for any
// alignment.
size_t split_workspace_bytes(const uint8_t *in, size_t nbytes);
size_t split_workspace_bound(size_t nbytes);
// prev4 (host, four values): the blocked-difference form (delta and rank
// false), x_i = g_i + x_{i-4} with x_{-4..-1} = prev4[0..3].
// table: decode by the table-driven steps of Sec. 4 (vbyte_table.cuh) in
// place of per-terminator assembly.
int enqueue_split(const uint8_t *in, size_t nbytes, uint32_t *out, size_t n, bool delta, uint32_t prev,
                  uint8_t *ws, uint32_t *status, cudaStream_t s, bool rank, const uint32_t *prev4 = nullptr,
                  bool table = false);
// The kernel vbyte_decode* use for an input of nbytes holding n values:
// 1 (single pass), 2 (count-then-decode) or 3 (split).
int choose_passes(size_t nbytes, size_t n, bool delta);
// The single-stream call with the per-stream workspace.
int launch_decode(const uint8_t *in, size_t nbytes, uint32_t *out, size_t n, bool delta, uint32_t prev,
                  cudaStream_t s, bool rank = false);
// The batched call with the per-stream workspace.
int launch_decode_batched(const BatchArgs &a, cudaStream_t s);
// Grow the per-stream workspace of s (current device) for single-stream and
// batched inputs of up to nbytes, so that later calls need no allocation.
int reserve_workspace(cudaStream_t s, size_t nbytes);
// The device status word of s's workspace (allocating a minimal one if none).
int status_word(cudaStream_t s, uint32_t **word);
// Free s's workspace (queued on s; call before destroying s).
void release_workspace(cudaStream_t s);

// For every 4 KiB tile of `in` (tile 0 at `in` rounded down to 16 bytes):
// the range of lists whose first byte lies in [tile start - 8, tile end),
// as two uint64 per tile in hr; also checks the offset arrays' contract.
int enqueue_head_ranges(const uint8_t *in, size_t nbytes, const uint64_t *bo, const uint64_t *vo, size_t L,
                        size_t n, uint64_t *hr, uint32_t *status, int sms, cudaStream_t s);
// Batched decode (vbyte_stream.cu): its scratch in ws (sbatched_workspace_bytes;
// ws[0..4) is the status word).
size_t sbatched_workspace_bytes(const BatchArgs &a);
int sbatched_max_ctas(bool delta);   // CTAs per SM of that kernel
// Load the decoders' code and query their occupancy now (not at first use).
int load_kernels();
int enqueue_sbatched(const BatchArgs &a, uint8_t *ws, const LaunchCfg &cfg, cudaStream_t s);

// Batched decoding as list items (vbyte_split.cu, for tuned plans): a whole
// list, or a chunk of a long one, per item; one warp decodes an item.
struct ListItem {
    unsigned long long b0, b1;   // input bytes [b0, b1) whose terminators the item owns
    uint32_t list;
    uint32_t flags;              // kItemOnly: the list's only item; kItemLast: it ends the list
};
constexpr uint32_t kItemOnly = 1u, kItemLast = 2u;
// Device arrays of one item set (owned by the plan).
struct ListPlan {
    ListItem *items;     // decode order (longest first)
    uint32_t nitems;
    uint32_t *citem;     // items of chunked lists, list by list, in chunk order
    uint32_t *cfirst;    // per chunked list its first citem entry, then the number of entries
    uint32_t ncl;        // chunked lists
    uint2 *cs;           // per item: count and sum
    uint2 *rel;          // per item: count and sum of its list's earlier chunks (zeros at creation)
    unsigned int *queue;
};
// table: the items' units decoded by the table-driven steps of Sec. 4.
int enqueue_list_plan(const BatchArgs &a, const ListPlan &lp, int warps_per_cta, uint32_t *status, cudaStream_t s,
                      bool table = false);

// Decoding from host buffers in pieces of about kPipePiece bytes with the
// copies and kernels overlapping (vbyte_split.cu); d_in and d_out hold the
// whole input and output, ws pipe_workspace_bytes(nbytes).
constexpr size_t kPipePiece = size_t(64) << 20;
size_t pipe_workspace_bytes(size_t nbytes);
int decode_host_pipelined(const uint8_t *h_in, size_t nbytes, uint32_t *h_out, size_t n, bool delta, uint32_t prev,
                          uint8_t *d_in, uint32_t *d_out, uint8_t *ws, uint32_t *status, cudaStream_t s,
                          size_t piece_bytes);

// A piece of a gather: len bytes from src + src_off to dst + dst_off.
struct GatherPiece {
    uint64_t src;
    uint64_t dst;
    uint32_t len;
    uint32_t pad;
};
// Load the gather kernel's code now rather than at its first launch.
int load_gather_kernel();
// Queue the copy of every piece (device array) from src to dst on s.
int enqueue_gather(const uint8_t *src, uint8_t *dst, const GatherPiece *d_pieces, size_t num_pieces, cudaStream_t s);

}  // namespace vbk
