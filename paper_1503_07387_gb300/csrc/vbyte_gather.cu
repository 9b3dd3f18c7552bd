// Gather of compressed lists for the serving loop: copies pieces of the
// resident pool into a contiguous staging buffer, so that the lists of a
// batch of queries lie end to end for the batched decode.
#include <cuda_runtime.h>
#include <stdint.h>

#include "vbyte.h"
#include "vbyte_internal.h"

namespace vbk {

// One CTA per piece.  Where source and destination agree modulo 16 the body
// moves in 16-byte vectors; otherwise byte by byte (coalesced either way).
__global__ void __launch_bounds__(256) gather_kernel(const uint8_t *__restrict__ src, uint8_t *__restrict__ dst,
                                                     const GatherPiece *__restrict__ pieces)
{
    const GatherPiece pc = pieces[blockIdx.x];
    const uint8_t *s = src + pc.src;
    uint8_t *d = dst + pc.dst;
    const uint32_t len = pc.len;
    const int tid = threadIdx.x;
    const uintptr_t sa = reinterpret_cast<uintptr_t>(s), da = reinterpret_cast<uintptr_t>(d);
    if (((sa ^ da) & 15u) == 0 && len >= 64) {
        const uint32_t head = static_cast<uint32_t>((16u - (da & 15u)) & 15u);
        const uint32_t nvec = (len - head) / 16;
        const uint32_t tail0 = head + 16 * nvec;
        for (uint32_t i = tid; i < head; i += blockDim.x) d[i] = s[i];
        const uint4 *sv = reinterpret_cast<const uint4 *>(s + head);
        uint4 *dv = reinterpret_cast<uint4 *>(d + head);
        for (uint32_t i = tid; i < nvec; i += blockDim.x) dv[i] = sv[i];
        for (uint32_t i = tail0 + tid; i < len; i += blockDim.x) d[i] = s[i];
    } else {
        for (uint32_t i = tid; i < len; i += blockDim.x) d[i] = s[i];
    }
}

int load_gather_kernel()
{
    cudaFuncAttributes fa;
    return cudaFuncGetAttributes(&fa, gather_kernel) == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
}

int enqueue_gather(const uint8_t *src, uint8_t *dst, const GatherPiece *d_pieces, size_t num_pieces, cudaStream_t s)
{
    if (num_pieces == 0) return VBYTE_OK;
    if (num_pieces > 0x7FFFFFFFu) return VBYTE_EINVAL;
    gather_kernel<<<static_cast<unsigned>(num_pieces), 256, 0, s>>>(src, dst, d_pieces);
    return cudaGetLastError() == cudaSuccess ? VBYTE_OK : VBYTE_ECUDA;
}

}  // namespace vbk
