// hd_copy.cu -- the piece-table copy kernel of the serving loop: packets
// submitted from pinned host memory are gathered into device staging before
// their wave's decode and the results scattered back after it, each direction
// one launch for the whole wave (the transfer stages T_PS and T_PR of the
// paper's asynchronous data transfer, Sec. III-B, Fig. 5).
#include "hd_batch_internal.h"
#include "hd_internal.h"

namespace hd {
namespace {

constexpr int kCopyThreads = 128;
constexpr int kCopyVecs = kPieceBytes / 16 / kCopyThreads;  // 16-byte vectors per thread
static_assert(kCopyVecs * 16 * kCopyThreads == (int)kPieceBytes, "a piece is one pass of the CTA");

// One CTA per piece (grid-strided): every thread issues all of its loads
// before its first store, so a CTA keeps a whole piece in flight, which
// hides the latency of reads from host memory; small pieces spread even a
// wave of a few packets over many SMs.
__global__ void __launch_bounds__(kCopyThreads) k_copy_pieces(const CopyPiece *__restrict__ pieces, uint32_t count)
{
    for (uint32_t pi = blockIdx.x; pi < count; pi += gridDim.x) {
        const CopyPiece pc = pieces[pi];
        const uint4 *src = static_cast<const uint4 *>(pc.src);
        uint4 *dst = static_cast<uint4 *>(pc.dst);
        const uint32_t nv = pc.bytes / 16u;
        uint4 v[kCopyVecs];
#pragma unroll
        for (int j = 0; j < kCopyVecs; ++j) {
            const uint32_t i = threadIdx.x + (uint32_t)j * kCopyThreads;
            if (i < nv) v[j] = src[i];
        }
#pragma unroll
        for (int j = 0; j < kCopyVecs; ++j) {
            const uint32_t i = threadIdx.x + (uint32_t)j * kCopyThreads;
            if (i < nv) dst[i] = v[j];
        }
        const uint32_t tail = pc.bytes & 15u;
        if (threadIdx.x < tail) {
            const uint32_t b = nv * 16u + threadIdx.x;
            static_cast<unsigned char *>(pc.dst)[b] = static_cast<const unsigned char *>(pc.src)[b];
        }
    }
}

}  // namespace

cudaError_t launch_copy_pieces(const CopyPiece *d_pieces, uint32_t count, cudaStream_t st)
{
    if (count == 0) return cudaSuccess;
    const int grid = (int)(count < 65535u ? count : 65535u);
    k_copy_pieces<<<grid, kCopyThreads, 0, st>>>(d_pieces, count);
    count_launch();
    return cudaGetLastError();
}

}  // namespace hd
