// hd_generic.cu -- warp-tile decoder and encoder for every supported n.
//
// One warp handles one warp tile of 32 consecutive codewords: n input words
// and k output words (n is odd, so 32 codewords always fill whole words).
// Lane L decodes codeword 32t + L in registers; the lanes then merge their
// data bits into the tile's output words through shared memory.  These
// kernels cover any n, any stream length and every ragged tail; the
// specialised streaming kernels of hd_decode.cu take the bulk of long streams.
#include <cstdint>

#include "hd_device.cuh"
#include "hd_generic.cuh"
#include "hd_internal.h"

namespace hd {
namespace {

constexpr int kGenericWarps = 8;

__global__ void __launch_bounds__(kGenericWarps * 32)
    k_decode_generic(const uint32_t *__restrict__ in, uint64_t in_words, uint32_t n, uint32_t m, uint64_t num_cw,
                     uint64_t tile_begin, uint64_t tile_end, uint32_t *__restrict__ out, uint64_t out_words,
                     void *__restrict__ syn, int syn_type, unsigned long long *__restrict__ err)
{
    __shared__ uint32_t sy[kGenericWarps][kWarpSlotWords];
    __shared__ uint32_t sd[kGenericWarps][kWarpSlotWords];
    const int wp = threadIdx.x >> 5;
    const unsigned long long cnt =
        generic_decode_tiles(in, in_words, n, m, num_cw, tile_begin + (uint64_t)blockIdx.x * kGenericWarps + wp,
                             tile_end, (uint64_t)gridDim.x * kGenericWarps, out, out_words, syn, syn_type, sy[wp],
                             sd[wp]);
    if (err != nullptr && (threadIdx.x & 31) == 0 && cnt != 0) atomicAdd(err, cnt);
}

__global__ void __launch_bounds__(kGenericWarps * 32)
    k_encode_generic(const uint32_t *__restrict__ data, uint64_t data_words, uint32_t n, uint32_t m, uint64_t num_cw,
                     uint64_t tile_begin, uint64_t tile_end, uint32_t *__restrict__ stream, uint64_t stream_words)
{
    __shared__ uint32_t sy[kGenericWarps][kWarpSlotWords];
    __shared__ uint32_t sd[kGenericWarps][kWarpSlotWords];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    uint32_t *my_y = &sy[wp][lane * kSlot];
    uint32_t *my_d = &sd[wp][lane * kSlot];
    const uint32_t k = n - m;
    const uint32_t wy = (n + 1) <= 32 ? 1u : (n + 1) >> 5;

    for (uint64_t t = tile_begin + (uint64_t)blockIdx.x * kGenericWarps + wp; t < tile_end;
         t += (uint64_t)gridDim.x * kGenericWarps) {
        const uint64_t i = t * 32 + lane;
        const bool valid = i < num_cw;
        // message bits of codeword i
        const uint32_t dw = (k + 31) >> 5;
#pragma unroll
        for (uint32_t w = 0; w < 8; ++w) {
            uint32_t v = 0;
            if (valid && w < dw) {
                v = load_window(data, data_words, (int64_t)(i * k) + 32 * (int64_t)w);
                const uint32_t left = k - 32 * w;
                if (left < 32) v &= (1u << left) - 1u;
            }
            my_d[w] = v;
            my_y[w] = 0;
        }
        my_d[8] = 0;
        my_y[8] = 0;
        // data bits to the non-power-of-two positions
        for (uint32_t j = 1; j < m; ++j)
            copy_bits(my_d, (1u << j) - j - 1u, my_y, (1u << j) + 1u, (1u << j) - 1u);
        uint32_t y[8];
#pragma unroll
        for (int w = 0; w < 8; ++w) y[w] = my_y[w];
        // checksum bit j goes to position 2^j, making the syndrome 0
        const uint32_t s = syndrome_y(y, wy);
        for (uint32_t j = 0; j < m; ++j) {
            const uint32_t p = 1u << j;
            if ((s >> j) & 1u) my_y[p >> 5] |= 1u << (p & 31u);
        }
        __syncwarp();
        // merge: stream word q of the tile holds tile bits [32q, 32q+32)
        for (uint32_t q = lane; q < n; q += 32) {
            const uint64_t g = t * n + q;
            if (g >= stream_words) break;
            uint32_t c = (32u * q) / n, o = 32u * q - c * n, v = 0, filled = 0;
            while (filled < 32 && c < 32) {
                const uint32_t avail = n - o, take = avail < 32 - filled ? avail : 32 - filled;
                v |= get_bits(&sy[wp][c * kSlot], o + 1, take) << filled;
                filled += take;
                ++c;
                o = 0;
            }
            stream[g] = v;
        }
        __syncwarp();
    }
}

int grid_for_tiles(uint64_t tiles)
{
    const uint64_t want = (tiles + kGenericWarps - 1) / kGenericWarps;
    const uint64_t cap = (uint64_t)num_sms() * 8;
    return decode_grid(want, cap);
}

}  // namespace

cudaError_t launch_decode_generic(const uint32_t *in, uint64_t in_words, uint32_t n, uint64_t num_cw,
                                  uint64_t tile_begin, uint64_t tile_end, uint32_t *out, uint64_t out_words,
                                  void *syn, int syn_type, unsigned long long *err, cudaStream_t st)
{
    if (tile_end <= tile_begin) return cudaSuccess;
    const uint32_t m = (uint32_t)code_m(n);
    const int grid = grid_for_tiles(tile_end - tile_begin);
    k_decode_generic<<<grid, kGenericWarps * 32, 0, st>>>(in, in_words, n, m, num_cw, tile_begin, tile_end, out,
                                                          out_words, syn, syn_type, err);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_encode_generic(const uint32_t *data, uint64_t data_words, uint32_t n, uint64_t num_cw,
                                  uint32_t *stream, uint64_t stream_words, cudaStream_t st)
{
    const uint64_t tiles = (num_cw + 31) / 32;
    if (tiles == 0) return cudaSuccess;
    const uint32_t m = (uint32_t)code_m(n);
    k_encode_generic<<<grid_for_tiles(tiles), kGenericWarps * 32, 0, st>>>(data, data_words, n, m, num_cw, 0, tiles,
                                                                          stream, stream_words);
    count_launch();
    return cudaGetLastError();
}

}  // namespace hd
