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
#include "hd_internal.h"

namespace hd {
namespace {

constexpr int kGenericWarps = 8;
constexpr int kSlot = 9;  // words per lane slot: 8 payload + 1 spare; odd stride avoids bank conflicts

__device__ __forceinline__ uint32_t get_bits(const uint32_t *a, uint32_t bit, uint32_t len)
{
    const uint32_t w = bit >> 5, sh = bit & 31u;
    const uint32_t v = sh ? __funnelshift_r(a[w], a[w + 1], sh) : a[w];
    return len >= 32 ? v : (v & ((1u << len) - 1u));
}

__device__ __forceinline__ void or_bits(uint32_t *a, uint32_t bit, uint32_t v, uint32_t len)
{
    const uint32_t w = bit >> 5, sh = bit & 31u;
    a[w] |= v << sh;
    if (sh != 0 && sh + len > 32) a[w + 1] |= v >> (32 - sh);
}

// Copy `len` bits from a[src..] to b[dst..] (b must be zero there).
__device__ __forceinline__ void copy_bits(const uint32_t *a, uint32_t src, uint32_t *b, uint32_t dst, uint32_t len)
{
    while (len > 0) {
        const uint32_t c = len < 32 ? len : 32;
        or_bits(b, dst, get_bits(a, src, c), c);
        src += c;
        dst += c;
        len -= c;
    }
}

// Checksum vector of a codeword held in the position domain y (bit p of the
// concatenated words is position p; bit 0 is not a position and is zero).
// Position p = 32w + j contributes j to the low five syndrome bits and w to
// the high bits, so the low bits come from the XOR of all words and the high
// bits from the parity of each word.
__device__ __forceinline__ uint32_t syndrome_y(const uint32_t (&y)[8], uint32_t wy)
{
    uint32_t f = 0, hi = 0;
#pragma unroll
    for (uint32_t w = 0; w < 8; ++w) {
        if (w < wy) {
            f ^= y[w];
            if (__popc(y[w]) & 1) hi ^= w;
        }
    }
    const uint32_t s = (__popc(f & 0xAAAAAAAAu) & 1u) | ((__popc(f & 0xCCCCCCCCu) & 1u) << 1) |
                       ((__popc(f & 0xF0F0F0F0u) & 1u) << 2) | ((__popc(f & 0xFF00FF00u) & 1u) << 3) |
                       ((__popc(f & 0xFFFF0000u) & 1u) << 4);
    return s | (hi << 5);
}

// Stream bits [start, start+32) with out-of-range words read as 0; start may
// be -1 (the bit before the first codeword), which reads as 0.
__device__ __forceinline__ uint32_t load_window(const uint32_t *__restrict__ in, uint64_t in_words, int64_t start)
{
    if (start < 0) return in_words ? (in[0] << 1) : 0u;
    const uint64_t a = (uint64_t)start >> 5;
    const uint32_t sh = (uint32_t)start & 31u;
    const uint32_t lo = a < in_words ? in[a] : 0u;
    if (sh == 0) return lo;
    const uint32_t hi = (a + 1 < in_words) ? in[a + 1] : 0u;
    return __funnelshift_r(lo, hi, sh);
}

template <int SYN>
__global__ void __launch_bounds__(kGenericWarps * 32)
    k_decode_generic(const uint32_t *__restrict__ in, uint64_t in_words, uint32_t n, uint32_t m, uint64_t num_cw,
                     uint64_t tile_begin, uint64_t tile_end, uint32_t *__restrict__ out, uint64_t out_words,
                     void *__restrict__ syn, unsigned long long *__restrict__ err)
{
    __shared__ uint32_t sy[kGenericWarps][32 * kSlot];
    __shared__ uint32_t sd[kGenericWarps][32 * kSlot];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    uint32_t *my_y = &sy[wp][lane * kSlot];
    uint32_t *my_d = &sd[wp][lane * kSlot];
    const uint32_t k = n - m;
    const uint32_t wy = (n + 1) <= 32 ? 1u : (n + 1) >> 5;
    unsigned long long cnt = 0;

    for (uint64_t t = tile_begin + (uint64_t)blockIdx.x * kGenericWarps + wp; t < tile_end;
         t += (uint64_t)gridDim.x * kGenericWarps) {
        const uint64_t i = t * 32 + lane;
        const bool valid = i < num_cw;
        // 1. received word in the position domain
        uint32_t y[8];
#pragma unroll
        for (uint32_t w = 0; w < 8; ++w)
            y[w] = (valid && w < wy) ? load_window(in, in_words, (int64_t)(i * n) - 1 + 32 * (int64_t)w) : 0u;
        if (n + 1 < 32) y[0] &= (1u << (n + 1)) - 1u;
        y[0] &= ~1u;
        // 2. checksum; 3. detect and correct (flip position s, branch-free)
        const uint32_t s = syndrome_y(y, wy);
#pragma unroll
        for (uint32_t w = 0; w < 8; ++w)
            if (w < wy) y[w] ^= shl_clamp(1u, s - 32u * w);
        // 4. redundancy removal: data run j = positions 2^j+1 .. 2^(j+1)-1
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            my_y[w] = y[w];
            my_d[w] = 0;
        }
        my_y[8] = 0;
        my_d[8] = 0;
        for (uint32_t j = 1; j < m; ++j)
            copy_bits(my_y, (1u << j) + 1u, my_d, (1u << j) - j - 1u, (1u << j) - 1u);
        __syncwarp();
        // 5. merge: output word q of the tile holds tile bits [32q, 32q+32)
        for (uint32_t q = lane; q < k; q += 32) {
            const uint64_t g = t * k + q;
            if (g >= out_words) break;
            uint32_t c = (32u * q) / k, o = 32u * q - c * k, v = 0, filled = 0;
            while (filled < 32 && c < 32) {
                const uint32_t avail = k - o, take = avail < 32 - filled ? avail : 32 - filled;
                v |= get_bits(&sd[wp][c * kSlot], o, take) << filled;
                filled += take;
                ++c;
                o = 0;
            }
            out[g] = v;
        }
        if (valid) {
            if (SYN == 1) static_cast<uint8_t *>(syn)[i] = (uint8_t)s;
            if (SYN == 2) static_cast<uint16_t *>(syn)[i] = (uint16_t)s;
        }
        cnt += __popc(__ballot_sync(0xFFFFFFFFu, valid && s != 0));
        __syncwarp();
    }
    if (err != nullptr && lane == 0 && cnt != 0) atomicAdd(err, cnt);
}

__global__ void __launch_bounds__(kGenericWarps * 32)
    k_encode_generic(const uint32_t *__restrict__ data, uint64_t data_words, uint32_t n, uint32_t m, uint64_t num_cw,
                     uint64_t tile_begin, uint64_t tile_end, uint32_t *__restrict__ stream, uint64_t stream_words)
{
    __shared__ uint32_t sy[kGenericWarps][32 * kSlot];
    __shared__ uint32_t sd[kGenericWarps][32 * kSlot];
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
    return (int)(want < cap ? want : cap);
}

}  // namespace

cudaError_t launch_decode_generic(const uint32_t *in, uint64_t in_words, uint32_t n, uint64_t num_cw,
                                  uint64_t tile_begin, uint64_t tile_end, uint32_t *out, uint64_t out_words,
                                  void *syn, int syn_type, unsigned long long *err, cudaStream_t st)
{
    if (tile_end <= tile_begin) return cudaSuccess;
    const uint32_t m = (uint32_t)code_m(n);
    const int grid = grid_for_tiles(tile_end - tile_begin);
    switch (syn_type) {
        case 1:
            k_decode_generic<1><<<grid, kGenericWarps * 32, 0, st>>>(in, in_words, n, m, num_cw, tile_begin, tile_end,
                                                                     out, out_words, syn, err);
            break;
        case 2:
            k_decode_generic<2><<<grid, kGenericWarps * 32, 0, st>>>(in, in_words, n, m, num_cw, tile_begin, tile_end,
                                                                     out, out_words, syn, err);
            break;
        default:
            k_decode_generic<0><<<grid, kGenericWarps * 32, 0, st>>>(in, in_words, n, m, num_cw, tile_begin, tile_end,
                                                                     out, out_words, syn, err);
            break;
    }
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
