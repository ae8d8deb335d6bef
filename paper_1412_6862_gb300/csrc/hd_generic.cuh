// hd_generic.cuh -- the generic warp-tile decoder as device functions: one
// warp decodes whole 32-codeword tiles of any supported n straight from global
// memory, with bounds checks, so it covers ragged tails and short packets.
// Lane L decodes codeword 32t + L in registers; the lanes then merge their data
// bits into the tile's output words through per-lane shared-memory slots.
#pragma once

#include <cstdint>

#include "hd_device.cuh"

namespace hd {

constexpr int kSlot = 9;  // words per lane slot: 8 payload + 1 spare; odd stride avoids bank conflicts
constexpr int kWarpSlotWords = 32 * kSlot;


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

// Decode warp tiles [tile_begin, tile_end) of one stream with this warp
// (stride tile_step).  sy/sd: this warp's two shared slot areas of
// kWarpSlotWords words each.  syn_type is 0 (none), 1 (u8) or 2 (u16).
// Returns the number of nonzero syndromes this warp saw (same in all lanes).
__device__ __forceinline__ unsigned long long generic_decode_tiles(
    const uint32_t *__restrict__ in, uint64_t in_words, uint32_t n, uint32_t m, uint64_t num_cw, uint64_t tile_begin,
    uint64_t tile_end, uint64_t tile_step, uint32_t *__restrict__ out, uint64_t out_words, void *__restrict__ syn,
    int syn_type, uint32_t *sy, uint32_t *sd)
{
    const int lane = threadIdx.x & 31;
    uint32_t *my_y = &sy[lane * kSlot];
    uint32_t *my_d = &sd[lane * kSlot];
    const uint32_t k = n - m;
    const uint32_t wy = (n + 1) <= 32 ? 1u : (n + 1) >> 5;
    unsigned long long cnt = 0;

    for (uint64_t t = tile_begin; t < tile_end; t += tile_step) {
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
                v |= get_bits(&sd[c * kSlot], o, take) << filled;
                filled += take;
                ++c;
                o = 0;
            }
            out[g] = v;
        }
        if (valid) {
            if (syn_type == 1) static_cast<uint8_t *>(syn)[i] = (uint8_t)s;
            if (syn_type == 2) static_cast<uint16_t *>(syn)[i] = (uint16_t)s;
        }
        cnt += __popc(__ballot_sync(0xFFFFFFFFu, valid && s != 0));
        __syncwarp();
    }
    return cnt;
}

}  // namespace hd
