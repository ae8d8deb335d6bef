// hd_tile.cuh -- the per-thread decode of one "thread tile": 32 consecutive
// codewords of a compile-time length n.  32 codewords of odd length fill
// exactly n input words and k output words, so every bit offset inside the
// tile is a compile-time constant once the codeword loop is unrolled: each
// codeword is pulled out with one funnel shift and its data bits are packed
// with constant shifts, with no cross-thread exchange.
//
// The steps follow the decoder of Sec. II-III of the paper (checksum, error
// detection and correction, redundancy removal, merge), restated for 32-bit
// words:
//  * position domain: y = the codeword shifted up by one bit, so bit p of y is
//    position p (Sec. III-A numbers positions from 1; bit 0 is unused);
//  * checksum bit i = parity(y & I_i) where I_i is the index set of Sec. III-A
//    as a mask; for codewords longer than a word, position p = 32w + j
//    contributes j to the low five bits and w to the high bits, so the low bits
//    come from the XOR of the words and the high bits from word parities;
//  * correction flips bit s of y branch-free (s = 0 flips the unused bit 0);
//  * redundancy removal keeps the runs between power-of-two positions.
#pragma once

#include "hd_device.cuh"

namespace hd {

// Bits j of a 32-bit word whose index j has bit i set (i < 5).
__host__ __device__ constexpr uint32_t bmask(int i)
{
    return i == 0 ? 0xAAAAAAAAu : i == 1 ? 0xCCCCCCCCu : i == 2 ? 0xF0F0F0F0u : i == 3 ? 0xFF00FF00u : 0xFFFF0000u;
}

// Four pending words held as scalars (an array here defeats scalar
// replacement once two packers are live and lands in local memory).
struct Pend4 {
    uint32_t p0 = 0, p1 = 0, p2 = 0, p3 = 0;
    __device__ __forceinline__ void set(int i, uint32_t v)
    {
        if (i == 0) p0 = v;
        else if (i == 1) p1 = v;
        else if (i == 2) p2 = v;
        else p3 = v;
    }
};

// Output bit packer with compile-time position: appends pieces of `len` clean
// bits and stores each completed word (in vectors of V words when the thread's
// output region is aligned for it).
template <int V>
struct OutPacker {
    uint32_t *dst;
    uint32_t acc = 0;
    int pos = 0;  // bits already in acc
    int q = 0;    // index of the word acc will become
    Pend4 pend;

    __device__ __forceinline__ explicit OutPacker(uint32_t *d) : dst(d) {}

    __device__ __forceinline__ void store(uint32_t w)
    {
        if constexpr (V == 1) {
            dst[q] = w;
        } else {
            pend.set(q % V, w);
            if (q % V == V - 1) {
                if constexpr (V == 2)
                    *reinterpret_cast<uint2 *>(dst + q - 1) = make_uint2(pend.p0, pend.p1);
                else
                    *reinterpret_cast<uint4 *>(dst + q - 3) = make_uint4(pend.p0, pend.p1, pend.p2, pend.p3);
            }
        }
        ++q;
    }

    // v must have no bits at or above `len`.
    __device__ __forceinline__ void append(uint32_t v, int len)
    {
        if (pos == 0)
            acc = v;
        else
            acc |= v << pos;
        if (pos + len >= 32) {
            store(acc);
            acc = (pos + len > 32) ? (v >> (32 - pos)) : 0u;
            pos = pos + len - 32;
        } else {
            pos += len;
        }
    }
};

// Syndrome packer: 4 (u8) or 2 (u16) syndromes per word; also counts the
// nonzero syndromes with a carry trick on the packed word (syndromes are
// below 2^7 for every n handled here, so a byte's bit 7 is free).
template <int SB, bool STORE>
struct SynPacker {
    uint8_t *dst;
    uint32_t w = 0;
    uint32_t cnt = 0;  // per-lane-of-word counters
    Pend4 pend;

    __device__ __forceinline__ explicit SynPacker(uint8_t *d) : dst(d) {}

    __device__ __forceinline__ void put(int c, uint32_t s)
    {
        constexpr int PER = SB == 1 ? 4 : 2;
        const int slot = c % PER;
        if (slot == 0)
            w = s;
        else
            w |= s << (slot * 8 * SB);
        if (slot == PER - 1) {
            if constexpr (SB == 1)
                cnt += ((w + 0x7F7F7F7Fu) >> 7) & 0x01010101u;
            else
                cnt += ((w + 0x7FFF7FFFu) >> 15) & 0x00010001u;
            if constexpr (STORE) {
                const int wi = c / PER;  // word index within the thread's syndromes
                pend.set(wi & 3, w);
                if ((wi & 3) == 3)
                    *reinterpret_cast<uint4 *>(dst + 16 * (wi >> 2)) =
                        make_uint4(pend.p0, pend.p1, pend.p2, pend.p3);
            }
        }
    }

    __device__ __forceinline__ uint32_t nonzero() const
    {
        if constexpr (SB == 1)
            return (cnt * 0x01010101u) >> 24;
        else
            return (cnt & 0xFFFFu) + (cnt >> 16);
    }
};

// Position-domain word w of codeword c of the thread tile held in r[0..n-1].
template <int N_>
__device__ __forceinline__ uint32_t tile_y(const uint32_t (&r)[N_], int c, int w)
{
    const int start = c * N_ - 1 + 32 * w;
    if (start < 0) return r[0] << 1;
    const int a = start >> 5, sh = start & 31;
    if (sh == 0) return r[a];
    const uint32_t hi = (a + 1 < N_) ? r[a + 1] : 0u;
    return __funnelshift_r(r[a], hi, sh);
}

template <int N_>
__device__ __forceinline__ uint32_t tile_syndrome(const uint32_t (&y)[Code<N_>::Wy])
{
    using C = Code<N_>;
    uint32_t s = 0;
    if constexpr (C::Wy == 1) {
#pragma unroll
        for (int i = 0; i < C::m; ++i) s |= (__popc(y[0] & qmask(N_, i)) & 1u) << i;
    } else {
        uint32_t f = 0;
#pragma unroll
        for (int w = 0; w < C::Wy; ++w) f ^= y[w];
#pragma unroll
        for (int i = 0; i < 5; ++i) s |= (__popc(f & bmask(i)) & 1u) << i;
#pragma unroll
        for (int t = 0; (1 << t) < C::Wy; ++t) {
            uint32_t g = 0;
#pragma unroll
            for (int w = 0; w < C::Wy; ++w)
                if ((w >> t) & 1) g ^= y[w];
            s |= (__popc(g) & 1u) << (5 + t);
        }
    }
    return s;
}

// Decode the thread tile r[] (32 codewords), appending the data bits to `op`
// and the syndromes to `sp`.
template <int N_, class OP, class SP>
__device__ __forceinline__ void decode_thread_tile(const uint32_t (&r)[N_], OP &op, SP &sp)
{
    using C = Code<N_>;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        uint32_t y[C::Wy];
#pragma unroll
        for (int w = 0; w < C::Wy; ++w) y[w] = tile_y<N_>(r, c, w);
        const uint32_t s = tile_syndrome<N_>(y);
        if constexpr (C::Wy == 1) {
            y[0] ^= 1u << s;
            uint32_t d = 0;
#pragma unroll
            for (int j = 1; j < C::m; ++j) d |= (y[0] >> (j + 2)) & run_mask(j);
            op.append(d, C::k);
        } else {
#pragma unroll
            for (int w = 0; w < C::Wy; ++w) y[w] ^= shl_clamp(1u, s - 32u * (uint32_t)w);
            uint32_t d0 = 0;
#pragma unroll
            for (int j = 1; j < 5; ++j) d0 |= (y[0] >> (j + 2)) & run_mask(j);
            op.append(d0, 26);
#pragma unroll
            for (int w = 1; w < C::Wy; ++w) {
                if ((w & (w - 1)) == 0)
                    op.append(y[w] >> 1, 31);  // position 32w is a checksum position
                else
                    op.append(y[w], 32);
            }
        }
        sp.put(c, s);
    }
}

}  // namespace hd
