// hd_tile.cuh -- per-thread decode of G consecutive codewords of a
// compile-time length n ("thread part").  A team of H = 32/G threads covers one
// 32-codeword tile: n input words and k output words (n is odd, so 32
// codewords always fill whole words).  Sub-thread h of a team starts at bit
// h*G*n of the tile's input and bit h*G*k of its output; it re-aligns its input
// with one funnel shift per word so that every bit offset inside its part is a
// compile-time constant once the codeword loop is unrolled, and it shifts its
// output back by h*G*k mod 32 on the way out (partial words at the two ends of
// its range are written bytewise; G >= 8 keeps them byte-aligned).
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

// Integer multiply-add.  Multiplying by 2^t shifts left; adding bit fields
// that do not overlap equals OR-ing them, so packing runs on the multiply pipe
// beside the logic operations of the decoder.
__device__ __forceinline__ uint32_t fma_lo(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// Bits of a where K is set, else bits of b: one three-input logic operation
// (truth table 0xCA = K ? a : b for the inputs K = 0xF0, a = 0xCC, b = 0xAA).
__device__ __forceinline__ uint32_t bitsel(uint32_t K, uint32_t a, uint32_t b)
{
    uint32_t r;
    asm("lop3.b32 %0, %1, %2, %3, 0xCA;" : "=r"(r) : "r"(K), "r"(a), "r"(b));
    return r;
}

// Redundancy removal within one position-domain word (bit p = position p):
// the data positions between the powers of two, run j = positions
// 2^j + 1 .. 2^(j+1) - 1 for j = 1 .. M - 1 (M <= 5), move down by j + 2 bits
// to data bits 0 ..  One shift by 3 moves every run; the remaining j - 1 bits
// are taken in binary: runs 2 and 4 move down one more bit, then runs 3 and 4
// two more, each step a select between the word and its shifted copy (the
// runs kept in place and the destinations of the moved runs never overlap).
// With M = 5 the result has no bits above the 26 data bits; for shorter codes
// the bits above the k data bits are whatever followed in the word.
template <int M>
__device__ __forceinline__ uint32_t compress_runs(uint32_t y)
{
    uint32_t d = y >> 3;  // run 1 at bit 0, run 2 at 2..4, run 3 at 6..12, run 4 at 14..28
    if constexpr (M >= 3) d = bitsel(0x00001FC1u, d, d >> 1);  // keep runs 1, 3; runs 2, 4 to 1..3, 13..27
    if constexpr (M >= 4) d = bitsel(0x0000000Fu, d, d >> 2);  // keep runs 1, 2; runs 3, 4 to 4..10, 11..25
    return d;
}

// Syndrome gather for codes whose m checksum bits come from one 32-bit word:
// the parity counts are summed into fields of F bits, the field LSBs kept, and
// one multiply moves LSB j (bit F*j) to bit 32-m+j.  All partial products land
// on distinct bits, so there are no carries into the top m bits.
template <int M>
struct SynGather {
    static constexpr int F = M <= 4 ? 8 : 6;
    static constexpr uint32_t lsbs()
    {
        uint32_t v = 0;
        for (int j = 0; j < M; ++j) v |= 1u << (F * j);
        return v;
    }
    static constexpr uint32_t mult()
    {
        uint32_t v = 0;
        for (int j = 0; j < M; ++j) v |= 1u << (32 - M + j - F * j);
        return v;
    }
    static_assert(32 - M + (M - 1) - F * (M - 1) >= 0, "gather multiplier fits");
};

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

// Store bytes [sb, eb) of v into the word at p (little-endian byte order).
__device__ __forceinline__ void store_bytes(uint32_t *p, uint32_t v, uint32_t sb, uint32_t eb)
{
    if (sb == 0 && eb >= 4) {
        *p = v;
        return;
    }
    uint8_t *b = reinterpret_cast<uint8_t *>(p);
    for (uint32_t i = sb; i < eb && i < 4; ++i) b[i] = (uint8_t)(v >> (8 * i));
}

// Output bit packer.  Appends pieces of `len` clean bits at compile-time
// positions.  GK = total bits of the part.  With ALIGNED the part starts on a
// word boundary (one thread per tile, or G*k a multiple of 32) and completed
// words are stored directly, in vectors of V words; otherwise every word is
// shifted up by the runtime offset `ob` (a multiple of 8) and the first and
// last words of the range are stored bytewise.
template <int GK, bool ALIGNED, int V>
struct OutPacker {
    static constexpr int QL = (GK + 31) / 32;  // local words
    uint32_t *dst;
    uint32_t ob;
    uint32_t acc = 0, prev = 0;
    int pos = 0;  // bits already in acc
    int q = 0;    // index of the local word acc will become
    Pend4 pend;

    __device__ __forceinline__ OutPacker(uint32_t *d, uint32_t off) : dst(d), ob(off) {}

    __device__ __forceinline__ void emit(uint32_t w)
    {
        if constexpr (ALIGNED) {
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
        } else {
            const uint32_t g = __funnelshift_l(prev, w, ob);  // (w << ob) | (prev >> (32 - ob))
            if (q == 0)
                store_bytes(dst, g, ob >> 3, 4);
            else if (q < QL - 1)
                dst[q] = g;
            else
                store_bytes(dst + q, g, 0, (ob + GK - 32 * q) >> 3);
            prev = w;
        }
        ++q;
    }

    // v must have no bits at or above `len`.  The shifts run on the FMA pipe.
    __device__ __forceinline__ void append(uint32_t v, int len)
    {
        if (pos == 0)
            acc = v;
        else
            acc = fma_lo(v, 1u << pos, acc);  // acc | (v << pos)
        if (pos + len >= 32) {
            emit(acc);
            acc = (pos + len > 32) ? v >> (32 - pos) : 0u;
            pos = pos + len - 32;
        } else {
            pos += len;
        }
    }

    // Flush the last partial local word and the spill into the next word.
    __device__ __forceinline__ void finish()
    {
        if (pos > 0) emit(acc);
        if constexpr (!ALIGNED) {
            // bits of the last local word shifted past its end land in word QL
            const int e = (int)ob + GK - 32 * QL;
            if (e > 0) store_bytes(dst + QL, __funnelshift_l(prev, 0u, ob), 0, (uint32_t)e >> 3);
        }
    }
};

// Syndrome packer: 4 (u8) or 2 (u16) syndromes per word; also counts the
// nonzero syndromes with a carry trick on the packed word (syndromes are
// below 2^7 for u8 lanes with n <= 127 and below 2^15 for u16 lanes, so the
// top bit of each lane is free; a popcount of the carried top bits counts the
// nonzero lanes).  For n = 255 with u8 lanes the count uses a compare.
template <int SB, bool STORE, int G, bool WIDE>
struct SynPacker {
    static constexpr int PER = SB == 1 ? 4 : 2;  // syndromes per word
    static constexpr int WORDS = G / PER;        // words of this part
    static constexpr int VEC = WORDS >= 4 ? 4 : WORDS;
    uint8_t *dst;
    uint32_t w = 0;
    uint32_t cnt = 0;
    Pend4 pend;

    __device__ __forceinline__ explicit SynPacker(uint8_t *d) : dst(d) {}

    __device__ __forceinline__ void put(int c, uint32_t s)
    {
        if constexpr (WIDE) cnt += (s != 0u);
        const int slot = c % PER;
        if (slot == 0)
            w = s;
        else
            w = fma_lo(s, 1u << (slot * 8 * SB), w);  // w | (s << lane offset)
        if (slot == PER - 1) {
            if constexpr (!WIDE) {
                // a lane is nonzero iff adding 0x7F..F carries into its top bit
                if constexpr (SB == 1)
                    cnt = fma_lo(__popc(fma_lo(w, 1u, 0x7F7F7F7Fu) & 0x80808080u), 1u, cnt);
                else
                    cnt = fma_lo(__popc(fma_lo(w, 1u, 0x7FFF7FFFu) & 0x80008000u), 1u, cnt);
            }
            if constexpr (STORE) {
                const int wi = c / PER;  // word index within the part
                pend.set(wi % VEC, w);
                if (wi % VEC == VEC - 1) {
                    uint8_t *p = dst + 4 * (wi - (VEC - 1));
                    if constexpr (VEC == 4)
                        *reinterpret_cast<uint4 *>(p) = make_uint4(pend.p0, pend.p1, pend.p2, pend.p3);
                    else if constexpr (VEC == 2)
                        *reinterpret_cast<uint2 *>(p) = make_uint2(pend.p0, pend.p1);
                    else
                        *reinterpret_cast<uint32_t *>(p) = pend.p0;
                }
            }
        }
    }

    __device__ __forceinline__ uint32_t nonzero() const { return cnt; }
};

// Position-domain word w of codeword c of a part held in r[0..R-1].
template <int N_, int R>
__device__ __forceinline__ uint32_t part_y(const uint32_t (&r)[R], int c, int w)
{
    const int start = c * N_ - 1 + 32 * w;
    if (start < 0) return r[0] << 1;
    const int a = start >> 5, sh = start & 31;
    if (sh == 0) return r[a];
    const uint32_t hi = (a + 1 < R) ? r[a + 1] : 0u;
    return __funnelshift_r(r[a], hi, sh);
}

// SECDED (XH): codeword c occupies bits [c*(n+1), (c+1)*(n+1)) of the part and
// position p is its bit p, so its words are the position domain directly
// (position 0 is the overall parity bit); shorter codewords are masked.
template <int N_, int R>
__device__ __forceinline__ uint32_t part_y_xh(const uint32_t (&r)[R], int c, int w)
{
    constexpr int L = N_ + 1;
    const int start = c * L + 32 * w;
    const int a = start >> 5, sh = start & 31;
    uint32_t v;
    if (sh == 0) {
        v = r[a];
    } else {
        const uint32_t hi = (a + 1 < R) ? r[a + 1] : 0u;
        v = __funnelshift_r(r[a], hi, sh);
    }
    if constexpr (L < 32) v &= (1u << L) - 1u;
    return v;
}

template <int N_>
__device__ __forceinline__ uint32_t part_syndrome(const uint32_t (&y)[Code<N_>::Wy])
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
        // low five bits (and for two words the sixth, the parity of word 1),
        // gathered from parity-count fields as in the one-word case
        constexpr int MG = C::Wy == 2 ? 6 : 5;
        using SG = SynGather<MG>;
        uint32_t pf = __popc(f & bmask(0));
#pragma unroll
        for (int i = 1; i < 5; ++i) pf = fma_lo(__popc(f & bmask(i)), 1u << (SG::F * i), pf);
        if constexpr (MG == 6) pf = fma_lo(__popc(y[1]), 1u << (SG::F * 5), pf);
        s = ((pf & SG::lsbs()) * SG::mult()) >> (32 - MG);
#pragma unroll
        for (int t = MG - 5; (1 << t) < C::Wy; ++t) {
            uint32_t g = 0;
#pragma unroll
            for (int w = 0; w < C::Wy; ++w)
                if ((w >> t) & 1) g ^= y[w];
            s |= (__popc(g) & 1u) << (5 + t);
        }
    }
    return s;
}

// Decode the G codewords of a part held in r[] (bit 0 of r[0] is position 1
// of its first codeword, or position 0 with XH), appending data bits to `op`
// and syndromes to `sp`.  XH (SECDED): the overall parity P of the n + 1 bits
// decides the correction (P = 1: flip position s; P = 0: flip nothing, and
// s != 0 is a detected double error, counted in `det`); the syndrome value is
// s | P << m.
template <int N_, int G, int R, bool XH = false, bool LUT = false, class OP, class SP>
__device__ __forceinline__ void decode_part(const uint32_t (&r)[R], OP &op, SP &sp, uint32_t &det,
                                            const uint16_t *lut = nullptr)
{
    using C = Code<N_>;
    if constexpr (LUT) {
        // one lookup per codeword: its n bits index data | s << k (SECDED: its
        // n + 1 bits index data | s << k | P << (k + m)).  All G lookups are
        // issued before any result is packed, so their shared-memory latencies
        // overlap.
        static_assert(N_ <= 15, "decode tables exist for n = 7 and 15");
        constexpr int L = N_ + (XH ? 1 : 0);
        uint32_t e[G];
#pragma unroll
        for (int c = 0; c < G; ++c) {
            const int start = c * L;  // a constant once the loop is unrolled
            const int a = start >> 5, sh = start & 31;
            uint32_t v;
            if (sh == 0)
                v = r[a];
            else if (a + 1 < R)
                v = __funnelshift_r(r[a], r[a + 1], sh);
            else
                v = r[a] >> sh;
            e[c] = lut[v & ((1u << L) - 1u)];
        }
#pragma unroll
        for (int c = 0; c < G; ++c) {
            op.append(e[c] & ((1u << C::k) - 1u), C::k);
            const uint32_t sv = e[c] >> C::k;  // s, or for SECDED s | P << m
            if constexpr (XH) det += (sv - 1u < (1u << C::m) - 1u) ? 1u : 0u;  // P = 0 and s != 0
            sp.put(c, sv);
        }
    } else {
#pragma unroll
        for (int c = 0; c < G; ++c) {
            uint32_t y[C::Wy];
#pragma unroll
            for (int w = 0; w < C::Wy; ++w) y[w] = XH ? part_y_xh<N_, R>(r, c, w) : part_y<N_, R>(r, c, w);
            if constexpr (C::Wy == 1) {
                // checksum: parities of y & I_i, summed into fields, gathered into
                // the top m bits of st
                using SG = SynGather<C::m>;
                uint32_t pf = __popc(y[0] & qmask(N_, 0));
#pragma unroll
                for (int i = 1; i < C::m; ++i) pf = fma_lo(__popc(y[0] & qmask(N_, i)), 1u << (SG::F * i), pf);
                const uint32_t st = (pf & SG::lsbs()) * SG::mult();
                const uint32_t s = st >> (32 - C::m);
                // correction: flip position s (s = 0 flips bit 0, which is no data position)
                if constexpr (XH) {
                    const uint32_t P = __popc(y[0]) & 1u;
                    y[0] ^= P << s;
                    det += (P == 0u && s != 0u) ? 1u : 0u;
                    sp.put(c, s | (P << C::m));
                } else {
                    y[0] ^= 1u << s;
                }
                // redundancy removal
                uint32_t d = compress_runs<C::m>(y[0]);
                if constexpr (C::m < 5) d &= (1u << C::k) - 1u;  // the word also holds the next codeword
                op.append(d, C::k);
                if constexpr (!XH) sp.put(c, s);
            } else {
                const uint32_t s = part_syndrome<N_>(y);
                uint32_t sf = s;  // the position to flip; past every word when nothing is flipped
                if constexpr (XH) {
                    uint32_t f = 0;
#pragma unroll
                    for (int w = 0; w < C::Wy; ++w) f ^= y[w];
                    const uint32_t P = __popc(f) & 1u;
                    sf = P ? s : 0xFFFFFFFFu;
                    det += (P == 0u && s != 0u) ? 1u : 0u;
                    sp.put(c, s | (P << C::m));
                }
#pragma unroll
                for (int w = 0; w < C::Wy; ++w) y[w] ^= shl_clamp(1u, sf - 32u * (uint32_t)w);
                op.append(compress_runs<5>(y[0]), 26);
#pragma unroll
                for (int w = 1; w < C::Wy; ++w) {
                    if ((w & (w - 1)) == 0)
                        op.append(y[w] >> 1, 31);  // position 32w is a checksum position
                    else
                        op.append(y[w], 32);
                }
                if constexpr (!XH) sp.put(c, s);
            }
        }
    }
    op.finish();
}

}  // namespace hd
