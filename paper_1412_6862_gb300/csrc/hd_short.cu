// hd_short.cu -- shortened Hamming codes: segments of any length n.
//
// The paper's decoder splits a packet of M bytes into t segments (Sec. II,
// Fig. 1; the evaluation of Sec. IV-A sweeps M = 400..2000 bytes and
// t = 2..6), and each segment carries its own checksum bits, so a segment is
// a codeword of a shortened code: n = k + r bits, r the smallest count with
// 2^r >= n + 1, checksum bits at the power-of-two positions 1..2^(r-1), data at
// the other positions.  A syndrome s <= n names the position to flip; a
// syndrome past n names none, and the codeword is counted as detected and
// left as received.
//
// Two decoders:
//  * k_short_tiles (k >= 64, i.e. n >= 71): each warp streams tiles of g whole
//    codewords through a ring of shared-memory stages filled by 1-D bulk
//    copies.  Per tile: (1) syndromes, teams of T lanes per codeword (T from a
//    cost model, 1..32), each lane folding its position-domain words into an
//    XOR and a parity mask, then a butterfly over the team; the corrections
//    flip bits in the stage.  (3) Every output word from a per-length table of
//    output-word offsets: a funnel shift (and, for short codewords, a merge at
//    the word's checksum position), lane-strided so stage reads are
//    conflict-free and stores coalesced.  (4) The words that hold a codeword's
//    first 26 data bits or cross into the next codeword, per codeword.  (5) For
//    long codewords, the few words that hold a checksum position.
//  * k_short_small (n <= 255): warp tiles of 32 codewords straight from global
//    memory, one codeword per lane, like the generic full-length kernel.
// The encoder (k_encode_short) is bit-serial, one thread per codeword: it is
// used to build inputs, not timed.
#include <algorithm>
#include <cstdint>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "hd_device.cuh"
#include "hd_generic.cuh"
#include "hd_internal.h"

namespace hd {
namespace {

constexpr uint32_t kShortMaxN = 32767;  // r <= 15: syndromes fit 16 bits
constexpr uint32_t kLongMinK = 64;      // k_short_tiles needs the first 58 data bits inside one codeword

__host__ __device__ inline uint32_t short_r(uint32_t n)
{
    uint32_t r = 0;
    while ((1u << r) < n + 1u) ++r;
    return r;
}

__device__ __forceinline__ uint32_t lowmask(uint32_t b) { return b >= 32 ? 0xFFFFFFFFu : (1u << b) - 1u; }

// Low five syndrome bits from the XOR of a codeword's position-domain words:
// bit i is the parity of the bits whose in-word index has bit i set.
__device__ __forceinline__ uint32_t fold5(uint32_t f)
{
    return (__popc(f & 0xAAAAAAAAu) & 1u) | ((__popc(f & 0xCCCCCCCCu) & 1u) << 1) |
           ((__popc(f & 0xF0F0F0F0u) & 1u) << 2) | ((__popc(f & 0xFF00FF00u) & 1u) << 3) |
           ((__popc(f & 0xFFFF0000u) & 1u) << 4);
}

struct ShortArgs {
    const uint32_t *in;
    uint32_t *out;
    void *syn;
    unsigned long long *err;
    unsigned long long *det;
    uint32_t *status;
    uint64_t num_cw;
    uint64_t in_words;
    uint64_t bulk_end;  // bytes of the input that 16-byte bulk copies may read
    uint64_t ntiles;
    uint32_t n, k, g;   // code length, data bits, codewords per tile
    uint32_t Y;         // position-domain words per codeword: ceil((n + 1) / 32)
    uint32_t ylast;     // valid-bit mask of the last position-domain word
    uint32_t tlog;      // log2 of the team size of the syndrome pass
    int syn_type;
    const void *table;      // output-word offsets (see output_table), tab_len entries of 2 or 4 bytes
    uint32_t tab_len;
    uint32_t nJ;            // data runs J >= 5 that end inside the codeword's data (D_J < k)
    uint32_t nJ_magic;      // ceil(2^32 / nJ) for nJ > 1: f / nJ = umulhi(f, nJ_magic) for the small f used
};

template <int SB>
struct TileGeom {
    // stage: 16-byte guard word area (read as word -1), SB data bytes, 16 bytes of slack
    static constexpr uint32_t stage_stride = SB + 32;
    static constexpr uint32_t max_g = 256;
};

// Codewords per tile: the tile's input plus 16-byte rounding at both ends fits SB bytes.
template <int SB>
inline uint32_t tile_codewords(uint32_t n)
{
    const uint32_t g = (uint32_t)((8u * SB - 256u) / n);
    return std::min<uint32_t>(g, TileGeom<SB>::max_g);
}

// Bytes of tile t that a bulk copy brings in, and where they start.
__device__ __forceinline__ void tile_span(const ShortArgs &a, uint64_t t, uint64_t &byte0, uint32_t &bytes,
                                          uint32_t &gcnt)
{
    const uint64_t c0 = t * a.g;
    gcnt = (uint32_t)min((uint64_t)a.g, a.num_cw - c0);
    const uint64_t bit0 = c0 * a.n, bit1 = (c0 + gcnt) * a.n;
    byte0 = (bit0 >> 7) << 4;
    uint64_t byte1 = ((bit1 + 127) >> 7) << 4;
    if (byte1 > a.bulk_end) byte1 = a.bulk_end;
    bytes = byte1 > byte0 ? (uint32_t)(byte1 - byte0) : 0u;
}

template <int SB>
__device__ __forceinline__ void issue_tile(const ShortArgs &a, uint64_t t, uint8_t *stage, uint64_t *bar)
{
    uint64_t byte0;
    uint32_t bytes, gcnt;
    tile_span(a, t, byte0, bytes, gcnt);
    mbar_arrive_expect_tx(bar, bytes);
    if (bytes) bulk_g2s(stage + 16, reinterpret_cast<const uint8_t *>(a.in) + byte0, bytes, bar);
}

// The first 32 data bits of the codeword whose position 1 is stage bit cb
// (positions 3, 5-7, 9-15, 17-31, 33-38).
__device__ __forceinline__ uint32_t head_word(const uint32_t *st, uint32_t cb)
{
    const int32_t q = (int32_t)cb - 1;
    const int32_t wi = q >> 5;  // -1 reads the guard word
    const uint32_t sh = (uint32_t)q & 31u;
    const uint32_t y0 = __funnelshift_r(st[wi], st[wi + 1], sh);
    const uint32_t y1 = __funnelshift_r(st[wi + 1], st[wi + 2], sh);
    return ((y0 >> 3) & 1u) | ((y0 >> 4) & 0xEu) | ((y0 >> 5) & 0x7F0u) | ((y0 >> 6) & 0x3FFF800u) |
           ((y1 << 25) & 0xFC000000u);
}

// 32 data bits of the codeword whose position 1 is stage bit cb, from data bit
// d >= 26 on (so at most one checksum position falls inside).
__device__ __forceinline__ uint32_t run_word(const uint32_t *st, uint32_t cb, uint32_t d)
{
    const uint32_t J1 = 31u - __clz(d);
    const uint32_t J = J1 + ((d + J1 + 2u) >> (J1 + 1u));  // data run of bit d
    const uint32_t q = cb + d + J + 1u;
    const uint32_t lo = st[q >> 5], hi = st[(q >> 5) + 1], sh = q & 31u;
    const uint32_t m = lowmask((2u << J) - J - 2u - d);
    return (__funnelshift_r(lo, hi, sh) & m) | (__funnelshift_rc(lo, hi, sh + 1u) & ~m);
}

template <int W, int S, int SB, bool TAB_SMEM, bool SPLIT>
__global__ void __launch_bounds__(W * 32) k_short_tiles(ShortArgs a)
{
    using Geom = TileGeom<SB>;
    extern __shared__ __align__(128) uint8_t smem[];
    constexpr uint32_t warp_bytes = S * Geom::stage_stride + 16 * S;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the output-word table, copied once per CTA when it fits next to the stages
    // SPLIT: 32-bit entries that also say where a word's checksum position falls, resolved
    // in pass 3; otherwise 16-bit entries and pass 5 rewrites those words
    using Entry = typename std::conditional<SPLIT, uint32_t, uint16_t>::type;
    const Entry *tab = static_cast<const Entry *>(a.table);
    if constexpr (TAB_SMEM) {
        Entry *s_tab = reinterpret_cast<Entry *>(smem + W * warp_bytes);
        for (uint32_t i = threadIdx.x; i < a.tab_len; i += W * 32) s_tab[i] = tab[i];
        __syncthreads();
        tab = s_tab;
    }
    uint8_t *wbase = smem + warp * warp_bytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(wbase + S * Geom::stage_stride);
    const uint64_t gw = (uint64_t)blockIdx.x * W + warp, tw = (uint64_t)gridDim.x * W;

    if (lane == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
        for (int s = 0; s < S; ++s) {
            const uint64_t t = gw + (uint64_t)s * tw;
            if (t < a.ntiles) issue_tile<SB>(a, t, wbase + s * Geom::stage_stride, &bar[s]);
        }
    }
    __syncwarp();

    // syndrome teams: T lanes per codeword, G codewords per round
    const uint32_t tlog = a.tlog, T = 1u << tlog, tl = lane & (T - 1u), team = lane >> tlog, G = 32u >> tlog;
    const uint32_t n = a.n, k = a.k, Ym1 = a.Y - 1u;
    const uint32_t tl_last = Ym1 & (T - 1u);
    const bool wide = ((a.Y + T - 1u) >> tlog) > 32u;  // a lane reads more than 32 words of a codeword
    const int32_t stage_bits = 8 * SB;  // reads past the data stay inside the stage's slack
    uint32_t errs = 0, dets = 0, it = 0;
    bool aborted = false;
    for (uint64_t t = gw; t < a.ntiles; t += tw, ++it) {
        const int s = (int)(it % S);
        const bool ok = mbar_wait_bounded(&bar[s], (it / S) & 1u);
        if (__any_sync(0xFFFFFFFFu, !ok)) {
            aborted = true;
            break;
        }
        uint8_t *stage = wbase + s * Geom::stage_stride;
        uint32_t *st = reinterpret_cast<uint32_t *>(stage + 16);
        uint64_t byte0;
        uint32_t bytes, gcnt;
        tile_span(a, t, byte0, bytes, gcnt);
        const uint64_t c0 = t * a.g;
        const uint32_t off0 = (uint32_t)((c0 * n) & 127u);
        {  // words past the last 16-byte boundary of the input arrive by plain loads
            const uint64_t w0 = byte0 >> 2, wb = (byte0 + bytes) >> 2;
            const uint64_t we = min(((c0 + gcnt) * n + 31) >> 5, a.in_words);
            if (wb < we) {
                for (uint64_t w = wb + lane; w < we; w += 32) st[w - w0] = a.in[w];
                __syncwarp();
            }
        }

        // 1. syndromes.  Lane tl of a team reads position-domain words j = tl + T*i (at most
        //    64); the low syndrome bits come from the XOR of all words, the high bits from the
        //    XOR of the indices j of the odd-parity words: bit i of pm0 (i < 32) or of pm1
        //    (i - 32) is the parity of word tl + T*i.
        for (uint32_t cbase = 0; cbase < gcnt; cbase += G) {
            const uint32_t c = cbase + team;
            uint32_t x = 0, pm0 = 0, pm1 = 0;
            if (c < gcnt) {
                const int32_t q0 = (int32_t)(off0 + c * n) - 1 + 32 * (int32_t)tl;  // position 0 is bit -1 of c
                const uint32_t sh = (uint32_t)q0 & 31u;
                int32_t wi = q0 >> 5;  // -1 reads the guard word
                uint32_t cnt = tl < Ym1 ? ((Ym1 - 1u - tl) >> tlog) + 1u : 0u;  // words before the last one
                const uint32_t n0 = min(cnt, 32u), n1 = cnt - n0;
                // a word's parity bit is shifted in (bit order reversed below)
                auto take = [&](uint32_t y, uint32_t &pm) {
                    x ^= y;
                    pm = (pm << 1) | (__popc(y) & 1u);
                };
                uint32_t lo = 0;  // only words of this codeword are read
                // plain shared-memory loads, so that the compiler issues the unrolled
                // iterations' loads ahead of their uses
                const uint32_t *ad = st + wi;
                if (T == 1) {  // one lane per codeword: each word is the next one's low half
                    lo = ad[0];
#pragma unroll 4
                    for (uint32_t i = 0; i < n0; ++i, ++ad) {
                        const uint32_t hi = ad[1];
                        take(__funnelshift_r(lo, hi, sh), pm0);
                        lo = hi;
                    }
#pragma unroll 4
                    for (uint32_t i = 0; i < n1; ++i, ++ad) {
                        const uint32_t hi = ad[1];
                        take(__funnelshift_r(lo, hi, sh), pm1);
                        lo = hi;
                    }
                } else {
#pragma unroll 4
                    for (uint32_t i = 0; i < n0; ++i, ad += T) take(__funnelshift_r(ad[0], ad[1], sh), pm0);
#pragma unroll 4
                    for (uint32_t i = 0; i < n1; ++i, ad += T) take(__funnelshift_r(ad[0], ad[1], sh), pm1);
                    if (tl == tl_last) lo = ad[0];
                }
                if (tl == tl_last) {  // the last word holds positions up to n only
                    const uint32_t y = __funnelshift_r(lo, ad[1], sh) & a.ylast;
                    if (cnt < 32u)
                        take(y, pm0);
                    else
                        take(y, pm1);
                    ++cnt;
                }
                const uint32_t m0 = min(cnt, 32u), m1 = cnt - m0;
                pm0 = m0 ? __brev(pm0) >> (32u - m0) : 0u;
                if (wide) pm1 = m1 ? __brev(pm1) >> (32u - m1) : 0u;
            }
            // indices i of the odd-parity words (those of pm1 are 32 + their bit index;
            // pm1 is used only when a lane reads more than 32 words)
            uint32_t fi = fold5(pm0), par = __popc(pm0);
            if (wide) {
                const uint32_t par1 = __popc(pm1) & 1u;
                fi ^= fold5(pm1) ^ (par1 << 5);
                par ^= par1;
            }
            uint32_t h = ((par & 1u) ? tl : 0u) ^ (fi << tlog);
            // XOR over the team: butterfly steps stay inside aligned groups of T lanes
            for (uint32_t o = T >> 1; o > 0; o >>= 1) {
                x ^= __shfl_xor_sync(0xFFFFFFFFu, x, o);
                h ^= __shfl_xor_sync(0xFFFFFFFFu, h, o);
            }
            if (tl == 0 && c < gcnt) {
                const uint32_t syn = (h << 5) | fold5(x);
                if (syn != 0) {
                    ++errs;
                    if (syn <= n) {
                        const uint32_t b = off0 + c * n + syn - 1u;
                        atomicXor(&st[b >> 5], 1u << (b & 31u));
                    } else {
                        ++dets;
                    }
                }
                if (a.syn_type == 1) static_cast<uint8_t *>(a.syn)[c0 + c] = (uint8_t)syn;
                if (a.syn_type == 2) static_cast<uint16_t *>(a.syn)[c0 + c] = (uint16_t)syn;
            }
        }
        __syncwarp();

        // 3. output words, lane-strided (conflict-free stage reads, coalesced stores).  The table
        //    describes output word idx of a 32-codeword period (k words): the distance from bit
        //    32*idx to the stage bit of the word's first data bit (counted from position 1 of the
        //    period's first codeword) and how many data bits precede its one checksum position.
        //    Words holding a codeword's head or a crossing are rewritten by pass 4.
        const uint64_t ob0 = c0 * k, ob1 = (c0 + gcnt) * k;
        const uint64_t F = ob0 >> 5, L = (ob1 - 1) >> 5;
        const bool fs = (ob0 & 31u) != 0, last_tile = (c0 + gcnt) == a.num_cw;
        const bool ls = (ob1 & 31u) != 0 && !last_tile;
        const int32_t nW = (int32_t)(L - F) + 1;                       // words of this tile
        const int32_t wlo = fs ? 1 : 0, whi = nW - 1 - (ls ? 1 : 0);  // words it writes whole
        {
            // the table runs past one period, so a tile's words never wrap: word w of the tile is
            // entry idxF + w, whose first data bit is at stage bit sb0 + 32 * (idxF + w) + delta
            const uint32_t cr = (uint32_t)(c0 & 31u);
            const int32_t idx0 = (int32_t)((cr * k) >> 5) + lane;
            int32_t sbw = (int32_t)off0 - (int32_t)(cr * n) + 32 * idx0;
            const Entry *tp = tab + idx0;
            uint32_t *outp = a.out + F + lane;
            // four words per lane per iteration, 32 apart.  Words past the tile come from
            // in-range entries and clamped stage bits and are never stored.
            for (int32_t w0 = lane; w0 <= whi; w0 += 128, outp += 128, tp += 128, sbw += 4096) {
                uint32_t e[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) e[u] = tp[32 * u];
                if (w0 - lane >= wlo && w0 - lane + 127 <= whi) {
                    // all 128 words of this step are the tile's own (warp-uniform): their first
                    // data bits lie inside the stage, so neither the clamp nor the store test
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int32_t q = sbw + 1024 * u + (int32_t)(e[u] & 0xFFFFu);
                        const uint32_t lo = st[q >> 5], hi = st[(q >> 5) + 1], sh = (uint32_t)q & 31u;
                        uint32_t v = __funnelshift_r(lo, hi, sh);
                        if constexpr (SPLIT) {
                            const uint32_t m = shl_clamp(1u, e[u] >> 16) - 1u;
                            v = (v & m) | (__funnelshift_rc(lo, hi, sh + 1u) & ~m);
                        }
                        outp[32 * u] = v;
                    }
                    continue;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int32_t q = max(0, min(sbw + 1024 * u + (int32_t)(e[u] & 0xFFFFu), stage_bits));
                    const uint32_t lo = st[q >> 5], hi = st[(q >> 5) + 1], sh = (uint32_t)q & 31u;
                    uint32_t v = __funnelshift_r(lo, hi, sh);
                    if constexpr (SPLIT) {
                        const uint32_t m = shl_clamp(1u, e[u] >> 16) - 1u;
                        v = (v & m) | (__funnelshift_rc(lo, hi, sh + 1u) & ~m);
                    }
                    const int32_t w = w0 + 32 * u;
                    if (w >= wlo && w <= whi) outp[32 * u] = v;
                }
            }
        }
        __syncwarp();  // orders pass 3's stores before pass 4 rewrites some of the same words

        // 4. per codeword: the word where its data starts (crossing from the previous codeword,
        //    or the tile's first word), the next word if it still holds head bits, and for the
        //    last codeword the tile's last word.  Word indices are tile-relative.
        for (uint32_t c = lane; c < gcnt; c += 32) {
            const uint32_t b = (uint32_t)(ob0 & 31u) + c * k;  // tile bit of the codeword's data bit 0
            const int32_t ws = (int32_t)(b >> 5);
            const uint32_t al = b & 31u;
            const uint32_t cb = off0 + c * n;  // stage bit of position 1
            const uint32_t head = head_word(st, cb);
            uint32_t *o = a.out + F + ws;
            if (c == 0 && fs) {
                const uint32_t own = ~lowmask(al), v = head << al;
                atomicAnd(o, v | ~own);
                atomicOr(o, v & own);
            } else if (ws <= whi) {
                *o = al == 0 ? head : (run_word(st, cb - n, k - al) & lowmask(al)) | (head << al);
            }
            if (al > 6 && ws + 1 <= whi) {
                // data bits 32 - al .. 63 - al: the head word's top bits, then data bits 32.. (positions
                // 39..63 of run 5, then run 6 after position 64)
                const uint32_t q = cb + 38u;
                const uint32_t lo = st[q >> 5], hi = st[(q >> 5) + 1], sh = q & 31u;
                const uint32_t x2 = (__funnelshift_r(lo, hi, sh) & 0x1FFFFFFu) |
                                    (__funnelshift_rc(lo, hi, sh + 1u) & ~0x1FFFFFFu);
                o[1] = (head >> (32u - al)) | (x2 << al);
            }
            if (c == gcnt - 1 && (ob1 & 31u) != 0) {
                const uint32_t rem = (uint32_t)(ob1 & 31u);
                const uint32_t v = run_word(st, cb, k - rem) & lowmask(rem);
                uint32_t *ol = a.out + L;
                if (ls) {
                    atomicAnd(ol, v | ~lowmask(rem));
                    atomicOr(ol, v);
                } else {
                    *ol = v;
                }
            }
        }
        // 5. words with a checksum position inside (data run J ends at data bit D_J = 2^(J+1) - J - 2,
        //    J >= 5): pass 3 read them with one shift; lanes take (codeword, J) pairs
        for (uint32_t f = lane; !SPLIT && f < gcnt * a.nJ; f += 32) {
            const uint32_t c = a.nJ == 1 ? f : __umulhi(f, a.nJ_magic), J = 5u + (f - c * a.nJ);
            const uint32_t b0 = (uint32_t)(ob0 & 31u) + c * k;   // tile bit of the codeword's data bit 0
            const uint32_t bd = b0 + (2u << J) - J - 2u;          // tile bit of data bit D_J
            const uint32_t dw = (bd & ~31u) - b0;                 // data bit at the start of its word (>= 26)
            if ((bd & 31u) != 0 && dw + 32u <= k) a.out[F + (bd >> 5)] = run_word(st, off0 + c * n, dw);
        }
        // the corrections wrote the stage through the generic proxy; the refill writes it through the async one
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
            const uint64_t tn = t + (uint64_t)S * tw;
            if (tn < a.ntiles) issue_tile<SB>(a, tn, stage, &bar[s]);
        }
        __syncwarp();
    }
    if (lane == 0 && aborted) {
        atomicOr(a.status, (uint32_t)HD_ERR_TIMEOUT);
        for (uint32_t j = it; j < it + S; ++j) {
            const uint64_t tj = gw + (uint64_t)j * tw;
            if (tj < a.ntiles) (void)mbar_wait_bounded(&bar[j % S], (j / S) & 1u);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        errs += __shfl_xor_sync(0xFFFFFFFFu, errs, o);
        dets += __shfl_xor_sync(0xFFFFFFFFu, dets, o);
    }
    if (lane == 0) {
        grid_dep_wait();  // the counters' clear ahead of a programmatic dependent launch
        if (a.err && errs) atomicAdd(a.err, (unsigned long long)errs);
        if (a.det && dets) atomicAdd(a.det, (unsigned long long)dets);
    }
}

// ---------------------------------------------------------------------------
// Short segments (n <= 255): warp tiles of 32 codewords, one per lane.
// 32 codewords of any length n fill exactly n input words and k output words.
// ---------------------------------------------------------------------------
constexpr int kSmallWarps = 8;

__global__ void __launch_bounds__(kSmallWarps * 32)
    k_short_small(const uint32_t *__restrict__ in, uint64_t in_words, uint32_t n, uint32_t r, uint64_t num_cw,
                  uint32_t *__restrict__ out, uint64_t out_words, void *__restrict__ syn, int syn_type,
                  unsigned long long *__restrict__ err, unsigned long long *__restrict__ det)
{
    __shared__ uint32_t sy[kSmallWarps][kWarpSlotWords];
    __shared__ uint32_t sd[kSmallWarps][kWarpSlotWords];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    uint32_t *my_y = &sy[wp][lane * kSlot];
    uint32_t *my_d = &sd[wp][lane * kSlot];
    const uint32_t k = n - r;
    const uint32_t wy = (n + 32) >> 5;  // ceil((n + 1) / 32)
    const uint32_t ylast = lowmask(n + 1 - 32 * (wy - 1));
    const uint64_t tiles = (num_cw + 31) / 32;
    uint32_t errs = 0, dets = 0;
    for (uint64_t t = (uint64_t)blockIdx.x * kSmallWarps + wp; t < tiles; t += (uint64_t)gridDim.x * kSmallWarps) {
        const uint64_t i = t * 32 + lane;
        const bool valid = i < num_cw;
        uint32_t y[8];
#pragma unroll
        for (uint32_t w = 0; w < 8; ++w)
            y[w] = (valid && w < wy) ? load_window(in, in_words, (int64_t)(i * n) - 1 + 32 * (int64_t)w) : 0u;
        y[0] &= ~1u;
#pragma unroll
        for (uint32_t w = 0; w < 8; ++w)
            if (w == wy - 1) y[w] &= ylast;
        const uint32_t s = syndrome_y(y, wy);
        const uint32_t fix = s <= n ? s : 0u;  // a syndrome past n names no position
#pragma unroll
        for (uint32_t w = 0; w < 8; ++w)
            if (w < wy) y[w] ^= shl_clamp(fix != 0 ? 1u : 0u, fix - 32u * w);
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            my_y[w] = y[w];
            my_d[w] = 0;
        }
        my_y[8] = 0;
        my_d[8] = 0;
        // data run j: positions 2^j + 1 .. min(2^(j+1) - 1, n)
        for (uint32_t j = 1; j < r; ++j) {
            const uint32_t first = (1u << j) + 1u, last = min((2u << j) - 1u, n);
            if (last >= first) copy_bits(my_y, first, my_d, (1u << j) - j - 1u, last - first + 1u);
        }
        __syncwarp();
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
            if (syn_type == 1) static_cast<uint8_t *>(syn)[i] = (uint8_t)s;
            if (syn_type == 2) static_cast<uint16_t *>(syn)[i] = (uint16_t)s;
        }
        errs += __popc(__ballot_sync(0xFFFFFFFFu, valid && s != 0));
        dets += __popc(__ballot_sync(0xFFFFFFFFu, valid && s > n));
        __syncwarp();
    }
    if (lane == 0) {
        grid_dep_wait();  // the counters' clear ahead of a programmatic dependent launch
        if (err && errs) atomicAdd(err, (unsigned long long)errs);
        if (det && dets) atomicAdd(det, (unsigned long long)dets);
    }
}

// ---------------------------------------------------------------------------
// Encoder: one thread per codeword, bit-serial.  The stream must be zero.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool is_pow2(uint32_t p) { return (p & (p - 1u)) == 0; }

__global__ void k_encode_short(const uint32_t *__restrict__ data, uint64_t data_words, uint32_t n, uint32_t r,
                               uint64_t num_cw, uint32_t *__restrict__ stream)
{
    const uint32_t k = n - r;
    for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < num_cw;
         c += (uint64_t)gridDim.x * blockDim.x) {
        // checksum vector of the message placed at the data positions
        uint32_t s = 0, d = 0, win = 0;
        for (uint32_t p = 3; p <= n; ++p) {
            if (is_pow2(p)) continue;
            if ((d & 31u) == 0) win = load_window(data, data_words, (int64_t)(c * k + d));
            if ((win >> (d & 31u)) & 1u) s ^= p;
            ++d;
        }
        // write positions 1..n: checksum bit j at position 2^j makes the syndrome 0
        const uint64_t b0 = c * n, b1 = b0 + n;
        uint32_t acc = 0;
        d = 0;
        for (uint32_t p = 1; p <= n; ++p) {
            uint32_t bit;
            if (is_pow2(p)) {
                bit = (s >> (31u - __clz(p))) & 1u;
            } else {
                if ((d & 31u) == 0) win = load_window(data, data_words, (int64_t)(c * k + d));
                bit = (win >> (d & 31u)) & 1u;
                ++d;
            }
            const uint64_t b = b0 + p - 1;
            acc |= bit << (b & 31u);
            if ((b & 31u) == 31u || p == n) {
                const uint64_t w = b >> 5;
                if ((w << 5) >= b0 && (w << 5) + 32 <= b1)
                    stream[w] = acc;
                else if (acc)
                    atomicOr(&stream[w], acc);
                acc = 0;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Variant table of the tile kernel (compiled configurations).
// ---------------------------------------------------------------------------
struct ShortVariant {
    int W, S, SB;
    uint32_t stage_smem;  // dynamic shared memory of the warps' stages
    // [0]: table in global memory; [1]: table in shared memory; [2]: shared, splits in pass 3
    const void *kernel[3];
    cudaError_t (*launch[3])(const ShortArgs &, int grid, uint32_t smem, cudaStream_t, bool pdl);
};

template <int W, int S, int SB, bool TAB_SMEM, bool SPLIT>
cudaError_t launch_tiles(const ShortArgs &a, int grid, uint32_t smem, cudaStream_t st, bool pdl)
{
    return launch_kernel(k_short_tiles<W, S, SB, TAB_SMEM, SPLIT>, dim3((unsigned)grid), dim3(W * 32), smem, st, pdl,
                         a);
}

template <int W, int S, int SB>
ShortVariant make_short_variant()
{
    constexpr uint32_t warp_bytes = S * TileGeom<SB>::stage_stride + 16 * S;
    return ShortVariant{W,
                        S,
                        SB,
                        W * warp_bytes,
                        {reinterpret_cast<const void *>(k_short_tiles<W, S, SB, false, false>),
                         reinterpret_cast<const void *>(k_short_tiles<W, S, SB, true, false>),
                         reinterpret_cast<const void *>(k_short_tiles<W, S, SB, true, true>)},
                        {&launch_tiles<W, S, SB, false, false>, &launch_tiles<W, S, SB, true, false>,
                         &launch_tiles<W, S, SB, true, true>}};
}

const ShortVariant kShortVariants[] = {
    // the built-in choice: fastest over the paper's (M, t) grid on GB300 (the
    // kernel waits on fixed-latency chains, so warps per SM count: two of these
    // CTAs hold 24 warps, two 8-warp CTAs of 4 KB stages only 16)
    make_short_variant<12, 2, 4096>(),
    make_short_variant<8, 2, 4096>(),
    make_short_variant<4, 2, 8192>(),
    make_short_variant<4, 3, 4096>(),
    make_short_variant<4, 4, 2048>(),
    make_short_variant<16, 2, 2048>(),
    make_short_variant<16, 2, 3072>(),
};
constexpr int kNumShortVariants = sizeof(kShortVariants) / sizeof(kShortVariants[0]);

// The configuration with the largest stages (the first of them), which holds a
// codeword of every supported length.
int largest_stage_variant()
{
    int best = 0;
    for (int v = 1; v < kNumShortVariants; ++v)
        if (kShortVariants[v].SB > kShortVariants[best].SB) best = v;
    return best;
}
constexpr uint32_t kTabSmemMax = 40u << 10;  // larger tables stay in global memory

std::mutex g_short_mu;
int g_short_choice[64] = {};  // variant pinned for every length on a device (index + 1; 0 = none)
struct TunedEntry {
    uint32_t n = 0;
    int v = -1;
};
TunedEntry g_short_tuned[64][64];  // per device: the autotuner's choice per length

struct OccEntry {
    int v = -1, tsm = 0;
    uint32_t smem = 0;
    int bps = 0;
};
OccEntry g_occ[64][32];

// Resident CTAs per SM of configuration v with `smem` bytes of dynamic shared memory.
int short_blocks_per_sm(int v, int tsm, uint32_t smem)
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    std::lock_guard<std::mutex> lk(g_short_mu);
    for (const OccEntry &e : g_occ[dev])
        if (e.v == v && e.tsm == tsm && e.smem == smem) return e.bps;
    const ShortVariant &sv = kShortVariants[v];
    // the attribute is per kernel: allow the device's largest opt-in size once, never a smaller one
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        (uint32_t)optin < smem ||
        cudaFuncSetAttribute(sv.kernel[tsm], cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess)
        return -1;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, sv.kernel[tsm], sv.W * 32, smem) != cudaSuccess ||
        bps <= 0)
        return -1;
    for (OccEntry &e : g_occ[dev])
        if (e.v < 0) {
            e = OccEntry{v, tsm, smem, bps};
            break;
        }
    return bps;
}

// The configuration for length n: a pinned one, else the autotuner's, else the built-in default.
int current_short_variant(uint32_t n)
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    std::lock_guard<std::mutex> lk(g_short_mu);
    if (g_short_choice[dev] > 0) return g_short_choice[dev] - 1;
    for (const TunedEntry &e : g_short_tuned[dev])
        if (e.n == n && e.v >= 0) return e.v;
    return 0;
}

void remember_short_variant(uint32_t n, int v)
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    std::lock_guard<std::mutex> lk(g_short_mu);
    TunedEntry *slot = nullptr;
    for (TunedEntry &e : g_short_tuned[dev]) {
        if (e.n == n) {
            slot = &e;
            break;
        }
        if (!slot && e.v < 0) slot = &e;
    }
    if (!slot) slot = &g_short_tuned[dev][n % 64];  // table full: overwrite one entry
    slot->n = n;
    slot->v = v;
}

// Team size of the syndrome pass: a team of T lanes reads a codeword's Y
// position-domain words, ceil(Y / T) per lane (at most 64: one bit each in the
// two parity masks), and a tile's codewords take ceil(g / (32 / T)) rounds.
// Each round ends in a chain of dependent steps (the reductions, the
// butterfly over the team, the correction), which on GB300 measured as long as
// about 31 word steps (the paper's (M, t) grid: 3 rounds of 13 words took 139
// µs where 1 round of 32 took 111), plus a little per butterfly step.  Pick
// the T with the lowest cost per tile.
uint32_t team_log(uint32_t Y, uint32_t g)
{
    uint32_t best = 5;
    uint64_t best_cost = ~0ull;
    for (uint32_t lg = 0; lg <= 5; ++lg) {
        const uint32_t T = 1u << lg, G = 32u >> lg, per_lane = (Y + T - 1) / T;
        if (per_lane > 64) continue;
        const uint64_t cost = (uint64_t)((g + G - 1) / G) * (per_lane * 10u + 310u + 30u * lg);
        if (cost < best_cost) {
            best_cost = cost;
            best = lg;
        }
    }
    return best;
}

// Output-word offsets: entry idx describes output word idx of a run of
// codewords that starts at a multiple of 32 (32 codewords fill k words, so a
// tile's first word is entry (c0 mod 32) * k / 32).  The table covers one
// period of k words plus the longest tile and a lane's last group of reads,
// so no tile wraps.  Entry = delta: the word's first data bit is at bit
// 32*idx + delta counted from position 1 of the run's first codeword
// (delta = c*r + J + 1 for data bit d of codeword c in data run J).  Words
// holding a codeword's first 26 data bits, crossing into the next codeword or
// holding a checksum position are rewritten by the kernel's per-codeword
// passes; the first two kinds only point inside their codeword.
std::vector<uint32_t> output_table(uint32_t n, uint32_t k, uint32_t max_tile_words)
{
    const uint32_t r = n - k;
    const uint32_t len = k + max_tile_words + 128;
    std::vector<uint32_t> t(len, 0);
    for (uint32_t idx = 0; idx < len; ++idx) {
        const uint64_t e = 32ull * idx;
        const uint32_t c = (uint32_t)(e / k), d = (uint32_t)(e % k);
        uint32_t delta = c * r + 1u, split = 32;
        if (d >= 26 && k - d >= 32) {
            uint32_t J = 5;
            while (d >= (2u << J) - J - 2u) ++J;  // data run J holds data bits 2^J - J - 1 .. 2^(J+1) - J - 3
            delta = c * r + J + 1u;
            split = std::min<uint32_t>(32u, (2u << J) - J - 2u - d);
        }
        t[idx] = delta | (split << 16);
    }
    return t;
}

// Where the words holding a checksum position are resolved: per word in the
// output pass (32-bit entries) when k is small, so that codewords have few
// words and such words are common; else in a per-codeword pass (16-bit
// entries, half the table).
bool split_in_pass3(uint32_t k) { return k < 1280; }

// Build the output-word table of length n on the current device: cudaMalloc
// and a synchronous copy (the only allocation of the shortened-code path).
cudaError_t build_short_table(uint32_t n, uint32_t k, void **dev, uint32_t *len)
{
    // the longest tile of any configuration: the largest stage's codewords, plus a partial word
    const uint32_t max_words = (uint32_t)(((uint64_t)tile_codewords<8192>(n) * k + 31) / 32) + 1;
    const std::vector<uint32_t> full = output_table(n, k, max_words);
    const bool wide = split_in_pass3(k);
    std::vector<uint16_t> narrow;
    if (!wide)
        for (uint32_t e : full) narrow.push_back((uint16_t)(e & 0xFFFFu));
    const size_t bytes = wide ? full.size() * 4 : narrow.size() * 2;
    const void *src = wide ? static_cast<const void *>(full.data()) : static_cast<const void *>(narrow.data());
    void *d = nullptr;
    cudaError_t e = cudaMalloc(&d, bytes);
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return e;
    }
    *dev = d;
    *len = (uint32_t)full.size();
    return cudaSuccess;
}

// The tables that hd_decode_short builds on first use of a length, per
// device, least recently used first out.  Each table's last use is an event on
// the stream that used it, so evicting a table waits for that use only; a
// table used while its stream was capturing may be read by any later replay
// of that graph and is never evicted.
struct TableEntry {
    uint32_t n = 0;
    void *dev = nullptr;
    uint32_t len = 0;
    uint64_t used = 0;
    cudaEvent_t last = nullptr;  // recorded after each uncaptured use
    bool pinned = false;         // used inside a stream capture
};
constexpr int kMaxTables = 32;
TableEntry g_tables[64][kMaxTables];
uint64_t g_table_clock = 0;

bool stream_capturing(cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

// The cached table of length n for a launch on `st` (built on a miss, which a
// capturing stream may not do: cudaErrorStreamCaptureUnsupported).
cudaError_t table_for(uint32_t n, uint32_t k, cudaStream_t st, TableEntry **entry)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const bool capturing = stream_capturing(st);
    std::lock_guard<std::mutex> lk(g_short_mu);
    TableEntry *slot = nullptr;
    for (TableEntry &e : g_tables[dev]) {
        if (e.n == n && e.dev) {
            e.used = ++g_table_clock;
            *entry = &e;
            return cudaSuccess;
        }
        if (e.pinned) continue;
        if (!slot || (!e.dev && slot->dev) || (e.dev && slot->dev && e.used < slot->used)) slot = &e;
    }
    if (capturing) return cudaErrorStreamCaptureUnsupported;
    if (!slot) return cudaErrorMemoryAllocation;  // every slot is held by a captured graph
    if (slot->dev) {  // evict once its last use has finished
        if (slot->last && cudaEventSynchronize(slot->last) != cudaSuccess) return cudaErrorUnknown;
        cudaFree(slot->dev);
        slot->dev = nullptr;
        slot->n = 0;
    }
    void *d = nullptr;
    uint32_t len = 0;
    cudaError_t e = build_short_table(n, k, &d, &len);
    if (e != cudaSuccess) return e;
    if (!slot->last && cudaEventCreateWithFlags(&slot->last, cudaEventDisableTiming) != cudaSuccess) {
        cudaFree(d);
        return cudaErrorUnknown;
    }
    slot->n = n;
    slot->dev = d;
    slot->len = len;
    slot->used = ++g_table_clock;
    *entry = slot;
    return cudaSuccess;
}

// Mark a cached table's use by a launch just enqueued on `st`.
void table_used(TableEntry *e, cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(g_short_mu);
    if (stream_capturing(st)) e->pinned = true;
    else cudaEventRecord(e->last, st);
}

cudaError_t launch_short_tiles(int vi, const uint32_t *in, uint32_t n, uint64_t num_cw, uint32_t *out, void *syn,
                               int syn_type, unsigned long long *err, unsigned long long *det, cudaStream_t st,
                               const void *table, uint32_t tab_len, bool pdl = false)
{
    const ShortVariant &v = kShortVariants[vi];
    const uint32_t r = short_r(n), k = n - r;
    ShortArgs a{};
    a.in = in;
    a.out = out;
    a.syn = syn;
    a.err = err;
    a.det = det;
    a.status = status_ptr();
    if (!a.status) return cudaErrorUnknown;
    a.num_cw = num_cw;
    a.in_words = words_for_bits(num_cw * n);
    a.bulk_end = (a.in_words * 4) >> 4 << 4;
    a.n = n;
    a.k = k;
    a.g = std::min<uint32_t>((8u * v.SB - 256u) / n, TileGeom<4096>::max_g);  // as tile_codewords<SB>
    if (a.g == 0) return cudaErrorInvalidValue;  // the caller picks a configuration whose stage holds a codeword
    a.ntiles = (num_cw + a.g - 1) / a.g;
    a.Y = (n + 32) / 32;
    const uint32_t lastbits = n + 1 - 32 * (a.Y - 1);
    a.ylast = lastbits >= 32 ? 0xFFFFFFFFu : (1u << lastbits) - 1u;
    a.tlog = team_log(a.Y, a.g);
    a.table = table;
    a.tab_len = tab_len;
    if (!a.table) return cudaErrorInvalidValue;
    a.syn_type = syn ? syn_type : 0;
    a.nJ = 0;
    for (uint32_t J = 5; (2u << J) - J - 2u < k; ++J) ++a.nJ;
    a.nJ_magic = a.nJ > 1 ? (uint32_t)((0x100000000ull + a.nJ - 1) / a.nJ) : 0u;
    const bool split = split_in_pass3(k);
    const uint32_t tab_bytes = (a.tab_len * (split ? 4u : 2u) + 15) & ~15u;
    const int tsm = split ? 2 : (tab_bytes <= kTabSmemMax ? 1 : 0);  // split tables are small
    const uint32_t smem = v.stage_smem + (tsm ? tab_bytes : 0u);
    if (split) a.nJ = 0;  // no per-codeword pass for checksum words
    const int bps = short_blocks_per_sm(vi, tsm, smem);
    if (bps <= 0) return cudaErrorInvalidConfiguration;
    const uint64_t cap = (uint64_t)num_sms() * (uint64_t)bps;
    const uint64_t want = (a.ntiles + v.W - 1) / v.W;
    const int grid = decode_grid(want, cap);
    return v.launch[tsm](a, grid, smem, st, pdl);
}

}  // namespace
}  // namespace hd

using namespace hd;

namespace {
bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
}  // namespace

extern "C" {

hd_status hd_short_params(uint32_t n, uint32_t *r, uint32_t *k)
{
    if (n < 3 || n > kShortMaxN) return HD_ERR_INVALID_N;
    const uint32_t rr = short_r(n);
    if (r) *r = rr;
    if (k) *k = n - rr;
    return HD_OK;
}

hd_status hd_segment_params(uint32_t packet_bytes, uint32_t t, uint32_t *n, uint32_t *k, uint32_t *r)
{
    if (packet_bytes == 0 || t == 0 || t > 8u * packet_bytes) return HD_ERR_INVALID_ARG;
    const uint64_t kk = (8ull * packet_bytes + t - 1) / t;  // data bits per segment
    uint32_t rr = 0;
    while ((1ull << rr) < kk + rr + 1) ++rr;
    const uint64_t nn = kk + rr;
    if (nn < 3 || nn > kShortMaxN) return HD_ERR_SIZE;
    if (n) *n = (uint32_t)nn;
    if (k) *k = (uint32_t)kk;
    if (r) *r = rr;
    return HD_OK;
}

}  // extern "C"

namespace {

hd_status check_short_args(const uint32_t *stream, uint64_t in_bits, uint32_t n, uint64_t num_codewords,
                           uint32_t *out_bits, void *syndromes, hd_syn_type syn_type)
{
    if (n < 3 || n > kShortMaxN) return HD_ERR_INVALID_N;
    if (syn_type != HD_SYN_NONE && syn_type != HD_SYN_U8 && syn_type != HD_SYN_U16) return HD_ERR_INVALID_ARG;
    if (syn_type == HD_SYN_U8 && n > 255) return HD_ERR_INVALID_ARG;
    if (num_codewords > (1ull << 40)) return HD_ERR_SIZE;
    if (in_bits != (uint64_t)n * num_codewords) return HD_ERR_SIZE;
    if (num_codewords != 0) {
        if (!stream || !out_bits) return HD_ERR_NULL;
        if (syn_type != HD_SYN_NONE && !syndromes) return HD_ERR_NULL;
        if (!aligned16(stream) || !aligned16(out_bits) || (syndromes && !aligned16(syndromes))) return HD_ERR_ALIGN;
    }
    return HD_OK;
}

// The decode itself, given the output-word table of n (unused for k < 64);
// pdl: launched as the programmatic dependent of the counters' clear.
hd_status decode_short_with(const uint32_t *stream, uint64_t in_bits, uint32_t n, uint64_t num_codewords,
                            uint32_t *out_bits, void *syndromes, hd_syn_type syn_type,
                            unsigned long long *err_count, unsigned long long *detected_count, cudaStream_t st,
                            const void *table, uint32_t tab_len, bool pdl)
{
    const uint32_t r = short_r(n), k = n - r;
    const int syn = syndromes ? (int)syn_type : 0;
    if (k >= kLongMinK) {
        int vi = current_short_variant(n);
        if (kShortVariants[vi].SB * 8u < n + 256u) vi = largest_stage_variant();  // stage too small for a codeword
        if (launch_short_tiles(vi, stream, n, num_codewords, out_bits, syndromes, syn, err_count, detected_count,
                               st, table, tab_len, pdl) != cudaSuccess)
            return HD_ERR_CUDA;
        return HD_OK;
    }
    const uint64_t tiles = (num_codewords + 31) / 32;
    const uint64_t want = (tiles + kSmallWarps - 1) / kSmallWarps, cap = (uint64_t)num_sms() * 8;
    return launch_kernel(k_short_small, dim3((unsigned)decode_grid(want, cap)), dim3(kSmallWarps * 32), 0, st, pdl,
                         stream, words_for_bits(in_bits), n, r, num_codewords, out_bits,
                         words_for_bits(num_codewords * k), syndromes, syn, err_count, detected_count) == cudaSuccess
               ? HD_OK
               : HD_ERR_CUDA;
}

// Clear the counters (a one-thread kernel the decode may overlap); true when
// the decode is to be launched as its programmatic dependent.
hd_status clear_counts(unsigned long long *err_count, unsigned long long *detected_count, cudaStream_t st,
                       bool *pdl)
{
    *pdl = false;
    if (!err_count && !detected_count) return HD_OK;
    if (launch_zero_counts(err_count, detected_count, st) != cudaSuccess) return HD_ERR_CUDA;
    *pdl = true;
    return HD_OK;
}

}  // namespace

struct hd_short_plan {
    int device = 0;
    uint32_t n = 0;
    void *table = nullptr;  // output-word table (k >= 64), owned by the plan
    uint32_t tab_len = 0;
};

extern "C" {

hd_status hd_decode_short(const uint32_t *stream, uint64_t in_bits, uint32_t n, uint64_t num_codewords,
                          uint32_t *out_bits, void *syndromes, hd_syn_type syn_type, unsigned long long *err_count,
                          unsigned long long *detected_count, void *cuda_stream)
{
    hd_status rc = check_short_args(stream, in_bits, n, num_codewords, out_bits, syndromes, syn_type);
    if (rc != HD_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const uint32_t k = n - short_r(n);
    TableEntry *e = nullptr;
    if (num_codewords != 0 && k >= kLongMinK) {
        const cudaError_t te = table_for(n, k, st, &e);
        if (te == cudaErrorStreamCaptureUnsupported) return HD_ERR_INVALID_ARG;  // build it outside the capture
        if (te != cudaSuccess) return HD_ERR_CUDA;
    }
    bool pdl = false;
    if ((rc = clear_counts(err_count, detected_count, st, &pdl)) != HD_OK) return rc;
    if (num_codewords == 0) return HD_OK;
    rc = decode_short_with(stream, in_bits, n, num_codewords, out_bits, syndromes, syn_type, err_count,
                           detected_count, st, e ? e->dev : nullptr, e ? e->len : 0, pdl);
    if (e && rc == HD_OK) table_used(e, st);
    return rc;
}

hd_status hd_short_plan_create(uint32_t n, hd_short_plan **plan)
{
    if (!plan) return HD_ERR_NULL;
    *plan = nullptr;
    if (n < 3 || n > kShortMaxN) return HD_ERR_INVALID_N;
    hd_short_plan *p = new (std::nothrow) hd_short_plan();
    if (!p) return HD_ERR_CAPACITY;
    p->n = n;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return HD_ERR_CUDA;
    }
    const uint32_t k = n - short_r(n);
    if (k >= kLongMinK && build_short_table(n, k, &p->table, &p->tab_len) != cudaSuccess) {
        delete p;
        return HD_ERR_CUDA;
    }
    *plan = p;
    return HD_OK;
}

hd_status hd_decode_short_plan(const hd_short_plan *plan, const uint32_t *stream, uint64_t in_bits,
                               uint64_t num_codewords, uint32_t *out_bits, void *syndromes, hd_syn_type syn_type,
                               unsigned long long *err_count, unsigned long long *detected_count, void *cuda_stream)
{
    if (!plan) return HD_ERR_NULL;
    hd_status rc = check_short_args(stream, in_bits, plan->n, num_codewords, out_bits, syndromes, syn_type);
    if (rc != HD_OK) return rc;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HD_ERR_CUDA;
    if (dev != plan->device) return HD_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    bool pdl = false;
    if ((rc = clear_counts(err_count, detected_count, st, &pdl)) != HD_OK) return rc;
    if (num_codewords == 0) return HD_OK;
    return decode_short_with(stream, in_bits, plan->n, num_codewords, out_bits, syndromes, syn_type, err_count,
                             detected_count, st, plan->table, plan->tab_len, pdl);
}

void hd_short_plan_destroy(hd_short_plan *plan)
{
    if (!plan) return;
    if (plan->table) {
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur != plan->device) cudaSetDevice(plan->device);
        cudaFree(plan->table);  // waits for the work that may still read it
        if (cur != plan->device) cudaSetDevice(cur);
    }
    delete plan;
}

hd_status hd_encode_short(const uint32_t *data_bits, uint32_t n, uint64_t num_codewords, uint32_t *stream,
                          void *cuda_stream)
{
    if (n < 3 || n > kShortMaxN) return HD_ERR_INVALID_N;
    if (num_codewords > (1ull << 40)) return HD_ERR_SIZE;
    if (num_codewords == 0) return HD_OK;
    if (!data_bits || !stream) return HD_ERR_NULL;
    if (!aligned16(data_bits) || !aligned16(stream)) return HD_ERR_ALIGN;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const uint32_t r = short_r(n), k = n - r;
    if (cudaMemsetAsync(stream, 0, words_for_bits(num_codewords * n) * 4, st) != cudaSuccess) return HD_ERR_CUDA;
    const uint64_t want = (num_codewords + 255) / 256, cap = (uint64_t)num_sms() * 16;
    k_encode_short<<<(int)std::min(want, cap), 256, 0, st>>>(data_bits, words_for_bits(num_codewords * k), n, r,
                                                             num_codewords, stream);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? HD_OK : HD_ERR_CUDA;
}

hd_status hd_short_autotune(uint32_t n, uint64_t num_codewords, uint32_t reps, void *cuda_stream, int32_t *chosen)
{
    if (n < 3 || n > kShortMaxN) return HD_ERR_INVALID_N;
    const uint32_t r = short_r(n), k = n - r;
    if (num_codewords == 0 || num_codewords > (1ull << 32)) return HD_ERR_SIZE;
    if (reps == 0) reps = 5;
    if (k < kLongMinK) {  // one kernel only
        if (chosen) *chosen = -1;
        return HD_OK;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const size_t in_b = words_for_bits(num_codewords * n) * 4 + 16, out_b = words_for_bits(num_codewords * k) * 4 + 16;
    void *din = nullptr, *dout = nullptr, *dsyn = nullptr, *dcnt = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    hd_status rc = HD_OK;
    int best = -1;
    float best_ms = 0.f;
    if (cudaMalloc(&din, in_b) != cudaSuccess || cudaMalloc(&dout, out_b) != cudaSuccess ||
        cudaMalloc(&dsyn, num_codewords * 2 + 16) != cudaSuccess || cudaMalloc(&dcnt, 16) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        rc = HD_ERR_CUDA;
    // all-zero segments are codewords: the timing sees the common no-error path
    if (rc == HD_OK && cudaMemsetAsync(din, 0, in_b, st) != cudaSuccess) rc = HD_ERR_CUDA;
    auto *cnt = static_cast<unsigned long long *>(dcnt);
    TableEntry *tab = nullptr;
    if (rc == HD_OK && table_for(n, k, st, &tab) != cudaSuccess) rc = HD_ERR_CUDA;
    for (int v = 0; rc == HD_OK && v < kNumShortVariants; ++v) {
        if (kShortVariants[v].SB * 8u < n + 256u) continue;
        auto go = [&]() {
            return launch_short_tiles(v, static_cast<const uint32_t *>(din), n, num_codewords,
                                      static_cast<uint32_t *>(dout), dsyn, HD_SYN_U16, cnt, cnt + 1, st, tab->dev,
                                      tab->len);
        };
        if (go() != cudaSuccess) {  // warm-up (also configures the kernel)
            rc = HD_ERR_CUDA;
            break;
        }
        cudaEventRecord(e0, st);
        for (uint32_t i = 0; i < reps; ++i) go();
        cudaEventRecord(e1, st);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = HD_ERR_CUDA;
            break;
        }
        if (best < 0 || ms < best_ms) {
            best = v;
            best_ms = ms;
        }
    }
    if (tab) table_used(tab, st);
    if (din) cudaFree(din);
    if (dout) cudaFree(dout);
    if (dsyn) cudaFree(dsyn);
    if (dcnt) cudaFree(dcnt);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc != HD_OK) return rc;
    if (best >= 0) remember_short_variant(n, best);
    if (chosen) *chosen = best;
    return HD_OK;
}

hd_status hd_short_variant_count(uint32_t *count)
{
    if (!count) return HD_ERR_NULL;
    *count = (uint32_t)kNumShortVariants;
    return HD_OK;
}

hd_status hd_short_variant_select(int32_t ordinal)
{
    if (ordinal >= kNumShortVariants) return HD_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return HD_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_short_mu);
    g_short_choice[dev] = ordinal < 0 ? 0 : ordinal + 1;
    return HD_OK;
}

}  // extern "C"
