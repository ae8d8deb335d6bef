// hd_batch.cu -- batched decode of many packets of mixed n and length in one
// persistent launch.
//
// A plan turns the packet table into a device table of tiles: every packet is
// cut into full warp chunks of 32*G codewords (G = 32 for n <= 31, 16 for
// n = 63, 8 for n = 127; n = 255 takes half-warp chunks of 16*8, so a chunk's
// input is at most 4 KB) and, when its length is not a multiple of that, one
// ragged tail tile.  The warps of a
// persistent kernel take tiles in table order (tiles grouped by n, each
// code's tails spread among its full tiles; claimed from an atomic counter, or
// dealt round-robin by the single-n kernels), prefetch their tiles into its own shared-memory stages with 1-D bulk copies,
// decodes full tiles with the same per-warp chunk decoder as the streaming
// kernel, decodes tails with the chunk decoder too (copied in, zero-padded to a
// chunk, copied back out; n = 3 tails use the generic warp-tile decoder), and
// adds each tile's nonzero-syndrome count to its packet's error counter.
// Cutting packets whose lengths span six orders of magnitude into bounded
// tiles is what balances the load.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "hd_batch_internal.h"
#include "hd_generic.cuh"
#include "hd_internal.h"
#include "hd_multi.cuh"
#include "hd_stream.cuh"

namespace hd {

struct DevPacket {
    const uint32_t *in;
    uint32_t *out;
    uint8_t *syn;
    uint64_t num_cw;
    uint64_t in_words;
    uint64_t out_words;
    uint32_t n;
    uint32_t m;
    uint32_t syn_type;
    uint32_t pad;
};

// Tails are cut to at most this many codewords (a tail of n >= 7 is shorter
// than one chunk anyway; n = 3 streams are all tail).
constexpr uint64_t kTailTile = 1024;

__host__ __device__ constexpr int batch_G(uint32_t n) { return n >= 127 ? 8 : (n >= 63 ? 16 : 32); }

// Lanes of a chunk: n = 255 decodes half-warp chunks (128 codewords, 4080
// bytes), so that every chunk's input fits a 4 KB stage.
__host__ __device__ constexpr int batch_lanes(uint32_t n) { return n >= 255 ? 16 : 32; }

// Codewords per chunk.
__host__ __device__ constexpr uint64_t batch_chunk_cw(uint32_t n)
{
    return (uint64_t)batch_G(n) * (uint64_t)batch_lanes(n);
}

// Chunks per full tile: small codes pack several chunks (at most 4096
// codewords) so that every tile moves several KB and the per-tile overhead
// and load latency are amortised.
__host__ __device__ constexpr int batch_chunks(uint32_t n) { return n <= 7 ? 4 : (n <= 15 ? 2 : 1); }

// The long codes' geometry in the split configuration (BIG): the streaming
// kernel's chunk shapes in 8 KB stages -- n = 63 with 32 codewords per thread
// (1024 per chunk, 8064 bytes), n = 127 with two 256-codeword chunks per tile
// (8128 bytes), n = 255 with full-warp chunks of 256 codewords (8160 bytes) --
// so that a tile holds twice the work of the 4 KB tiles, and n = 63 and 255
// decode whole 32-codeword tiles per thread part (n = 255: 0.42 -> 0.57 of
// the HBM peak on its share of the batched workload).  The same 8 KB tiles
// measured no faster for n = 7 and 31, and n = 15's kernel holds its 64 KB
// table beside its warps, so the other codes keep the 4 KB geometry.
__host__ __device__ constexpr bool big_geometry(uint32_t n) { return n == 63 || n == 127 || n == 255; }
__host__ __device__ constexpr int geo_G(uint32_t n, bool big) { return big && n == 63 ? 32 : batch_G(n); }
__host__ __device__ constexpr int geo_lanes(uint32_t n, bool big) { return big ? 32 : batch_lanes(n); }
__host__ __device__ constexpr uint64_t geo_chunk_cw(uint32_t n, bool big)
{
    return (uint64_t)geo_G(n, big) * (uint64_t)geo_lanes(n, big);
}
__host__ __device__ constexpr int geo_chunks(uint32_t n, bool big)
{
    return !big ? batch_chunks(n) : (n == 127 ? 2 : 1);
}

uint64_t packet_tiles(uint32_t n, uint64_t num_codewords)
{
    const uint64_t chunk = batch_chunk_cw(n);
    const uint64_t nfull = n == 3 ? 0 : num_codewords / chunk;  // n = 3: all tail
    const uint64_t per = (uint64_t)batch_chunks(n);
    return (nfull + per - 1) / per + (num_codewords - nfull * chunk + kTailTile - 1) / kTailTile;
}

// One packet as the tile builders see it.
struct PacketView {
    const uint32_t *in;
    uint32_t *out;
    uint8_t *syn;
    uint64_t num_cw;
    uint32_t n, m, syn_type;
};

// Emit the tiles of every packet of code length n, without allocating: full
// tiles in packet order, with the packets' ragged tails spread evenly among
// them (after each full tile, tails until their share matches), so that the
// latency-bound tails overlap the streaming of full tiles instead of running
// as a phase of their own.  view(i) describes packet i; emit(tile) takes a tile.
template <class View, class Emit>
void emit_code_tiles(uint32_t n, uint32_t num_packets, View view, Emit emit, bool big = false)
{
    big = big && big_geometry(n);
    const uint64_t chunk = geo_chunk_cw(n, big);
    const uint64_t per = (uint64_t)geo_chunks(n, big);
    auto nfull_of = [&](const PacketView &p) { return n == 3 ? 0 : p.num_cw / chunk; };  // n = 3: all tail
    uint64_t nf = 0, nt = 0;  // full tiles and tail tiles of this n
    for (uint32_t i = 0; i < num_packets; ++i) {
        const PacketView p = view(i);
        if (p.n != n) continue;
        const uint64_t f = nfull_of(p);
        nf += (f + per - 1) / per;
        nt += (p.num_cw - f * chunk + kTailTile - 1) / kTailTile;
    }
    uint32_t ti = 0;  // tail cursor: packet and next codeword
    uint64_t tc = 0;
    auto next_tail = [&]() -> bool {
        for (; ti < num_packets; ++ti, tc = 0) {
            const PacketView p = view(ti);
            if (p.n != n) continue;
            tc = std::max(tc, nfull_of(p) * chunk);
            if (tc < p.num_cw) {
                // a chunk-decoded tail prefetches the whole 16-byte groups of its
                // input with the stage's bulk copy (it starts on a chunk boundary,
                // so 16-byte aligned); the last words are loaded when it is decoded
                const uint32_t cnt = (uint32_t)std::min<uint64_t>(kTailTile, p.num_cw - tc);
                const uint32_t bulk = n == 3 ? 0u : (uint32_t)(((uint64_t)cnt * n + 31) / 32 * 4) & ~15u;
                emit(make_tile(p.in, p.out, p.syn, p.num_cw, n, p.m, p.syn_type, ti, tc, cnt, bulk));
                tc += kTailTile;
                return true;
            }
        }
        return false;
    };
    uint64_t done_full = 0, done_tail = 0;
    for (uint32_t i = 0; i < num_packets; ++i) {
        const PacketView p = view(i);
        if (p.n != n) continue;
        const uint64_t f = nfull_of(p);
        for (uint64_t j = 0; j < f; j += per) {
            const uint64_t c = std::min(per, f - j);
            emit(make_tile(p.in, p.out, p.syn, p.num_cw, n, p.m, p.syn_type, i, j * chunk,
                           (uint32_t)(c * chunk) | kFullTile, (uint32_t)(c * chunk * n / 8)));
            ++done_full;
            while (done_tail * nf < done_full * nt && next_tail()) ++done_tail;
        }
    }
    while (next_tail()) ++done_tail;
}

// Largest tile input (n = 255 half chunk: 4080 B; n = 127: 4064; n = 63: 4032;
// n = 31: 3968; n = 15, two chunks: 3840; n = 7, four: 3584) plus a spare
// group for the funnel read; 4 KB stages let 16 one-warp CTAs share an SM.
constexpr uint32_t kBatchStageBytes = 4096 + 16;
constexpr uint32_t kBigStageBytes = 8192 + 16;  // the split configuration's long codes
// Full tiles write their syndromes straight to global memory (each lane's run
// of G syndromes is contiguous); only a ragged tail, at most one chunk, stages
// them here before the copy that keeps within the packet.
constexpr uint32_t kBatchSynBytes = 32 * 32 * 2;  // one chunk of at most 1024 codewords, u16

template <int WARPS, int S, bool T15, bool BIG = false>
struct BatchCfg {
    static constexpr uint32_t stage_bytes = BIG ? kBigStageBytes : kBatchStageBytes;
    static constexpr uint32_t off_bar = 0;
    static constexpr uint32_t off_claim = 64;  // per stage: the claimed tile index and its descriptor
    static constexpr uint32_t off_desc = 128;
    static constexpr uint32_t off_stage = off_desc + 8 * 64;
    static constexpr uint32_t off_syn = off_stage + S * stage_bytes;
    static constexpr uint32_t warp_bytes = (off_syn + kBatchSynBytes + 127) / 128 * 128;
    // behind the warps' areas: the n = 7 decode table, (T15) the n = 15 one,
    // and the mbarrier of the n = 15 table's bulk copies
    static constexpr uint32_t off_lut7 = WARPS * warp_bytes;
    static constexpr uint32_t off_lut15 = off_lut7 + (2u << 7);
    static constexpr uint32_t lut15_bytes = T15 ? (2u << 15) : 0u;
    static constexpr uint32_t off_lut_bar = off_lut15 + lut15_bytes;
    static constexpr uint32_t smem = off_lut_bar + 16;
    static_assert(S >= 2 && S <= 8, "refills lag one iteration: at least two stages");
    static_assert(kWarpSlotWords * 4 * 2 <= kBatchStageBytes, "generic slots fit a stage");
    static_assert(smem <= 232448, "shared memory per CTA");
};

// Decode the `chunks` whole chunks of a full tile held in `stage`, in place:
// chunk c's output goes to stage + c*out_words, which never overlaps a later
// chunk's input because k < n.  Chunk c's syndromes go to sdst + c * (bytes of
// one chunk's syndromes): global memory for a full tile, the warp's staging
// buffer for a tail.
template <int N_, int SYN, bool LUT, bool BIG = false>
__device__ __forceinline__ uint32_t batch_chunk(const uint32_t *stage, uint8_t *sdst, int lane, uint32_t chunks,
                                                const uint16_t *lut)
{
    constexpr bool B = BIG && big_geometry(N_);
    constexpr int G = geo_G(N_, B), LN = geo_lanes(N_, B);
    using Q = ChunkGeom<N_, SYN, G, false, LN>;
    uint32_t e = 0, unused = 0;
    for (uint32_t c = 0; c < chunks; ++c)
        e += decode_warp_chunk<N_, SYN, G, false, LUT, LN>(stage + c * Q::in_words,
                                                           const_cast<uint32_t *>(stage) + c * Q::out_words,
                                                           sdst + c * Q::syn_bytes, lane, unused, lut);
    return e;
}

// LUT: decode with the table `lut` in shared memory (n = 7 and 15 only).
template <int N_, bool LUT = false, bool BIG = false>
__device__ __forceinline__ uint32_t batch_chunk_syn(uint32_t syn_type, const uint32_t *stage, uint8_t *sdst, int lane,
                                                    uint32_t chunks, const uint16_t *lut = nullptr)
{
    switch (syn_type) {
        case 1: return batch_chunk<N_, 1, LUT, BIG>(stage, sdst, lane, chunks, lut);
        case 2: return batch_chunk<N_, 2, LUT, BIG>(stage, sdst, lane, chunks, lut);
        default: return batch_chunk<N_, 0, LUT, BIG>(stage, sdst, lane, chunks, lut);
    }
}

__device__ __forceinline__ uint32_t chunk_codewords(uint32_t n, bool big = false)
{
    return (uint32_t)geo_chunk_cw(n, big && big_geometry(n));
}

// lut7 (or nullptr: arithmetic decode) and, with T15, lut15 (required) are
// the global decode tables of n = 7 and 15; the kernel copies them into shared
// memory once per CTA.  NSEL = 0 decodes tiles of every n; NSEL = n compiles
// only the decoder of that n (every tile of the table must be of that n), so
// that the kernel's code fits the instruction cache.
template <int WARPS, int S, bool T15, int NSEL = 0, bool BIG = false>
__global__ void __launch_bounds__(WARPS * 32)
    k_decode_batch(const DevTile *__restrict__ tiles, uint32_t num_tiles, uint32_t *__restrict__ counter,
                   unsigned long long *__restrict__ err_counts, uint32_t *__restrict__ status,
                   const uint16_t *__restrict__ lut7, const uint16_t *__restrict__ lut15)
{
    using Cfg = BatchCfg<WARPS, S, T15, BIG>;
    static_assert(!BIG || big_geometry(NSEL), "the 8 KB geometry is for the long codes' single-n kernels");
    extern __shared__ __align__(128) uint8_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t *lut_bar = reinterpret_cast<uint64_t *>(smem + Cfg::off_lut_bar);
    if constexpr (T15) {
        // the n = 15 table: bulk copies on the CTA's table barrier, in flight
        // while the warps claim and load their first tiles
        if (threadIdx.x == 0) {
            mbar_init(lut_bar, 1);
            fence_mbar_init();
            mbar_arrive_expect_tx(lut_bar, Cfg::lut15_bytes);
#pragma unroll
            for (uint32_t o = 0; o < Cfg::lut15_bytes; o += 16384u)
                bulk_g2s(smem + Cfg::off_lut15 + o, reinterpret_cast<const uint8_t *>(lut15) + o, 16384u, lut_bar);
        }
    }
    if ((NSEL == 0 || NSEL == 7) && lut7 != nullptr && threadIdx.x < 16)  // 256 bytes
        reinterpret_cast<uint4 *>(smem + Cfg::off_lut7)[threadIdx.x] =
            __ldg(reinterpret_cast<const uint4 *>(lut7) + threadIdx.x);
    __syncthreads();  // the n = 7 table is in place and the table barrier initialised
    const uint16_t *s_lut7 = reinterpret_cast<const uint16_t *>(smem + Cfg::off_lut7);
    const uint16_t *s_lut15 = reinterpret_cast<const uint16_t *>(smem + Cfg::off_lut15);
    uint8_t *wbase = smem + warp * Cfg::warp_bytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(wbase + Cfg::off_bar);
    volatile uint32_t *claim = reinterpret_cast<volatile uint32_t *>(wbase + Cfg::off_claim);
    DevTile *desc = reinterpret_cast<DevTile *>(wbase + Cfg::off_desc);
    uint8_t *s_stage = wbase + Cfg::off_stage;
    uint8_t *s_syn = wbase + Cfg::off_syn;

    // lane 0: record claim t with descriptor d in stage s's slot and start its
    // load (tails are read by the whole warp later; past-the-end claims load nothing)
    auto issue = [&](int s, uint32_t t, const DevTile &d) {
        claim[s] = t;
        if (t < num_tiles) desc[s] = d;
        if (t < num_tiles && d.bytes != 0) {
            mbar_arrive_expect_tx(&bar[s], d.bytes);
            bulk_g2s(s_stage + s * Cfg::stage_bytes, d.in + d.c0 * d.n / 32u, d.bytes, &bar[s]);
        } else {
            mbar_arrive(&bar[s]);
        }
    };
    // Which tile a warp takes next.  The single-n kernels (NSEL != 0) deal
    // tiles round-robin: warp gw takes tiles gw, gw + tw, gw + 2 tw, ... (tw
    // warps in the grid), which balances their tiles of one code without an
    // atomic per tile on one shared address.  The all-n kernel, whose tiles
    // differ more in cost, claims them from the atomic counter, so that a warp
    // that finished early takes more (measured: 250 µs claimed against 267 µs
    // dealt for it; 246 against 239 µs for the single-n kernels).  Either way the
    // next tile is claimed, and its descriptor fetched, one iteration ahead.
    const uint64_t gw = (uint64_t)blockIdx.x * WARPS + (uint64_t)warp, tw = (uint64_t)gridDim.x * WARPS;
    uint32_t seq = 0;  // lane 0: tiles dealt to this warp so far
    auto deal = [&]() -> uint32_t {
        if constexpr (NSEL == 0) {
            return atomicAdd(counter, 1u);
        } else {
            const uint64_t t = gw + (uint64_t)(seq++) * tw;
            return t < (uint64_t)num_tiles ? (uint32_t)t : num_tiles;
        }
    };
    // The single-n kernels fetch a descriptor two iterations before its tile
    // is issued (next_d is in registers when its refill is due, after_d is in
    // flight), since one of their decodes can be shorter than a load from L2;
    // the all-n kernel, at its register limit, fetches one iteration ahead.
    constexpr bool kAhead2 = NSEL != 0;
    uint32_t next_t = 0, after_t = 0;
    DevTile next_d{}, after_d{};
    if (lane == 0) {
#pragma unroll
        for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
        // the claim counter and the error counters are cleared by the kernel
        // ahead of this one, which a programmatic dependent launch overlaps
        grid_dep_wait();
        for (int s = 0; s < S; ++s) {
            const uint32_t t = deal();
            DevTile d{};
            if (t < num_tiles) d = tiles[t];
            issue(s, t, d);
        }
        next_t = deal();
        if constexpr (kAhead2) {
            if (next_t < num_tiles) next_d = tiles[next_t];  // issued at the end of iteration 1
            after_t = deal();
        }
    }
    __syncwarp();

    uint32_t it = 0;
    bool aborted = false;
    if constexpr (T15) aborted = __any_sync(0xFFFFFFFFu, !mbar_wait_bounded(lut_bar, 0));
    for (; !aborted; ++it) {
        const int s = (int)(it % S);
        const bool ok = mbar_wait_bounded(&bar[s], (it / S) & 1u);
        if (__any_sync(0xFFFFFFFFu, !ok)) {
            aborted = true;
            break;
        }
        const uint32_t t = claim[s];
        if (t >= num_tiles) break;  // claims only grow: every later stage is past the end too
        // from the second iteration on, every iteration refills the previous
        // iteration's stage at its end: fetch the descriptor of the tile claimed
        // last iteration and claim the next one
        uint32_t later_t = 0;
        if (lane == 0 && it > 0) {
            if constexpr (kAhead2) {
                if (after_t < num_tiles) after_d = tiles[after_t];  // used at the end of the next iteration
            } else {
                if (next_t < num_tiles) next_d = tiles[next_t];  // used at the end of this iteration
            }
            later_t = deal();  // its descriptor is fetched next iteration
        }
        const DevTile tl = desc[s];  // written by lane 0 before the stage's arrive
        // the single-n kernels know n at compile time: the per-tile index
        // arithmetic (word counts, chunks per tile) folds to constants
        const uint32_t pn = NSEL != 0 ? (uint32_t)NSEL : (uint32_t)tl.n;
        const uint32_t pm = NSEL != 0 ? (uint32_t)log2_exact(NSEL + 1) : (uint32_t)tl.m;
        struct {
            const uint32_t *in;
            uint32_t *out;
            uint8_t *syn;
            uint64_t num_cw, in_words, out_words;
            uint32_t n, m, syn_type;
        } p{tl.in, tl.out, tl.syn, tl.num_cw, (tl.num_cw * pn + 31) / 32, (tl.num_cw * (pn - pm) + 31) / 32,
            pn, pm, tl.syn_type};
        const bool full = (tl.count & kFullTile) != 0;
        const uint32_t chunks = full ? (tl.count & ~kFullTile) / chunk_codewords(p.n, BIG) : 0u;
        uint32_t *stage = reinterpret_cast<uint32_t *>(s_stage + s * Cfg::stage_bytes);
        uint8_t *sbuf = s_syn;
        uint8_t *sdst = (full && p.syn_type != 0) ? p.syn + tl.c0 * (p.syn_type == 2 ? 2u : 1u) : sbuf;
        unsigned long long errs = 0;
        const bool chunked = NSEL == 0 ? (full || p.n != 3) : NSEL != 3;  // n = 3 tiles are all tails
        if (chunked) {
            const uint32_t cwords = chunk_codewords(p.n, BIG);
            const uint32_t k = p.n - p.m;
            const uint32_t cnt = tl.count & ~kFullTile;
            if (!full) {
                // ragged tail of cnt < one chunk: its whole 16-byte groups came
                // with the stage's bulk copy (tl.bytes); load the last words,
                // drop the input pad bits and zero-fill the chunk, so that the
                // padding decodes to zero data bits and zero syndromes
                const uint32_t iw = (cnt * p.n + 31) / 32, cw_words = cwords * p.n / 32 + 4;
                const uint32_t tail_bits = (cnt * p.n) & 31u;
                const uint32_t *src = p.in + tl.c0 * p.n / 32u;
                const uint32_t have = tl.bytes / 4;  // words already in the stage
                for (uint32_t w = have + lane; w < cw_words; w += 32) {
                    uint32_t v = w < iw ? src[w] : 0u;
                    if (w == iw - 1 && tail_bits != 0) v &= (1u << tail_bits) - 1u;
                    stage[w] = v;
                }
                if (lane == 0 && tail_bits != 0 && iw - 1 < have) stage[iw - 1] &= (1u << tail_bits) - 1u;
                __syncwarp();
            }
            uint32_t e = 0;
            const uint32_t nch = full ? chunks : 1u;
            if constexpr (NSEL == 0) {
                switch (p.n) {
                    case 7:
                        e = lut7 != nullptr ? batch_chunk_syn<7, true>(p.syn_type, stage, sdst, lane, nch, s_lut7)
                                            : batch_chunk_syn<7>(p.syn_type, stage, sdst, lane, nch);
                        break;
                    case 15:
                        if constexpr (T15)
                            e = batch_chunk_syn<15, true>(p.syn_type, stage, sdst, lane, nch, s_lut15);
                        else
                            e = batch_chunk_syn<15>(p.syn_type, stage, sdst, lane, nch);
                        break;
                    case 31: e = batch_chunk_syn<31>(p.syn_type, stage, sdst, lane, nch); break;
                    case 63: e = batch_chunk_syn<63>(p.syn_type, stage, sdst, lane, nch); break;
                    case 127: e = batch_chunk_syn<127>(p.syn_type, stage, sdst, lane, nch); break;
                    case 255: e = batch_chunk_syn<255>(p.syn_type, stage, sdst, lane, nch); break;
                    default: break;  // the plan never makes chunk tiles of other lengths
                }
            } else if constexpr (NSEL == 7) {
                e = lut7 != nullptr ? batch_chunk_syn<7, true>(p.syn_type, stage, sdst, lane, nch, s_lut7)
                                    : batch_chunk_syn<7>(p.syn_type, stage, sdst, lane, nch);
            } else if constexpr (NSEL == 15) {
                if constexpr (T15)
                    e = batch_chunk_syn<15, true>(p.syn_type, stage, sdst, lane, nch, s_lut15);
                else
                    e = batch_chunk_syn<15>(p.syn_type, stage, sdst, lane, nch);
            } else if constexpr (NSEL != 3) {
                e = batch_chunk_syn<NSEL, false, BIG>(p.syn_type, stage, sdst, lane, nch);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xFFFFFFFFu, e, o);
            errs = e;
            if (!full) {
                // write back only the tail's words and syndromes
                __syncwarp();
                const uint32_t ow = (cnt * k + 31) / 32;
                uint32_t *dst = p.out + tl.c0 * k / 32u;
                for (uint32_t w = lane; w < ow; w += 32) dst[w] = stage[w];
                if (p.syn_type == 1)
                    for (uint32_t i = lane; i < cnt; i += 32) p.syn[tl.c0 + i] = sbuf[i];
                else if (p.syn_type == 2)
                    for (uint32_t i = lane; i < cnt; i += 32)
                        reinterpret_cast<uint16_t *>(p.syn)[tl.c0 + i] = reinterpret_cast<const uint16_t *>(sbuf)[i];
            }
            fence_proxy_async_smem();
            __syncwarp();
        } else {
            // n = 3: generic warp tiles, the (unloaded) stage as slot memory
            errs = generic_decode_tiles(p.in, p.in_words, p.n, p.m, p.num_cw, tl.c0 / 32, (tl.c0 + tl.count + 31) / 32,
                                        1, p.out, p.out_words, p.syn, (int)p.syn_type, stage, stage + kWarpSlotWords);
            fence_proxy_async_smem();
            __syncwarp();
        }
        if (lane == 0) {
            // the previous iteration's stage held that tile's output; its store
            // has had this whole decode to read it: refill the stage with the
            // tile claimed last iteration (so the lookahead is S - 1 tiles)
            if (it > 0) {
                bulk_wait_read<0>();
                issue((int)((it - 1) % S), next_t, next_d);
                if constexpr (kAhead2) {
                    next_t = after_t;
                    next_d = after_d;
                    after_t = later_t;
                } else {
                    next_t = later_t;
                }
            }
            if (full) {
                const uint32_t cw = tl.count & ~kFullTile;
                const uint32_t k = p.n - p.m;
                bulk_s2g(p.out + tl.c0 * k / 32u, stage, cw * k / 8u);
                bulk_commit();
            }
            if (err_counts != nullptr && errs != 0) atomicAdd(&err_counts[tl.packet], errs);
        }
        __syncwarp();
    }
    if (lane == 0) {
        if (aborted) {
            atomicOr(status, (uint32_t)HD_ERR_TIMEOUT);
            // loads still in flight: the S of the prologue before the first
            // iteration, afterwards S - 1 (refills lag one iteration)
            const uint32_t pending = it > 0 ? S - 1 : S;
            for (uint32_t j = it; j < it + pending; ++j) (void)mbar_wait_bounded(&bar[j % S], (j / S) & 1u);
            if constexpr (T15) (void)mbar_wait_bounded(lut_bar, 0);
        }
        bulk_wait_all<0>();
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct BatchVariant {
    int warps, stages;
    bool t15;  // holds the n = 15 decode table (needs it at launch)
    uint32_t smem;
    const void *kernel;
    void (*launch)(int grid, uint32_t smem, cudaStream_t st, const DevTile *, uint32_t, uint32_t *,
                   unsigned long long *, uint32_t *, const uint16_t *, const uint16_t *, bool pdl);
};

template <int W, int S, bool T15, int NSEL = 0, bool BIG = false>
void launch_batch_kernel(int grid, uint32_t smem, cudaStream_t st, const DevTile *tiles, uint32_t num_tiles,
                         uint32_t *counter, unsigned long long *err, uint32_t *status, const uint16_t *lut7,
                         const uint16_t *lut15, bool pdl)
{
    // the callers count batch launches (a plan's once per graph replay)
    (void)launch_kernel_uncounted(k_decode_batch<W, S, T15, NSEL, BIG>, dim3((unsigned)grid), dim3(W * 32), smem, st,
                                  pdl, tiles, num_tiles, counter, err, status, lut7, lut15);
}

// Clears a plan's claim counters and error counters, then lets the next
// kernel of the stream start (programmatic dependent launch).
__global__ void k_clear_plan(uint32_t *counters, uint32_t num_counters, unsigned long long *err, uint32_t num_err)
{
    grid_dep_launch_dependents();
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    for (uint32_t j = i; j < num_counters; j += stride) counters[j] = 0u;
    if (err != nullptr)
        for (uint32_t j = i; j < num_err; j += stride) err[j] = 0ull;
}

template <int W, int S, bool T15 = false, int NSEL = 0, bool BIG = false>
BatchVariant make_batch_variant()
{
    BatchVariant v;
    v.warps = W;
    v.stages = S;
    v.t15 = T15;
    v.smem = BatchCfg<W, S, T15, BIG>::smem;
    v.kernel = reinterpret_cast<const void *>(k_decode_batch<W, S, T15, NSEL, BIG>);
    v.launch = &launch_batch_kernel<W, S, T15, NSEL, BIG>;
    return v;
}

// The split configuration: one kernel per code length, each compiled for its
// n only, launched as concurrent branches of the plan's graph.  Index i
// follows kSplitOrder; n = 15 has a second kernel that holds its decode table
// (used when the table is filled).
constexpr uint32_t kSplitOrder[] = {255, 127, 63, 31, 15, 7, 3};
constexpr int kSplitGroups = 7;

struct SplitKernels {
    BatchVariant group[kSplitGroups];
    BatchVariant n15_table;
};

template <int W, int S>
SplitKernels make_split_kernels()
{
    SplitKernels s;
    s.group[0] = make_batch_variant<W, S, false, 255, true>();
    s.group[1] = make_batch_variant<W, S, false, 127, true>();
    s.group[2] = make_batch_variant<W, S, false, 63, true>();
    s.group[3] = make_batch_variant<W, S, false, 31>();
    s.group[4] = make_batch_variant<W, S, false, 15>();
    s.group[5] = make_batch_variant<W, S, false, 7>();
    s.group[6] = make_batch_variant<W, S, false, 3>();
    s.n15_table = make_batch_variant<14, 2, true, 15>();
    return s;
}

static const std::vector<BatchVariant> &batch_variants()
{
    // index 0 is the built-in choice (and the serving and allocation-free
    // paths' configuration); it holds no n = 15 table
    static const std::vector<BatchVariant> v = {
        make_batch_variant<1, 3>(),        make_batch_variant<1, 2>(),        make_batch_variant<1, 4>(),
        make_batch_variant<2, 2>(),        make_batch_variant<4, 2>(),        make_batch_variant<8, 2, true>(),
        make_batch_variant<12, 2, true>(), make_batch_variant<14, 2, true>()};
    return v;
}

// The split configurations (warps per CTA and stages of the single-n
// kernels).  One-warp CTAs with three stages: on the 10,000-packet workload
// 241 µs, against 261 µs with two-warp CTAs (three stages) and 263 µs with
// four-warp CTAs (two stages).
const std::vector<SplitKernels> &split_kernels()
{
    static const std::vector<SplitKernels> k = {make_split_kernels<1, 3>()};
    return k;
}

// The stream-group configuration's kernels (hd_multi_a.cu, hd_multi_b.cu):
// the streaming decoder over the whole chunks of many packets of one n.
const std::vector<MultiVariant> &multi_variants()
{
    static const std::vector<MultiVariant> v = [] {
        std::vector<MultiVariant> r;
        register_multi_a(r);
        register_multi_b(r);
        return r;
    }();
    return v;
}

// The kernel of group (n, syn): the one holding the decode table when `lut`
// and one is compiled, else one without a table (nullptr: n has none).
const MultiVariant *multi_for(uint32_t n, int syn, bool lut)
{
    const MultiVariant *plain = nullptr;
    for (const MultiVariant &v : multi_variants()) {
        if (v.n != n || v.syn != syn) continue;
        if (lut && v.lut) return &v;
        if (!v.lut && !plain) plain = &v;
    }
    return plain;
}

// Codewords per item of code n in the stream-group configuration (every
// kernel of one n, with or without a table, uses the same chunk); 0: none.
uint64_t multi_chunk_cw(uint32_t n)
{
    const MultiVariant *v = multi_for(n, 0, false);
    return v ? v->chunk_cw : 0;
}

// Groups of the stream-group configuration: (n, syndrome type) pairs.
constexpr int kMaxGroups = 18;
}  // namespace hd

using namespace hd;

struct hd_plan {
    int device = 0;
    uint32_t num_packets = 0;
    uint32_t num_tiles = 0;
    uint32_t full_tiles = 0;
    uint64_t codewords = 0;
    uint64_t in_bytes = 0, out_bytes = 0, syn_bytes = 0;
    void *dmem = nullptr;
    DevTile *d_tiles = nullptr;
    uint32_t *d_counter = nullptr;
    int variant = 0;
    float tuned_us = -1.f;
    cudaStream_t capture = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long *graph_err = nullptr;
    bool graph_ok = false;
    uint64_t graph_kernels = 0;  // kernels one replay of the graph launches
    // the split configuration: each code group's tile range (tiles are grouped
    // by n in kSplitOrder), a stream per group and the fork/join events
    uint32_t grp_begin[kSplitGroups] = {}, grp_end[kSplitGroups] = {};
    DevTile *d_split = nullptr;  // the split configuration's own tile table (8 KB tiles for the long codes)
    cudaStream_t gstream[kSplitGroups] = {};
    cudaEvent_t fork = nullptr, join[kSplitGroups] = {};
    // the stream-group configuration: one k_decode_multi launch per (n,
    // syndrome type) group over its runs of whole chunks, and one batch-kernel
    // launch over the tiles of the n = 3 packets
    struct Group {
        uint32_t n;
        int syn;
        uint32_t run_begin, num_runs, nitems;
    };
    std::vector<Group> groups;
    bool groups_ok = false;  // the configuration is available for this plan
    MultiRun *d_runs = nullptr;
    DevTile *d_rest = nullptr;
    uint32_t num_rest = 0;
    cudaStream_t mstream[kMaxGroups + 1] = {};  // [0]: the n = 3 tiles; [1 + g]: group g
    cudaEvent_t mjoin[kMaxGroups + 1] = {};
};

namespace {

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Validate the table and build the packet and tile arrays.
hd_status build_tables(const hd_packet *table, uint32_t num_packets, std::vector<DevPacket> &pk,
                       std::vector<DevTile> &tiles, hd_plan *stats, std::vector<DevTile> *split = nullptr)
{
    if (num_packets > 0 && table == nullptr) return HD_ERR_NULL;
    pk.resize(num_packets);
    uint64_t ntiles = 0;
    for (uint32_t i = 0; i < num_packets; ++i) {
        const hd_packet &q = table[i];
        const int m = code_m(q.n);
        if (m == 0) return HD_ERR_INVALID_N;
        if (q.syn_type > 2) return HD_ERR_INVALID_ARG;
        if (q.num_codewords > (1ull << 40)) return HD_ERR_SIZE;
        if (q.num_codewords > 0) {
            if (!q.in || !q.out || (q.syn_type != 0 && !q.syndromes)) return HD_ERR_NULL;
            if (!aligned16(q.in) || !aligned16(q.out) || (q.syn_type != 0 && !aligned16(q.syndromes)))
                return HD_ERR_ALIGN;
        }
        DevPacket &d = pk[i];
        d.in = q.in;
        d.out = q.out;
        d.syn = static_cast<uint8_t *>(q.syndromes);
        d.num_cw = q.num_codewords;
        d.n = q.n;
        d.m = (uint32_t)m;
        d.syn_type = q.syndromes ? q.syn_type : 0;
        d.in_words = words_for_bits(q.num_codewords * q.n);
        d.out_words = words_for_bits(q.num_codewords * (q.n - (uint32_t)m));
        d.pad = 0;
        ntiles += packet_tiles(q.n, q.num_codewords);
        if (stats) {
            stats->codewords += q.num_codewords;
            stats->in_bytes += (q.num_codewords * q.n + 7) / 8;
            stats->out_bytes += (q.num_codewords * (q.n - (uint32_t)m) + 7) / 8;
            stats->syn_bytes += q.num_codewords * (d.syn_type == 2 ? 2 : d.syn_type);
        }
    }
    if (ntiles >= 0xFFFFFFF0ull) return HD_ERR_CAPACITY;
    tiles.clear();
    tiles.reserve(ntiles);
    // tiles grouped by n (long codes first), each code's tails among its full tiles
    uint32_t nfull_tiles = 0;
    for (int gi = 0; gi < kSplitGroups; ++gi) {
        if (stats) stats->grp_begin[gi] = (uint32_t)tiles.size();
        emit_code_tiles(
            kSplitOrder[gi], num_packets,
            [&](uint32_t i) {
                const DevPacket &d = pk[i];
                return PacketView{d.in, d.out, d.syn, d.num_cw, d.n, d.m, d.syn_type};
            },
            [&](const DevTile &t) {
                tiles.push_back(t);
                if (t.count & kFullTile) ++nfull_tiles;
            });
        if (stats) stats->grp_end[gi] = (uint32_t)tiles.size();
    }
    if (stats) stats->full_tiles = nfull_tiles;
    if (split) {
        // the split configuration's table: the same order, the long codes cut
        // with the 8 KB geometry; its group ranges replace the ones above
        split->clear();
        for (int gi = 0; gi < kSplitGroups; ++gi) {
            if (stats) stats->grp_begin[gi] = (uint32_t)split->size();
            emit_code_tiles(
                kSplitOrder[gi], num_packets,
                [&](uint32_t i) {
                    const DevPacket &d = pk[i];
                    return PacketView{d.in, d.out, d.syn, d.num_cw, d.n, d.m, d.syn_type};
                },
                [&](const DevTile &t) { split->push_back(t); }, true);
            if (stats) stats->grp_end[gi] = (uint32_t)split->size();
        }
        if (split->size() >= 0xFFFFFFF0ull) return HD_ERR_CAPACITY;
    }
    return HD_OK;
}

// The stream-group configuration's tables.  For each (n, syndrome type) group
// (long codes first): the packets' whole chunks, in the streaming kernel's
// chunk geometry and in packet order, with the packets' ragged tails spread
// evenly among them (a tail costs more than a chunk -- a plain load of its
// last words, a zero-filled chunk, a word-by-word copy out -- and each warp
// decodes a contiguous range of items, so tails grouped together would load
// a few warps with most of them).  A record describes consecutive chunks of
// one packet up to the next tail, or one tail (kTailItems items: the first
// decodes it, the others are padding).  n = 3 packets (no streaming kernel)
// are cut into batch tiles.  With 2^22 - 1 packets or more (the records'
// packet field) the configuration is not available.
hd_status build_group_tables(const std::vector<DevPacket> &pk, std::vector<MultiRun> &runs,
                             std::vector<DevTile> &rest, std::vector<hd_plan::Group> &groups, bool *available)
{
    const uint32_t np = (uint32_t)pk.size();
    *available = np <= kPacketMask;  // index kPacketMask with the longest tail would read as padding
    if (!*available) return HD_OK;
    for (uint32_t n : kSplitOrder) {
        const uint64_t chunk = multi_chunk_cw(n);
        if (chunk == 0) continue;
        for (int syn = 0; syn <= 2; ++syn) {
            const uint64_t sb = syn == 2 ? 2u : (uint64_t)syn;
            // record of codewords [c0, ...) of packet i; a chunk fills whole 16-byte
            // groups of input, output and syndromes, so every record starts aligned
            auto record = [&](uint32_t i, uint64_t c0, uint32_t c_begin, uint32_t tail) {
                const DevPacket &d = pk[i];
                const uint32_t k = d.n - d.m;
                return MultiRun{d.in + c0 * n / 32u, d.out + c0 * k / 32u, syn != 0 ? d.syn + c0 * sb : nullptr,
                                c_begin, i | tail << kTailShift};
            };
            uint64_t nf = 0, nt = 0;  // whole chunks and tails of the group
            for (uint32_t i = 0; i < np; ++i) {
                const DevPacket &d = pk[i];
                if (d.n != n || (int)d.syn_type != syn) continue;
                nf += d.num_cw / chunk;
                nt += (d.num_cw % chunk) != 0;
            }
            if (nf + nt == 0) continue;
            if (nf + nt * kTailItems >= 0xFFFFFFF0ull) return HD_ERR_CAPACITY;
            hd_plan::Group g{n, syn, (uint32_t)runs.size(), 0u, (uint32_t)(nf + nt * kTailItems)};
            uint64_t items = 0, done_full = 0, done_tail = 0;
            uint32_t tp = 0;  // tail cursor: the next packet whose tail may be due
            auto next_tail = [&]() {
                for (; tp < np; ++tp) {
                    const DevPacket &d = pk[tp];
                    if (d.n != n || (int)d.syn_type != syn || d.num_cw % chunk == 0) continue;
                    runs.push_back(record(tp, d.num_cw / chunk * chunk, (uint32_t)items, (uint32_t)(d.num_cw % chunk)));
                    items += kTailItems;
                    ++done_tail;
                    ++tp;
                    return;
                }
            };
            for (uint32_t i = 0; i < np; ++i) {
                const DevPacket &d = pk[i];
                if (d.n != n || (int)d.syn_type != syn) continue;
                const uint64_t whole = d.num_cw / chunk;
                for (uint64_t j = 0; j < whole;) {
                    // chunks until the next tail is due: the first x >= 1 with
                    // (done_full + x) * nt > done_tail * nf
                    uint64_t x = whole - j;
                    if (done_tail < nt) x = std::min(x, done_tail * nf / nt + 1 - done_full);
                    runs.push_back(record(i, j * chunk, (uint32_t)items, 0u));
                    items += x;
                    done_full += x;
                    j += x;
                    while (done_tail < nt && done_tail * nf < done_full * nt) next_tail();
                }
            }
            while (done_tail < nt) next_tail();
            g.num_runs = (uint32_t)runs.size() - g.run_begin;
            groups.push_back(g);
        }
    }
    emit_code_tiles(
        3, np,
        [&](uint32_t i) {
            const DevPacket &d = pk[i];
            return PacketView{d.in, d.out, d.syn, d.num_cw, d.n, d.m, d.syn_type};
        },
        [&](const DevTile &t) { rest.push_back(t); });
    if (rest.size() >= 0xFFFFFFF0ull) return HD_ERR_CAPACITY;
    return HD_OK;
}

int batch_grid(const BatchVariant &v, uint32_t num_tiles)
{
    const int bps = stream_blocks_per_sm(v.kernel, v.warps * 32, v.smem);
    if (bps <= 0) return -1;
    const uint64_t cap = (uint64_t)num_sms() * (uint64_t)bps;
    const uint64_t want = ((uint64_t)num_tiles + v.warps - 1) / v.warps;
    return decode_grid(want, cap);
}

// Resolve everything that touches device state before a (possibly captured)
// enqueue: kernel attributes, occupancy, the status word address and the
// decode tables (filled on `st` on first use; `st` must not be capturing for
// that, else the n = 7 tiles decode arithmetically and a configuration that
// holds the n = 15 table gives way to the built-in one).
struct LaunchGeom {
    int variant;
    int grid;
    uint32_t *status;
    const uint16_t *lut7, *lut15;
    bool split = false;
    const BatchVariant *gk[kSplitGroups] = {};  // split: the kernel of each code group
    int ggrid[kSplitGroups] = {};
    bool groups = false;                        // the stream-group configuration
    const MultiVariant *mk[kMaxGroups] = {};    // its kernel per group
    int mgrid[kMaxGroups] = {};
    int rest_grid = 0;                          // the batch kernel's grid for the n = 3 tiles
};

// Index of the first split configuration among a plan's configurations
// (after the single-kernel ones), of the stream-group configuration (the
// last), and the number of configurations.
inline int split_variant() { return (int)batch_variants().size(); }
inline int group_variant() { return split_variant() + (int)split_kernels().size(); }
inline int plan_variants() { return group_variant() + 1; }

cudaError_t prepare_plan(hd_plan *p, LaunchGeom *g, cudaStream_t st)
{
    g->status = status_ptr();
    if (g->status == nullptr) return cudaErrorInvalidSymbol;
    g->variant = p->variant;
    g->lut7 = lut_ptr(7, st);
    if (g->variant == group_variant() && !p->groups_ok) g->variant = 0;
    if (g->variant == group_variant()) {
        g->groups = true;
        g->lut15 = lut_ptr(15, st);
        g->grid = 0;
        if (p->num_rest != 0) {
            g->rest_grid = batch_grid(batch_variants()[0], p->num_rest);
            if (g->rest_grid <= 0) return cudaErrorInvalidConfiguration;
            g->grid += g->rest_grid;
        }
        for (size_t gi = 0; gi < p->groups.size(); ++gi) {
            const hd_plan::Group &gr = p->groups[gi];
            const bool lut = (gr.n == 7 && g->lut7 != nullptr) || (gr.n == 15 && g->lut15 != nullptr);
            const MultiVariant *mv = multi_for(gr.n, gr.syn, lut);
            if (mv == nullptr) return cudaErrorInvalidConfiguration;
            const int bps = stream_blocks_per_sm(mv->kernel, mv->T, mv->smem);
            if (bps <= 0) return cudaErrorInvalidConfiguration;
            const uint32_t warps = (uint32_t)mv->T / 32u;
            g->mk[gi] = mv;
            g->mgrid[gi] = decode_grid((gr.nitems + warps - 1) / warps, (uint64_t)num_sms() * (uint64_t)bps);
            g->grid += g->mgrid[gi];
        }
        return cudaSuccess;
    }
    if (g->variant >= split_variant()) {
        g->split = true;
        g->lut15 = lut_ptr(15, st);
        g->grid = 0;
        const SplitKernels &sk = split_kernels()[g->variant - split_variant()];
        for (int gi = 0; gi < kSplitGroups; ++gi) {
            const uint32_t nt = p->grp_end[gi] - p->grp_begin[gi];
            if (nt == 0) continue;
            g->gk[gi] = (kSplitOrder[gi] == 15 && g->lut15 != nullptr) ? &sk.n15_table : &sk.group[gi];
            g->ggrid[gi] = batch_grid(*g->gk[gi], nt);
            if (g->ggrid[gi] <= 0) return cudaErrorInvalidConfiguration;
            g->grid += g->ggrid[gi];
        }
        return cudaSuccess;
    }
    g->lut15 = batch_variants()[g->variant].t15 ? lut_ptr(15, st) : nullptr;
    if (batch_variants()[g->variant].t15 && g->lut15 == nullptr) g->variant = 0;
    g->grid = batch_grid(batch_variants()[g->variant], p->num_tiles);
    return g->grid > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

cudaError_t enqueue_plan(hd_plan *p, const LaunchGeom &g, unsigned long long *err_counts, cudaStream_t st,
                         bool clear = true)
{
    uint32_t *status = g.status;
    cudaError_t e = cudaSuccess;
    if (clear) {
        // one claim counter per code group (the split configuration), else the
        // first, and the error counters: one small kernel, which the single-kernel
        // configurations' decode overlaps (programmatic dependent launch)
        const uint32_t nc = g.split ? kSplitGroups : 1u;
        const uint32_t work = std::max(nc, err_counts ? p->num_packets : 0u);
        const int blocks = (int)std::min<uint32_t>(64u, (work + 255u) / 256u);
        k_clear_plan<<<std::max(blocks, 1), 256, 0, st>>>(p->d_counter, nc, err_counts, p->num_packets);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (p->num_tiles == 0) return cudaSuccess;
    if (g.groups) {
        // the groups, long codes first, and the n = 3 packets' batch kernel,
        // each a branch forked from `st` and joined back into it
        if ((e = cudaEventRecord(p->fork, st)) != cudaSuccess) return e;
        auto join = [&](int b) -> cudaError_t {
            cudaError_t r = cudaGetLastError();
            if (r == cudaSuccess) r = cudaEventRecord(p->mjoin[b], p->mstream[b]);
            if (r == cudaSuccess) r = cudaStreamWaitEvent(st, p->mjoin[b], 0);
            return r;
        };
        if (p->num_rest != 0) {
            if ((e = cudaStreamWaitEvent(p->mstream[0], p->fork, 0)) != cudaSuccess) return e;
            const BatchVariant &v = batch_variants()[0];
            v.launch(g.rest_grid, v.smem, p->mstream[0], p->d_rest, p->num_rest, p->d_counter, err_counts, status,
                     g.lut7, nullptr, false);
            if ((e = join(0)) != cudaSuccess) return e;
        }
        for (size_t gi = 0; gi < p->groups.size(); ++gi) {
            const hd_plan::Group &gr = p->groups[gi];
            const MultiVariant &mv = *g.mk[gi];
            cudaStream_t gs = p->mstream[1 + gi];
            if ((e = cudaStreamWaitEvent(gs, p->fork, 0)) != cudaSuccess) return e;
            MultiArgs a;
            a.runs = p->d_runs + gr.run_begin;
            a.err = err_counts;
            a.status = status;
            a.lut = !mv.lut ? nullptr : (gr.n == 7 ? g.lut7 : g.lut15);
            a.num_runs = gr.num_runs;
            a.nitems = gr.nitems;
            if ((e = mv.launch(g.mgrid[gi], gs, a)) != cudaSuccess) return e;
            if ((e = join(1 + (int)gi)) != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    if (g.split) {
        // the code groups as concurrent branches forked from `st` and joined back into it
        if ((e = cudaEventRecord(p->fork, st)) != cudaSuccess) return e;
        for (int gi = 0; gi < kSplitGroups; ++gi) {
            if (!g.gk[gi]) continue;
            cudaStream_t gs = p->gstream[gi];
            if ((e = cudaStreamWaitEvent(gs, p->fork, 0)) != cudaSuccess) return e;
            const BatchVariant &v = *g.gk[gi];
            v.launch(g.ggrid[gi], v.smem, gs, p->d_split + p->grp_begin[gi], p->grp_end[gi] - p->grp_begin[gi],
                     p->d_counter + gi, err_counts, status, g.lut7, g.lut15, false);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if ((e = cudaEventRecord(p->join[gi], gs)) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(st, p->join[gi], 0)) != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const BatchVariant &v = batch_variants()[g.variant];
    v.launch(g.grid, v.smem, st, p->d_tiles, p->num_tiles, p->d_counter, err_counts, status, g.lut7, g.lut15, clear);
    return cudaGetLastError();
}

// Kernels enqueued by one launch of a prepared plan.
uint64_t plan_kernels(const hd_plan *p, const LaunchGeom &g)
{
    if (p->num_tiles == 0) return 1;  // the counters' clear
    if (g.groups) return 1 + (p->num_rest != 0 ? 1u : 0u) + (uint64_t)p->groups.size();
    if (!g.split) return 2;
    uint64_t c = 1;
    for (int gi = 0; gi < kSplitGroups; ++gi) c += g.gk[gi] != nullptr;
    return c;
}

void drop_graph(hd_plan *p)
{
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->exec = nullptr;
    p->graph = nullptr;
    p->graph_ok = false;
}

}  // namespace

namespace hd {

hd_status build_tile_table(const hd_packet *table, uint32_t num_packets, std::vector<DevTile> &tiles,
                           uint64_t *bytes)
{
    std::vector<DevPacket> pk;
    hd_plan stats;
    const hd_status rc = build_tables(table, num_packets, pk, tiles, &stats);
    if (rc == HD_OK && bytes) *bytes += stats.in_bytes + stats.out_bytes + stats.syn_bytes;
    return rc;
}

cudaError_t launch_tile_table(const DevTile *d_tiles, uint32_t num_tiles, uint32_t *d_counter,
                              unsigned long long *d_err, uint32_t num_packets, cudaStream_t st, uint32_t *status,
                              bool clear)
{
    hd_plan p;
    p.num_packets = num_packets;
    p.num_tiles = num_tiles;
    p.d_tiles = const_cast<DevTile *>(d_tiles);
    p.d_counter = d_counter;
    LaunchGeom geom;
    cudaError_t e = prepare_plan(&p, &geom, st);
    if (status != nullptr) geom.status = status;
    if (e == cudaSuccess) e = enqueue_plan(&p, geom, d_err, st, clear);
    if (e == cudaSuccess && num_tiles) count_launch();
    return e;
}

}  // namespace hd

extern "C" {

hd_status hd_plan_create(const hd_packet *table, uint32_t num_packets, hd_plan **out)
{
    if (!out) return HD_ERR_NULL;
    *out = nullptr;
    hd_plan *p = new (std::nothrow) hd_plan();
    if (!p) return HD_ERR_CAPACITY;
    std::vector<DevPacket> pk;
    std::vector<DevTile> tiles, split, rest;
    std::vector<MultiRun> runs;
    hd_status rc = build_tables(table, num_packets, pk, tiles, p, &split);
    if (rc == HD_OK) rc = build_group_tables(pk, runs, rest, p->groups, &p->groups_ok);
    if (rc != HD_OK) {
        delete p;
        return rc;
    }
    cudaGetDevice(&p->device);
    p->num_packets = num_packets;
    p->num_tiles = (uint32_t)tiles.size();
    p->num_rest = (uint32_t)rest.size();
    auto rounded = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t tl_b = rounded(tiles.size() * sizeof(DevTile)), sp_b = rounded(split.size() * sizeof(DevTile));
    const size_t ru_b = rounded(runs.size() * sizeof(MultiRun)), re_b = rounded(rest.size() * sizeof(DevTile));
    if (cudaMalloc(&p->dmem, tl_b + 256 + sp_b + ru_b + re_b) != cudaSuccess) {
        delete p;
        return HD_ERR_CUDA;
    }
    char *base = static_cast<char *>(p->dmem);
    p->d_tiles = reinterpret_cast<DevTile *>(base);
    p->d_counter = reinterpret_cast<uint32_t *>(base + tl_b);
    p->d_split = reinterpret_cast<DevTile *>(base + tl_b + 256);
    p->d_runs = reinterpret_cast<MultiRun *>(base + tl_b + 256 + sp_b);
    p->d_rest = reinterpret_cast<DevTile *>(base + tl_b + 256 + sp_b + ru_b);
    auto upload = [](void *dst, const void *src, size_t bytes) {
        return bytes == 0 || cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    bool ok = upload(p->d_tiles, tiles.data(), tiles.size() * sizeof(DevTile)) &&
              upload(p->d_split, split.data(), split.size() * sizeof(DevTile)) &&
              upload(p->d_runs, runs.data(), runs.size() * sizeof(MultiRun)) &&
              upload(p->d_rest, rest.data(), rest.size() * sizeof(DevTile)) &&
              cudaStreamCreateWithFlags(&p->capture, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int gi = 0; ok && gi < kSplitGroups; ++gi)
        ok = cudaStreamCreateWithFlags(&p->gstream[gi], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&p->join[gi], cudaEventDisableTiming) == cudaSuccess;
    for (size_t b = 0; ok && b <= p->groups.size(); ++b)
        ok = cudaStreamCreateWithFlags(&p->mstream[b], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&p->mjoin[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        hd_plan_destroy(p);
        return HD_ERR_CUDA;
    }
    *out = p;
    return HD_OK;
}

hd_status hd_plan_launch(hd_plan *p, unsigned long long *err_counts, void *cuda_stream)
{
    if (!p) return HD_ERR_NULL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (!p->graph_ok || p->graph_err != err_counts) {
        drop_graph(p);
        LaunchGeom geom;
        if (prepare_plan(p, &geom, st) != cudaSuccess) return HD_ERR_CUDA;
        if (cudaStreamBeginCapture(p->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return HD_ERR_CUDA;
        const cudaError_t e = enqueue_plan(p, geom, err_counts, p->capture);
        g_launches.fetch_sub(1, std::memory_order_relaxed);  // the clear recorded here runs (and counts) per replay
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(p->capture, &g);
        if (e != cudaSuccess || e2 != cudaSuccess || g == nullptr) {
            if (g) cudaGraphDestroy(g);
            return HD_ERR_CUDA;
        }
        p->graph = g;
        if (cudaGraphInstantiate(&p->exec, g, 0) != cudaSuccess) {
            drop_graph(p);
            return HD_ERR_CUDA;
        }
        p->graph_err = err_counts;
        p->graph_ok = true;
        p->graph_kernels = plan_kernels(p, geom);
    }
    if (cudaGraphLaunch(p->exec, st) != cudaSuccess) return HD_ERR_CUDA;
    count_launch(p->graph_kernels);
    return HD_OK;
}

hd_status hd_plan_autotune(hd_plan *p, uint32_t reps, void *cuda_stream, hd_plan_info *chosen)
{
    if (!p) return HD_ERR_NULL;
    if (reps == 0) reps = 3;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return HD_ERR_CUDA;
    int best = -1;
    float best_us = 0.f;
    const int keep = p->variant;
    hd_status rc = HD_OK;
    // every configuration timed as hd_plan_launch runs it: recorded as a CUDA
    // graph, then replayed (err_counts NULL: the counts are not part of the choice)
    for (int i = 0; i < plan_variants(); ++i) {
        p->variant = i;
        LaunchGeom geom;
        if (prepare_plan(p, &geom, st) != cudaSuccess || geom.variant != i) continue;
        drop_graph(p);
        if ((rc = hd_plan_launch(p, nullptr, st)) != HD_OK) break;  // records the graph and runs it once
        cudaEventRecord(e0, st);
        for (uint32_t r = 0; r < reps; ++r)
            if ((rc = hd_plan_launch(p, nullptr, st)) != HD_OK) break;
        cudaEventRecord(e1, st);
        if (rc != HD_OK || cudaEventSynchronize(e1) != cudaSuccess) {
            if (rc == HD_OK) rc = HD_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const float us = ms * 1000.f / (float)reps;
        if (best < 0 || us < best_us) {
            best = i;
            best_us = us;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->variant = best >= 0 ? best : keep;
    p->tuned_us = best >= 0 ? best_us : -1.f;
    drop_graph(p);
    if (rc != HD_OK) return rc;
    if (chosen) return hd_plan_get_info(p, chosen);
    return HD_OK;
}

hd_status hd_plan_get_info(const hd_plan *p, hd_plan_info *info)
{
    if (!p || !info) return HD_ERR_NULL;
    std::memset(info, 0, sizeof(*info));
    const bool groups = p->variant == group_variant();
    const bool split = p->variant >= split_variant() && !groups;
    const BatchVariant &v = split ? split_kernels()[p->variant - split_variant()].group[0]
                                  : batch_variants()[groups ? 0 : p->variant];
    info->num_packets = p->num_packets;
    info->num_tiles = p->num_tiles;
    info->full_tiles = p->full_tiles;
    info->codewords = p->codewords;
    info->in_bytes = p->in_bytes;
    info->out_bytes = p->out_bytes;
    info->syn_bytes = p->syn_bytes;
    info->warps_per_cta = (uint32_t)v.warps;
    info->stages = (uint32_t)v.stages;
    info->smem_bytes = v.smem;
    if (groups && !p->groups.empty()) {
        // the kernel of the first group (the longest code present)
        const MultiVariant *mv = multi_for(p->groups[0].n, p->groups[0].syn, false);
        if (mv) {
            info->warps_per_cta = (uint32_t)mv->T / 32u;
            info->stages = (uint32_t)mv->S;
            info->smem_bytes = mv->smem;
        }
    }
    info->variant = (uint32_t)p->variant;
    info->num_variants = (uint32_t)plan_variants();
    info->measured_us = p->tuned_us;
    info->table_lookup = 1u | (v.t15 || split || groups ? 2u : 0u);
    return HD_OK;
}

hd_status hd_plan_select(hd_plan *p, uint32_t variant)
{
    if (!p) return HD_ERR_NULL;
    if (variant >= (uint32_t)plan_variants()) return HD_ERR_INVALID_ARG;
    p->variant = (int)variant;
    drop_graph(p);
    return HD_OK;
}

void hd_plan_destroy(hd_plan *p)
{
    if (!p) return;
    drop_graph(p);
    if (p->capture) cudaStreamDestroy(p->capture);
    for (int gi = 0; gi < kSplitGroups; ++gi) {
        if (p->gstream[gi]) cudaStreamDestroy(p->gstream[gi]);
        if (p->join[gi]) cudaEventDestroy(p->join[gi]);
    }
    for (int b = 0; b <= kMaxGroups; ++b) {
        if (p->mstream[b]) cudaStreamDestroy(p->mstream[b]);
        if (p->mjoin[b]) cudaEventDestroy(p->mjoin[b]);
    }
    if (p->fork) cudaEventDestroy(p->fork);
    if (p->dmem) cudaFree(p->dmem);
    delete p;
}

hd_status hd_decode_batch(const hd_packet *table, uint32_t num_packets, unsigned long long *err_counts,
                          void *cuda_stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    std::vector<DevPacket> pk;
    std::vector<DevTile> tiles;
    hd_plan p;
    hd_status rc = build_tables(table, num_packets, pk, tiles, &p);
    if (rc != HD_OK) return rc;
    p.num_packets = num_packets;
    p.num_tiles = (uint32_t)tiles.size();
    const size_t tl_b = (tiles.size() * sizeof(DevTile) + 255) / 256 * 256;
    // stream-ordered scratch: freed on the stream once the kernel has run
    if (cudaMallocAsync(&p.dmem, tl_b + 256, st) != cudaSuccess) return HD_ERR_CUDA;
    p.d_tiles = static_cast<DevTile *>(p.dmem);
    p.d_counter = reinterpret_cast<uint32_t *>(static_cast<char *>(p.dmem) + tl_b);
    // pageable source: the copy has read the host vector when this call returns
    if (!tiles.empty() && cudaMemcpyAsync(p.d_tiles, tiles.data(), tiles.size() * sizeof(DevTile),
                                          cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaFreeAsync(p.dmem, st);
        return HD_ERR_CUDA;
    }
    LaunchGeom geom;
    cudaError_t e = prepare_plan(&p, &geom, st);
    if (e == cudaSuccess) e = enqueue_plan(&p, geom, err_counts, st);
    if (p.num_tiles && e == cudaSuccess) count_launch();
    cudaFreeAsync(p.dmem, st);
    p.dmem = nullptr;
    return e == cudaSuccess ? HD_OK : HD_ERR_CUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched decode without allocation.
//
// For callers that must not allocate device memory -- a process that budgets
// every byte of device memory up front, an application whose allocator hooks
// forbid allocations from inside libraries, or a latency-critical receive
// path where an allocation could stall or fail -- the tile table and the
// claim counter of the batched decoder live in one fixed array
// compiled into this library.  The array is kNoAllocBytes (1 MiB) on every
// device that loads the library and stays there until the process exits.
// ---------------------------------------------------------------------------
namespace hd {
namespace {

constexpr uint32_t kNoAllocBytes = 1u << 20;
constexpr uint32_t kNoAllocMaxPackets = 4096;
constexpr uint32_t kNoAllocTilesOff = 256;  // the claim counter sits at offset 0
constexpr uint32_t kNoAllocMaxTiles = (kNoAllocBytes - kNoAllocTilesOff) / sizeof(DevTile);
static_assert(sizeof(DevTile) == 64, "table layout");

// The device scratch.  In host code this name is only a handle for
// cudaGetSymbolAddress; kernels receive the device address it returns.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// The tile table reaches the array through kernel parameters: each upload
// launch carries up to kUploadTiles descriptors by value (within the 32 KB
// parameter limit), so no host staging and no host-to-device copy is needed.
constexpr uint32_t kUploadTiles = 480;
struct TileUpload {
    DevTile tiles[kUploadTiles];
    uint32_t first;  // index of tiles[0] in the table
    uint32_t count;
};
static_assert(sizeof(TileUpload) <= 32000, "kernel parameter space");

__global__ void k_upload_tiles(const __grid_constant__ TileUpload u, DevTile *__restrict__ table)
{
    for (uint32_t i = threadIdx.x; i < u.count; i += blockDim.x) table[u.first + i] = u.tiles[i];
}

std::mutex g_noalloc_mu;  // serialises host threads (the device array is shared)
constexpr int kNoAllocMaxDevices = 64;
unsigned char *g_noalloc_dev[kNoAllocMaxDevices];  // device address of the scratch, per device
uint32_t *g_noalloc_status[kNoAllocMaxDevices];

// One-time set-up on the current device: the scratch array's device address,
// the status word and the kernel's launch attributes.
hd_status noalloc_setup(int dev)
{
    if (dev < 0 || dev >= kNoAllocMaxDevices) return HD_ERR_CAPACITY;
    if (g_noalloc_dev[dev] != nullptr) return HD_OK;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return HD_ERR_CUDA;
    uint32_t *status = status_ptr();
    if (status == nullptr) return HD_ERR_CUDA;
    const BatchVariant &v = batch_variants()[0];
    if (stream_blocks_per_sm(v.kernel, v.warps * 32, v.smem) <= 0) return HD_ERR_CUDA;
    g_noalloc_status[dev] = status;
    g_noalloc_dev[dev] = static_cast<unsigned char *>(p);
    return HD_OK;
}

}  // namespace
}  // namespace hd

extern "C" hd_status hd_batch_tiles(const hd_packet *table, uint32_t num_packets, uint64_t *tiles)
{
    if (tiles == nullptr || (num_packets > 0 && table == nullptr)) return HD_ERR_NULL;
    uint64_t t = 0;
    for (uint32_t i = 0; i < num_packets; ++i) {
        const hd_packet &q = table[i];
        if (code_m(q.n) == 0) return HD_ERR_INVALID_N;
        if (q.syn_type > 2) return HD_ERR_INVALID_ARG;
        if (q.num_codewords > (1ull << 40)) return HD_ERR_SIZE;
        t += packet_tiles(q.n, q.num_codewords);
    }
    *tiles = t;
    return HD_OK;
}

extern "C" hd_status hd_decode_batch_noalloc(const hd_packet *table, uint32_t num_packets,
                                             unsigned long long *err_counts, void *cuda_stream)
{
    if (num_packets > 0 && table == nullptr) return HD_ERR_NULL;
    if (num_packets > kNoAllocMaxPackets) return HD_ERR_CAPACITY;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HD_ERR_CUDA;
    // validate and count tiles before touching anything
    uint64_t ntiles = 0;
    for (uint32_t i = 0; i < num_packets; ++i) {
        const hd_packet &q = table[i];
        const int m = code_m(q.n);
        if (m == 0) return HD_ERR_INVALID_N;
        if (q.syn_type > 2) return HD_ERR_INVALID_ARG;
        if (q.num_codewords > (1ull << 40)) return HD_ERR_SIZE;
        if (q.num_codewords > 0) {
            if (!q.in || !q.out || (q.syn_type != 0 && !q.syndromes)) return HD_ERR_NULL;
            if (!aligned16(q.in) || !aligned16(q.out) || (q.syn_type != 0 && !aligned16(q.syndromes)))
                return HD_ERR_ALIGN;
        }
        ntiles += packet_tiles(q.n, q.num_codewords);
    }
    if (ntiles > kNoAllocMaxTiles) return HD_ERR_CAPACITY;
    const hd_status su = noalloc_setup(dev);
    if (su != HD_OK) return su;
    unsigned char *dbase = g_noalloc_dev[dev];
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    // the claim counter must start at zero; the error counters are overwritten
    uint32_t *counter = reinterpret_cast<uint32_t *>(dbase);
    DevTile *dtab = reinterpret_cast<DevTile *>(dbase + kNoAllocTilesOff);
    if (cudaMemsetAsync(counter, 0, sizeof(uint32_t), st) != cudaSuccess) return HD_ERR_CUDA;
    if (err_counts && num_packets &&
        cudaMemsetAsync(err_counts, 0, sizeof(unsigned long long) * num_packets, st) != cudaSuccess)
        return HD_ERR_CUDA;
    // tiles grouped by n (long codes first), each code's tails among its full
    // tiles, uploaded kUploadTiles at a time by kernels that carry them
    static TileUpload up;  // 30 KB, off the thread's stack; guarded by g_noalloc_mu
    up.first = 0;
    up.count = 0;
    uint32_t t = 0;
    bool ok = true;
    auto flush = [&]() {
        if (up.count == 0 || !ok) return;
        k_upload_tiles<<<1, 128, 0, st>>>(up, dtab);
        count_launch();
        ok = cudaGetLastError() == cudaSuccess;
        up.first += up.count;
        up.count = 0;
    };
    static const uint32_t order[] = {255, 127, 63, 31, 15, 7, 3};
    for (uint32_t n : order)
        emit_code_tiles(
            n, num_packets,
            [&](uint32_t i) {
                const hd_packet &q = table[i];
                return PacketView{q.in, q.out, static_cast<uint8_t *>(q.syndromes), q.num_codewords, q.n,
                                  (uint32_t)code_m(q.n), q.syndromes ? q.syn_type : 0u};
            },
            [&](const DevTile &tile) {
                up.tiles[up.count++] = tile;
                ++t;
                if (up.count == kUploadTiles) flush();
            });
    flush();
    if (!ok) return HD_ERR_CUDA;
    if (t == 0) return HD_OK;
    const BatchVariant &v = batch_variants()[0];
    const int grid = batch_grid(v, t);
    if (grid <= 0) return HD_ERR_CUDA;
    // no decode tables: this path never fills or synchronises anything
    v.launch(grid, v.smem, st, dtab, t, counter, err_counts, g_noalloc_status[dev], nullptr, nullptr, false);
    if (cudaGetLastError() != cudaSuccess) return HD_ERR_CUDA;
    count_launch();
    return HD_OK;
}
