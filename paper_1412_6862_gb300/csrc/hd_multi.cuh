// hd_multi.cuh -- the streaming decoder run over many packets of one code
// length (the batched decoder's stream-group configuration).
//
// Every packet of one (n, syndrome type) group becomes items of one sequence:
// its whole chunks (32*G codewords each), in packet order, and its ragged
// tail, if any, as one more item, the tails spread evenly among the chunks
// (the plan builds the records).  Each warp of a persistent grid
// decodes one contiguous, equal share of that sequence through the same
// per-warp bulk-copy ring, chunk decoder and bulk stores as the single-stream
// kernel (hd_stream.cuh), in the single-stream kernel's chunk geometry.  The
// per-item additions are small: finding the item's record, a window of 32
// consecutive records held one per lane in registers (a ballot over their
// first items, then shuffles; the window moves on only after 31 records, and
// an item of the record in hand needs no lookup at all); and a 32-byte slot
// per stage with the item's output and syndrome addresses and packet, written
// before the stage's load is announced.  A tail is bulk-copied up to its last
// whole 16-byte group, completed by 4-byte asynchronous copies that the
// stage's barrier also awaits, zero-padded to a chunk,
// decoded by the same chunk decoder and copied out word by word (its
// syndromes through a small per-warp buffer).  Nonzero-syndrome counts
// accumulate per lane and go to a packet's counter when the warp moves on to
// the next packet.
#pragma once

#include <cstdint>
#include <vector>

#include "hd_stream.cuh"

namespace hd {

// One packet's whole chunks (items c_begin .. the next record's c_begin - 1
// are its chunks 0, 1, ...), or one packet's ragged tail (its first item, of
// `count` codewords, 0 < count < 32*G; the record's further items are
// padding, which weighs a tail against the chunks of a warp's share).
struct MultiRun {
    const uint32_t *in;  // chunk 0's (or the tail's) input, 16-byte aligned
    uint32_t *out;       // its output words
    uint8_t *syn;        // its syndromes (unused when the group has none)
    uint32_t c_begin;    // the group's item index of chunk 0 (or of the tail)
    uint32_t info;       // packet index | count << kTailShift (count 0: whole chunks)
};
static_assert(sizeof(MultiRun) == 32, "two 16-byte loads per record");
constexpr uint32_t kTailShift = 22;  // packets of a stream-group plan: fewer than 2^22 - 1
constexpr uint32_t kPacketMask = (1u << kTailShift) - 1u;  // packet kPacketMask is never used
constexpr uint32_t kTailItems = 2;  // items a tail weighs (measured: a tail costs about two chunks)

struct MultiArgs {
    const MultiRun *runs;      // the group's records in item order
    unsigned long long *err;   // per packet, or NULL
    uint32_t *status;          // HD_ERR_TIMEOUT is latched here
    const uint16_t *lut;       // decode table (table configurations only)
    uint32_t num_runs;
    uint32_t nitems;           // items of the group (< 0xFFFFFFFF)
};

// Per-warp layout: S mbarriers, S 32-byte stage slots (output and syndrome
// addresses, packet, tail count), S input stages, (unless INPLACE) two
// output staging buffers and (with syndromes) a tail's syndrome buffer; the
// decode table and its mbarrier behind the warps.
template <int N_, int SYN, int T, int S, int G, int INPLACE, bool LUT>
struct MultiCfg {
    using Q = ChunkGeom<N_, SYN, G, false>;
    static constexpr int WARPS = T / 32;
    static constexpr uint32_t stage_bytes = Q::in_bytes + 16;  // one spare 16-byte group for the funnel read
    static constexpr uint32_t out_buf_bytes = Q::out_bytes + 16;
    static constexpr uint32_t off_bar = 0;
    static constexpr uint32_t off_meta = 64;
    static constexpr uint32_t off_in = off_meta + 32 * S;
    static constexpr uint32_t off_out = off_in + S * stage_bytes;
    static constexpr uint32_t off_syn = off_out + (INPLACE ? 0 : 2 * out_buf_bytes);
    static constexpr uint32_t syn_stage_bytes = SYN != 0 ? (Q::syn_bytes + 15) / 16 * 16 : 0u;
    static constexpr uint32_t warp_bytes = (off_syn + syn_stage_bytes + 127) / 128 * 128;
    static constexpr uint32_t lut_bytes = LUT ? (2u << N_) : 0u;
    static constexpr uint32_t off_lut = WARPS * warp_bytes;
    static constexpr uint32_t smem = off_lut + (LUT ? lut_bytes + 16u : 0u);
    static constexpr bool fits = smem <= 232448;
    static constexpr uint32_t chunk_cw = 32u * G;
    static_assert(T % 32 == 0 && S >= 1 && S <= 8, "whole warps, at most 8 stages");
    static_assert(!INPLACE || S >= 2, "in-place refills lag one iteration");
    static_assert(!INPLACE || Q::out_bytes + 16 <= stage_bytes, "in-place output fits the input stage");
    static_assert(off_in % 16 == 0 && stage_bytes % 16 == 0 && out_buf_bytes % 16 == 0, "bulk copy alignment");
    static_assert(!LUT || N_ == 7 || N_ == 15, "decode tables exist for n = 7 and 15");
    static_assert(chunk_cw <= (1u << (32 - kTailShift)), "a tail's count fits its field");
    static_assert(Q::ALIGNED || Q::GK % 8 == 0, "a part's unaligned output ends are written bytewise: whole bytes");
};

// A 4-byte asynchronous copy into shared memory, and an arrive on `bar` once
// every such copy this thread has issued is complete (the arrival it adds is
// expected too, so the barrier's phase waits for the copies).
__device__ __forceinline__ void cp_async4(void *dst_smem, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst_smem)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_arrive(uint64_t *bar)
{
    asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ uint64_t shfl_u64(uint64_t v, int src)
{
    const uint32_t lo = __shfl_sync(0xFFFFFFFFu, (uint32_t)v, src);
    const uint32_t hi = __shfl_sync(0xFFFFFFFFu, (uint32_t)(v >> 32), src);
    return (uint64_t)hi << 32 | lo;
}


template <int N_, int SYN, int T, int S, int G, int INPLACE, bool LUT>
__global__ void __launch_bounds__(T) k_decode_multi(const MultiArgs a)
{
    using Cfg = MultiCfg<N_, SYN, T, S, G, INPLACE, LUT>;
    using Q = typename Cfg::Q;
    constexpr uint32_t FULL = 0xFFFFFFFFu;
    extern __shared__ __align__(128) uint8_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    grid_dep_launch_dependents();
    uint64_t *lut_bar = nullptr;
    if constexpr (LUT) {
        // the decode table: bulk copies into shared memory behind the warps'
        // areas, in flight while the warps find their first records
        lut_bar = reinterpret_cast<uint64_t *>(smem + Cfg::off_lut + Cfg::lut_bytes);
        if (threadIdx.x == 0) {
            mbar_init(lut_bar, 1);
            fence_mbar_init();
            mbar_arrive_expect_tx(lut_bar, Cfg::lut_bytes);
            constexpr uint32_t piece = Cfg::lut_bytes < 16384u ? Cfg::lut_bytes : 16384u;
            static_assert(Cfg::lut_bytes % piece == 0, "whole pieces");
#pragma unroll
            for (uint32_t o = 0; o < Cfg::lut_bytes; o += piece)
                bulk_g2s(smem + Cfg::off_lut + o, reinterpret_cast<const uint8_t *>(a.lut) + o, piece, lut_bar);
        }
        __syncthreads();  // the barrier is initialised before any thread waits on it
    }
    uint8_t *wbase = smem + warp * Cfg::warp_bytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(wbase + Cfg::off_bar);
    uint4 *meta = reinterpret_cast<uint4 *>(wbase + Cfg::off_meta);  // slot s: meta[2s], meta[2s + 1]
    uint8_t *s_in = wbase + Cfg::off_in;
    uint8_t *s_out = wbase + Cfg::off_out;
    uint8_t *s_syn = wbase + Cfg::off_syn;
    const uint64_t gw = (uint64_t)blockIdx.x * Cfg::WARPS + warp, tw = (uint64_t)gridDim.x * Cfg::WARPS;
    // this warp's items: an equal share of the sequence, in one piece
    const uint32_t lo = (uint32_t)(gw * a.nitems / tw), hi = (uint32_t)((gw + 1) * a.nitems / tw);
    grid_dep_wait();  // the kernels ahead (the counters' clear) have finished

    // the record holding item lo: a 32-way search over the records' first
    // items (runs[left].c_begin <= lo throughout; three steps for 32768 records)
    uint32_t left = 0, right = a.num_runs;
    if (lo < hi) {
        while (right - left > 1) {
            const uint32_t step = (right - left + 31) / 32;
            const uint32_t idx = left + (uint32_t)lane * step;
            const bool le = idx < right && __ldg(&a.runs[idx].c_begin) <= lo;
            const uint32_t mask = __ballot_sync(FULL, le);  // bit 0 is set: idx = left
            left += (uint32_t)(31 - __clz(mask | 1u)) * step;
            right = min(right, left + step);
        }
    }
    // the window: lane l holds record wb + l (a first item of 0xFFFFFFFF past the last record)
    uint32_t wb = left;
    uint64_t w_in = 0, w_out = 0, w_syn = 0;
    uint32_t w_cb = FULL, w_info = 0;
    auto load_window = [&]() {
        const uint32_t r = wb + (uint32_t)lane;
        w_cb = FULL;
        if (r < a.num_runs) {
            const uint4 *rp = reinterpret_cast<const uint4 *>(a.runs + r);
            const uint4 x = __ldg(rp), y = __ldg(rp + 1);
            w_in = (uint64_t)x.y << 32 | x.x;
            w_out = (uint64_t)x.w << 32 | x.z;
            w_syn = (uint64_t)y.y << 32 | y.x;
            w_cb = y.z;
            w_info = y.w;
        }
    };
    if (lo < hi) load_window();

    // The record in hand (items r_cb .. r_end - 1), the same in every lane.
    // Item c (asked for in increasing order) into stage s: a new record is the
    // last one of the window that starts at or before c; when that is the
    // window's last lane, a later record may start before c too, so the window
    // moves on.
    uint64_t r_in = 0, r_out = 0, r_syn = 0;
    uint32_t r_cb = 0, r_info = 0, r_end = 0;
    auto issue = [&](uint32_t c, int s) {
        if (c >= r_end) {
            int j;
            for (;;) {
                const uint32_t mask = __ballot_sync(FULL, w_cb <= c);
                j = 31 - __clz(mask | 1u);
                if (j < 31 || wb + 32 >= a.num_runs) break;
                wb += 31;
                load_window();
            }
            r_cb = __shfl_sync(FULL, w_cb, j);
            r_info = __shfl_sync(FULL, w_info, j);
            const uint32_t next = __shfl_sync(FULL, w_cb, j < 31 ? j + 1 : 31);
            r_end = j < 31 ? next : FULL;
            r_in = shfl_u64(w_in, j);
            r_out = shfl_u64(w_out, j);
            r_syn = shfl_u64(w_syn, j);
        }
        if (lane == 0) {
            const uint32_t cnt = r_info >> kTailShift;
            const uint64_t local = c - r_cb;  // 0 for a tail, > 0 for its padding
            if (cnt != 0 && local != 0) {
                // a tail's padding item (a tail weighs kTailItems items, so that a
                // warp's share holds fewer chunks when it holds a tail): nothing to load
                meta[2 * s + 1] = make_uint4(FULL, 0u, 0u, 0u);
                mbar_arrive(&bar[s]);
                return;
            }
            const uint64_t src = r_in + local * Q::in_bytes, o = r_out + local * Q::out_bytes;
            const uint64_t y = SYN != 0 ? r_syn + local * Q::syn_bytes : 0ull;
            meta[2 * s] = make_uint4((uint32_t)o, (uint32_t)(o >> 32), (uint32_t)y, (uint32_t)(y >> 32));
            meta[2 * s + 1] = make_uint4(r_info, 0u, 0u, 0u);
            // a chunk whole; a tail's whole 16-byte groups by the bulk copy, its last
            // (at most three) words by 4-byte copies that the stage's barrier also awaits
            uint32_t bytes = Q::in_bytes;
            if (cnt != 0) {
                const uint32_t iw = (cnt * (uint32_t)N_ + 31u) / 32u;
                bytes = (iw * 4u) & ~15u;
                if (bytes / 4u < iw) {
                    for (uint32_t w = bytes / 4u; w < iw; ++w)
                        cp_async4(s_in + s * Cfg::stage_bytes + 4u * w, reinterpret_cast<const uint32_t *>(src) + w);
                    cp_async_arrive(&bar[s]);
                }
            }
            // the slot's stores come before the arrive, which the consumers' wait acquires
            if (bytes != 0) {
                mbar_arrive_expect_tx(&bar[s], bytes);
                bulk_g2s(s_in + s * Cfg::stage_bytes, reinterpret_cast<const void *>(src), bytes, &bar[s]);
            } else {
                mbar_arrive(&bar[s]);
            }
        }
    };

    if (lo < hi) {
        if (lane == 0) {
#pragma unroll
            for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
            fence_mbar_init();
        }
        __syncwarp();
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (lo + (uint32_t)s < hi) issue(lo + (uint32_t)s, s);
    }

    // nonzero syndromes of the packet in hand, per lane; added to its counter
    // when the warp moves on to another packet, and at the end
    unsigned long long acc = 0;
    uint32_t cur_pk = FULL;
    auto flush = [&]() {
        unsigned long long e = acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(FULL, e, o);
        if (lane == 0 && e != 0 && a.err != nullptr) atomicAdd(&a.err[cur_pk], e);
        acc = 0;
    };

    uint32_t it = 0;
    bool aborted = false;
    const uint16_t *s_lut = nullptr;
    if constexpr (LUT) {
        const bool ok = mbar_wait_bounded(lut_bar, 0);
        aborted = __any_sync(FULL, !ok);
        s_lut = reinterpret_cast<const uint16_t *>(smem + Cfg::off_lut);
    }
    for (uint32_t c = lo; !aborted && c < hi; ++c, ++it) {
        const int s = (int)(it % S);
        const bool ok = mbar_wait_bounded(&bar[s], (it / S) & 1u);
        if (__any_sync(FULL, !ok)) {
            aborted = true;
            break;
        }
        if constexpr (!INPLACE) {
            if (lane == 0) bulk_wait_read<1>();  // staging buffer it & 1 no longer read by the store of it - 2
            __syncwarp();
        }
        const uint4 m0 = meta[2 * s], m1 = meta[2 * s + 1];
        const bool pad = m1.x == FULL;  // a tail's padding item: the same in every lane
        const uint32_t pk = m1.x & kPacketMask, cnt = pad ? 0u : m1.x >> kTailShift;
        uint32_t *stage = reinterpret_cast<uint32_t *>(s_in + s * Cfg::stage_bytes);
        uint32_t *obase = INPLACE ? stage : reinterpret_cast<uint32_t *>(s_out + (it & 1u) * Cfg::out_buf_bytes);
        uint32_t *gout = reinterpret_cast<uint32_t *>((uint64_t)m0.y << 32 | m0.x);
        uint8_t *gsyn = reinterpret_cast<uint8_t *>((uint64_t)m0.w << 32 | m0.z);
        // a tail's output and syndromes: whole 16-byte groups by bulk stores below
        const uint32_t ob = (cnt * (uint32_t)Code<N_>::k + 31u) / 32u * 4u, yb = cnt * (uint32_t)Q::SB;
        if (!pad) {
            if (pk != cur_pk) {
                if (cur_pk != FULL) flush();
                cur_pk = pk;
            }
            uint32_t unused = 0;
            // A whole chunk's syndromes go straight to global memory (each lane's run
            // of G is contiguous).  A tail of cnt codewords (all iw of its input words
            // are in the stage) drops its input pad bits and zero-fills the chunk (zero
            // codewords decode to zero data and syndromes); its syndromes go to the
            // warp's buffer, and only its own words and syndromes are stored.  Both
            // decode through one call, so that the kernel holds one copy of the chunk
            // decoder (two measured instruction-cache misses as the top stall).
            if (cnt != 0) {
                const uint32_t bits = cnt * (uint32_t)N_, iw = (bits + 31u) / 32u, tail_bits = bits & 31u;
                for (uint32_t w = iw + (uint32_t)lane; w < Q::in_words + 4u; w += 32u) stage[w] = 0u;
                if (lane == 0 && tail_bits != 0u) stage[iw - 1u] &= (1u << tail_bits) - 1u;
                if constexpr (SYN != 0) {
                    if (lane == 0) bulk_wait_read<0>();  // an earlier tail's store has read the buffer
                }
                __syncwarp();
            }
            uint8_t *sdst = SYN == 0 ? s_in : (cnt == 0 ? gsyn : s_syn);
            acc += decode_warp_chunk<N_, SYN, G, false, LUT>(stage, obase, sdst, lane, unused, s_lut);
            if (cnt != 0) {
                // the last (at most three) words and (fewer than 16) syndrome bytes
                __syncwarp();
                const uint32_t w = (ob & ~15u) / 4u + (uint32_t)lane;
                if (w < ob / 4u) gout[w] = obase[w];
                if constexpr (SYN != 0) {
                    const uint32_t b = (yb & ~15u) + (uint32_t)lane;
                    if (b < yb) gsyn[b] = s_syn[b];
                }
            }
        }
        // the decode wrote the stage through the generic proxy; the bulk stores
        // and the refill access it through the async one
        fence_proxy_async_smem();
        __syncwarp();
        if constexpr (INPLACE) {
            // the store issued last iteration has finished reading its stage: refill that
            // stage with the item S - 1 after this one (in place, the lookahead is S - 1)
            if (lane == 0) bulk_wait_read<0>();
            if (it > 0 && c - 1u + (uint32_t)S < hi) issue(c - 1u + (uint32_t)S, (int)((it - 1) % S));
        }
        if (lane == 0 && !pad) {
            if (cnt == 0) {
                bulk_s2g(gout, obase, Q::out_bytes);
            } else {
                if (ob >= 16u) bulk_s2g(gout, obase, ob & ~15u);
                if (SYN != 0 && yb >= 16u) bulk_s2g(gsyn, s_syn, yb & ~15u);
            }
            bulk_commit();
        }
        if constexpr (!INPLACE) {
            if (c + (uint32_t)S < hi) issue(c + (uint32_t)S, s);  // the stage was consumed by this iteration
        }
        __syncwarp();
    }
    if (cur_pk != FULL) flush();
    if (lane == 0) {
        if (aborted) {
            atomicOr(a.status, (uint32_t)HD_ERR_TIMEOUT);
            // wait (bounded) for every load still in flight into this warp's ring
            // (after the first iteration in-place refills lag one iteration)
            const uint32_t pending = (INPLACE && it > 0) ? S - 1 : S;
            for (uint32_t j = it; j < it + pending; ++j)
                if ((uint64_t)lo + j < hi) (void)mbar_wait_bounded(&bar[j % S], (j / S) & 1u);
        }
        bulk_wait_all<0>();
    }
    if constexpr (LUT) {
        // the thread that started the table's copies leaves none of them in flight
        if (threadIdx.x == 0 && aborted) (void)mbar_wait_bounded(lut_bar, 0);
    }
}

// One compiled configuration of the multi-packet streaming decoder.
struct MultiVariant {
    uint32_t n;
    int syn;             // 0 none, 1 u8, 2 u16
    int lut;             // holds the decode table of n = 7 or 15
    int T, S, G, inplace;
    uint32_t smem;
    uint64_t chunk_cw;   // codewords per whole-chunk item (32*G)
    const void *kernel;
    cudaError_t (*launch)(int grid, cudaStream_t st, const MultiArgs &a);
};

template <int N_, int SYN, int T, int S, int G, int INPLACE, bool LUT>
cudaError_t launch_multi(int grid, cudaStream_t st, const MultiArgs &a)
{
    using Cfg = MultiCfg<N_, SYN, T, S, G, INPLACE, LUT>;
    return launch_kernel_uncounted(k_decode_multi<N_, SYN, T, S, G, INPLACE, LUT>, dim3((unsigned)grid), dim3(T),
                                   Cfg::smem, st, false, a);
}

template <int N_, int SYN, int T, int S, int G, int INPLACE, bool LUT>
MultiVariant make_multi_variant()
{
    using Cfg = MultiCfg<N_, SYN, T, S, G, INPLACE, LUT>;
    static_assert(Cfg::fits, "shared memory per CTA");
    MultiVariant v;
    v.n = N_;
    v.syn = SYN;
    v.lut = LUT ? 1 : 0;
    v.T = T;
    v.S = S;
    v.G = G;
    v.inplace = INPLACE;
    v.smem = Cfg::smem;
    v.chunk_cw = Cfg::chunk_cw;
    v.kernel = reinterpret_cast<const void *>(k_decode_multi<N_, SYN, T, S, G, INPLACE, LUT>);
    v.launch = &launch_multi<N_, SYN, T, S, G, INPLACE, LUT>;
    return v;
}

// One configuration for every syndrome type.
template <int N_, int T, int S, int G, int INPLACE, bool LUT = false>
void add_multi_variants(std::vector<MultiVariant> &out)
{
    out.push_back(make_multi_variant<N_, 0, T, S, G, INPLACE, LUT>());
    out.push_back(make_multi_variant<N_, 1, T, S, G, INPLACE, LUT>());
    out.push_back(make_multi_variant<N_, 2, T, S, G, INPLACE, LUT>());
}

// The compiled configurations (hd_multi_a.cu: n = 7, 15, 31; hd_multi_b.cu:
// n = 63, 127, 255), in the order registered.
void register_multi_a(std::vector<MultiVariant> &v);
void register_multi_b(std::vector<MultiVariant> &v);

}  // namespace hd
