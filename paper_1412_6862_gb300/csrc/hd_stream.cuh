// hd_stream.cuh -- the streaming decoder kernel for long single-n streams.
//
// Persistent CTAs whose warps each walk the stream in chunks of 32*G codewords
// (G per thread, so G tiles of 32 codewords per warp).  Lane 0 of every warp
// streams the warp's input chunks into its own S-stage shared-memory ring with
// 1-D bulk copies (cp.async.bulk completing on one mbarrier per stage); every
// thread decodes its part out of shared memory; the decoded words and
// syndromes are staged in shared memory and written back with bulk stores.
// HBM sees one read of every input byte and one write of every output byte.
//
// INPLACE: the decoded words overwrite the chunk's own input stage (the warp
// first copies the chunk to registers), which removes the output staging
// buffers so that more warps fit on an SM; a stage is refilled one iteration
// later, once its bulk store has finished reading it (waiting for that read
// right after issuing the store costs more than the lost lookahead).
#pragma once

#include <cstdint>
#include <vector>

#include "hd_device.cuh"
#include "hd_internal.h"
#include "hd_tile.cuh"

namespace hd {

// One compiled configuration of the streaming decoder.
struct StreamVariant {
    uint32_t n;
    int syn;      // 0 none, 1 u8, 2 u16
    int G;        // codewords per thread
    int T;        // threads per CTA
    int S;        // input stages per warp
    int inplace;  // output written into the input stage
    uint32_t smem;
    uint64_t chunk_cw;  // codewords per warp iteration (32*G)
    cudaError_t (*launch)(const StreamVariant &v, const uint32_t *in, uint64_t nchunks, uint32_t *out, void *syn,
                          unsigned long long *err, uint32_t *status, cudaStream_t st, unsigned long long *det,
                          const uint16_t *lut, bool pdl);
    const void *kernel;
    int xh = 0;   // SECDED: codewords of n + 1 bits with the overall parity bit at position 0
    int lut = 0;  // decode table (n = 7, 15): one shared-memory lookup per codeword
};

// Geometry of one warp chunk of code n: LANES*G codewords (LANES = 32, or 16
// for a half-warp chunk), LANES*G/32 tiles of 32.  XH: SECDED codewords of
// L = n + 1 bits (32 of them fill L words).
template <int N_, int SYN, int G, bool XH = false, int LANES = 32>
struct ChunkGeom {
    using C = Code<N_>;
    static constexpr int L = N_ + (XH ? 1 : 0);                       // input bits per codeword
    static constexpr int H = 32 / G;                                  // threads per 32-codeword tile
    static constexpr int TEAMS = LANES / H;                           // tiles per warp chunk
    static constexpr int SB = SYN == 2 ? 2 : 1;                       // syndrome bytes (packing width)
    // syndrome values of 8 or more bits (m = 8, or SECDED's s | P << m with m >= 7) leave no
    // free top bit in a byte lane: count them by compare instead of the carry trick
    static constexpr bool WIDE = (SB == 1 && C::m + (XH ? 1 : 0) >= 8);
    static constexpr int GK = G * C::k;                               // output bits per thread
    static constexpr bool ALIGNED = (H == 1) || (GK % 32 == 0);
    static constexpr int R = (G * L + 31) / 32;                       // input words per thread after re-alignment
    static constexpr uint32_t in_words = TEAMS * L;
    static constexpr uint32_t in_bytes = in_words * 4;
    // PADDED (SECDED with n >= 63): each thread's part (R words, whole codewords) has its own
    // stage slot of R + 4 words, loaded by its own bulk copy, so that 128-bit reads of the 32
    // parts fall on distinct banks (a part stride that is a multiple of 32 words would put every
    // lane on the same bank).  For n = 63 this measured 56 µs against 64 µs per 2^24
    // codewords on GB300; for n <= 31 one bulk copy per chunk measured faster despite the
    // conflicts (n = 31: 40 µs against 46).
    static constexpr bool PADDED = XH && N_ >= 63;
    static constexpr uint32_t part_words = R + 4;
    static constexpr uint32_t stage_payload = PADDED ? 32 * part_words * 4 : in_bytes;
    static_assert(!PADDED || (R % 4 == 0 && 32 * R == (int)in_words), "padded parts are whole 16-byte groups");
    static constexpr uint32_t out_words = TEAMS * C::k;
    static constexpr uint32_t out_bytes = out_words * 4;
    static constexpr uint32_t syn_bytes = SYN ? LANES * G * SB : 0;
    static_assert(LANES == 32 || (LANES == 16 && !PADDED && H <= 16), "whole tiles on the active lanes");
    static constexpr int V = !ALIGNED                                ? 1
                             : (C::k % 4 == 0 && (GK / 32) % 4 == 0) ? 4
                             : (C::k % 2 == 0 && (GK / 32) % 2 == 0) ? 2
                                                                     : 1;
    static_assert(in_bytes % 16 == 0 && out_bytes % 16 == 0 && syn_bytes % 16 == 0, "bulk copies need 16B sizes");
};

// Decode one warp chunk held in shared memory at `stage` (its input words,
// plus one spare word).  Writes the chunk's output words at `obase` (which may
// equal `stage`: every lane copies its part to registers and the warp
// synchronises before the first write) and its syndromes at `sbase`.  Returns
// this lane's count of nonzero syndromes.  With LANES = 16 the chunk is half
// as long: lanes 16..31 read and write nothing (they only join the warp's
// synchronisation) and return 0.
template <int N_, int SYN, int G, bool XH = false, bool LUT = false, int LANES = 32>
__device__ __forceinline__ uint32_t decode_warp_chunk(const uint32_t *stage, uint32_t *obase, uint8_t *sbase, int lane,
                                                      uint32_t &det, const uint16_t *lut = nullptr)
{
    using Q = ChunkGeom<N_, SYN, G, XH, LANES>;
    const bool active = LANES == 32 || lane < LANES;
    constexpr int H = Q::H;
    const int team = lane / H, h = lane % H;
    const uint32_t in_bit = (uint32_t)h * (uint32_t)(G * Q::L);
    const uint32_t in_w = team * Q::L + (in_bit >> 5), in_sh = in_bit & 31u;
    const uint32_t out_bit = (uint32_t)h * (uint32_t)Q::GK;
    const uint32_t out_w = team * Code<N_>::k + (out_bit >> 5), out_sh = out_bit & 31u;
    uint32_t r[Q::R];
    if (!active) {
        // no part: keep the registers defined, never used
#pragma unroll
        for (int w = 0; w < Q::R; ++w) r[w] = 0u;
    } else if constexpr (Q::PADDED) {
        const uint4 *part = reinterpret_cast<const uint4 *>(stage + lane * Q::part_words);
#pragma unroll
        for (int t = 0; t < Q::R / 4; ++t) {
            const uint4 v = part[t];
            r[4 * t] = v.x;
            r[4 * t + 1] = v.y;
            r[4 * t + 2] = v.z;
            r[4 * t + 3] = v.w;
        }
    } else if constexpr (H == 1) {
#pragma unroll
        for (int w = 0; w < Q::R; ++w) r[w] = stage[in_w + w];
    } else {
        uint32_t lo = stage[in_w];
#pragma unroll
        for (int w = 0; w < Q::R; ++w) {
            const uint32_t hi = stage[in_w + w + 1];
            r[w] = __funnelshift_r(lo, hi, in_sh);
            lo = hi;
        }
    }
    __syncwarp();  // the whole chunk is in registers
    if (!active) return 0u;
    OutPacker<Q::GK, Q::ALIGNED, Q::V> op(obase + out_w, out_sh);
    SynPacker<Q::SB, SYN != 0, G, Q::WIDE> sp(sbase + (uint32_t)lane * G * Q::SB);
    decode_part<N_, G, Q::R, XH, LUT>(r, op, sp, det, lut);
    return sp.nonzero();
}

// Every warp is an independent pipeline: it owns S input stages with one
// mbarrier each and (unless INPLACE) two output staging buffers.  Lane 0
// issues the warp's bulk loads and data stores; the syndromes go from the
// lanes' registers straight to global memory (each lane's run of G syndromes
// is contiguous, stored in 16-byte vectors).  Warps never wait for one
// another, so one warp's memory wait overlaps the others' arithmetic.
template <int N_, int SYN, int T, int S, int G, int INPLACE, bool XH = false, bool LUT = false>
struct StreamCfg : ChunkGeom<N_, SYN, G, XH> {
    using Q = ChunkGeom<N_, SYN, G, XH>;
    static constexpr int WARPS = T / 32;
    static constexpr uint32_t stage_bytes = Q::stage_payload + 16;  // one spare 16-byte group for the funnel read
    static constexpr uint32_t out_buf_bytes = Q::out_bytes + 16;  // room for a spill word
    // per-warp layout
    static constexpr uint32_t off_bar = 0;
    static constexpr uint32_t off_in = 64;
    static constexpr uint32_t off_out = off_in + S * stage_bytes;
    static constexpr uint32_t warp_bytes = (off_out + (INPLACE ? 0 : 2 * out_buf_bytes) + 127) / 128 * 128;
    static constexpr uint32_t lut_bytes = LUT ? (2u << (N_ + (XH ? 1 : 0))) : 0u;  // u16 per codeword value
    static constexpr uint32_t off_lut = WARPS * warp_bytes;         // the table, then its mbarrier
    static constexpr uint32_t smem = off_lut + (LUT ? lut_bytes + 16u : 0u);
    static constexpr bool fits = smem <= 232448;  // the opt-in maximum per CTA
    static_assert(T % 32 == 0 && S <= 8, "whole warps, at most 8 stages");
    static_assert(!INPLACE || Q::out_bytes + 16 <= stage_bytes, "in-place output fits the input stage");
    static_assert(!INPLACE || S >= 2, "in-place refills lag one iteration");
};

// Load chunk c into a stage; called by every lane of the warp.  Unpadded
// stages: lane 0 issues one bulk copy.  Padded: lane 0 announces the bytes,
// then every lane copies its own part into its slot.
template <class Cfg, bool XH>
__device__ __forceinline__ void issue_chunk(const uint32_t *in, uint64_t c, uint8_t *stage, uint64_t *bar, int lane)
{
    if constexpr (!Cfg::PADDED) {
        if (lane == 0) {
            mbar_arrive_expect_tx(bar, Cfg::in_bytes);
            bulk_g2s(stage, in + c * (uint64_t)Cfg::in_words, Cfg::in_bytes, bar);
        }
    } else {
        if (lane == 0) mbar_arrive_expect_tx(bar, Cfg::in_bytes);
        __syncwarp();
        bulk_g2s(stage + lane * Cfg::part_words * 4, in + c * (uint64_t)Cfg::in_words + (uint64_t)lane * Cfg::R,
                 Cfg::R * 4, bar);
    }
}

template <int N_, int SYN, int T, int S, int G, int INPLACE, bool XH = false, bool LUT = false>
__global__ void __launch_bounds__(T)
    k_decode_stream(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, uint8_t *__restrict__ syn,
                    unsigned long long *__restrict__ err, uint32_t *__restrict__ status, uint64_t nchunks,
                    unsigned long long *__restrict__ det, const uint16_t *__restrict__ lut)
{
    using Cfg = StreamCfg<N_, SYN, T, S, G, INPLACE, XH, LUT>;
    extern __shared__ __align__(128) uint8_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // Programmatic dependent launch, both ways: the next kernel of the stream
    // may launch now (an hd_decode behind this one starts its launch and
    // prologue while this one drains), and this kernel may have started before
    // the kernel ahead of it finished, so it touches no global memory other
    // than the library's own decode table before grid_dep_wait() below.
    grid_dep_launch_dependents();
    uint64_t *lut_bar = nullptr;
    if constexpr (LUT) {
        // the decode table: bulk copies into shared memory behind the warps'
        // areas, in flight together with the warps' first chunks
        static_assert(Cfg::lut_bytes % 16 == 0 && Cfg::off_lut % 16 == 0, "bulk copy granularity");
        lut_bar = reinterpret_cast<uint64_t *>(smem + Cfg::off_lut + Cfg::lut_bytes);
        if (threadIdx.x == 0) {
            mbar_init(lut_bar, 1);
            fence_mbar_init();
            mbar_arrive_expect_tx(lut_bar, Cfg::lut_bytes);
            constexpr uint32_t piece = Cfg::lut_bytes < 16384u ? Cfg::lut_bytes : 16384u;
            static_assert(Cfg::lut_bytes % piece == 0, "whole pieces");
#pragma unroll
            for (uint32_t o = 0; o < Cfg::lut_bytes; o += piece)
                bulk_g2s(smem + Cfg::off_lut + o, reinterpret_cast<const uint8_t *>(lut) + o, piece, lut_bar);
        }
        __syncthreads();  // the barrier is initialised before any thread waits on it
    }
    uint8_t *wbase = smem + warp * Cfg::warp_bytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(wbase + Cfg::off_bar);
    uint8_t *s_in = wbase + Cfg::off_in;
    uint8_t *s_out = wbase + Cfg::off_out;
    const uint64_t gw = (uint64_t)blockIdx.x * Cfg::WARPS + warp;  // global warp index
    const uint64_t tw = (uint64_t)gridDim.x * Cfg::WARPS;          // warps in the grid
    grid_dep_wait();  // the kernels ahead (the counters' clear, and what produced the input) have finished

    if constexpr (!Cfg::PADDED) {
        if (lane == 0) {
#pragma unroll
            for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
            fence_mbar_init();
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const uint64_t c = gw + (uint64_t)s * tw;
                if (c < nchunks) {
                    mbar_arrive_expect_tx(&bar[s], Cfg::in_bytes);
                    bulk_g2s(s_in + s * Cfg::stage_bytes, in + c * (uint64_t)Cfg::in_words, Cfg::in_bytes, &bar[s]);
                }
            }
        }
    } else {
        if (lane == 0) {
#pragma unroll
            for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
            fence_mbar_init();
        }
        __syncwarp();  // every lane's copies complete on the barriers
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const uint64_t c = gw + (uint64_t)s * tw;
            if (c < nchunks) issue_chunk<Cfg, true>(in, c, s_in + s * Cfg::stage_bytes, &bar[s], lane);
        }
    }
    __syncwarp();

    uint32_t errs = 0, dets = 0;
    uint32_t it = 0;
    bool aborted = false;
    const uint16_t *s_lut = nullptr;
    if constexpr (LUT) {
        const bool ok = mbar_wait_bounded(lut_bar, 0);
        aborted = __any_sync(0xFFFFFFFFu, !ok);
        s_lut = reinterpret_cast<const uint16_t *>(smem + Cfg::off_lut);
    }
    for (uint64_t c = gw; !aborted && c < nchunks; c += tw, ++it) {
        const int s = (int)(it % S);
        const uint32_t parity = (it / S) & 1u;
        const int ob = (int)(it & 1u);
        const bool ok = mbar_wait_bounded(&bar[s], parity);
        if (__any_sync(0xFFFFFFFFu, !ok)) {
            aborted = true;
            break;
        }
        if constexpr (!INPLACE) {
            if (lane == 0) bulk_wait_read<1>();  // staging buffer ob no longer read by the store of it-2
            __syncwarp();
        }
        const uint32_t *stage = reinterpret_cast<const uint32_t *>(s_in + s * Cfg::stage_bytes);
        uint32_t *obase = INPLACE ? reinterpret_cast<uint32_t *>(s_in + s * Cfg::stage_bytes)
                                  : reinterpret_cast<uint32_t *>(s_out + ob * Cfg::out_buf_bytes);
        // syndromes go straight to global memory: each lane's run of G is contiguous
        uint8_t *sdst = SYN != 0 ? syn + c * (uint64_t)Cfg::syn_bytes : s_in;
        errs += decode_warp_chunk<N_, SYN, G, XH, LUT>(stage, obase, sdst, lane, dets, s_lut);
        fence_proxy_async_smem();
        __syncwarp();
        if constexpr (Cfg::PADDED) {
            if constexpr (INPLACE) {
                if (lane == 0) bulk_wait_read<0>();  // last iteration's store has read its stage
                __syncwarp();
                if (it > 0) {
                    const uint64_t cn = c - tw + (uint64_t)S * tw;
                    if (cn < nchunks)
                        issue_chunk<Cfg, true>(in, cn, s_in + (int)((it - 1) % S) * Cfg::stage_bytes,
                                               &bar[(it - 1) % S], lane);
                }
            }
            if (lane == 0) {
                bulk_s2g(out + c * (uint64_t)Cfg::out_words, obase, Cfg::out_bytes);
                bulk_commit();
            }
            if constexpr (!INPLACE) {
                const uint64_t cn = c + (uint64_t)S * tw;
                if (cn < nchunks) issue_chunk<Cfg, true>(in, cn, s_in + s * Cfg::stage_bytes, &bar[s], lane);
            }
        } else if (lane == 0) {
            if constexpr (INPLACE) {
                // the store issued last iteration has finished reading its stage: refill that
                // stage with the chunk S iterations after it (so in place the lookahead is S - 1)
                bulk_wait_read<0>();
                if (it > 0) {
                    const uint64_t cn = c - tw + (uint64_t)S * tw;
                    if (cn < nchunks) {
                        const int ps = (int)((it - 1) % S);
                        mbar_arrive_expect_tx(&bar[ps], Cfg::in_bytes);
                        bulk_g2s(s_in + ps * Cfg::stage_bytes, in + cn * (uint64_t)Cfg::in_words, Cfg::in_bytes,
                                 &bar[ps]);
                    }
                }
            }
            bulk_s2g(out + c * (uint64_t)Cfg::out_words, obase, Cfg::out_bytes);
            bulk_commit();
            if constexpr (!INPLACE) {
                // the stage was consumed by this iteration: prefetch the chunk S iterations ahead
                const uint64_t cn = c + (uint64_t)S * tw;
                if (cn < nchunks) {
                    mbar_arrive_expect_tx(&bar[s], Cfg::in_bytes);
                    bulk_g2s(s_in + s * Cfg::stage_bytes, in + cn * (uint64_t)Cfg::in_words, Cfg::in_bytes, &bar[s]);
                }
            }
        }
        __syncwarp();
    }
    if (lane == 0) {
        if (aborted) {
            atomicOr(status, (uint32_t)HD_ERR_TIMEOUT);
            // wait (bounded) for every load still in flight into this warp's ring
            // (after the first iteration in-place refills lag one iteration, so
            // one fewer is outstanding) and for the table
            const uint32_t pending = (INPLACE && it > 0) ? S - 1 : S;
            for (uint32_t j = it; j < it + pending; ++j) {
                const uint64_t cj = gw + (uint64_t)j * tw;
                if (cj < nchunks) (void)mbar_wait_bounded(&bar[j % S], (j / S) & 1u);
            }
            if constexpr (LUT) (void)mbar_wait_bounded(lut_bar, 0);
        }
        bulk_wait_all<0>();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) errs += __shfl_xor_sync(0xFFFFFFFFu, errs, o);
    if constexpr (XH) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dets += __shfl_xor_sync(0xFFFFFFFFu, dets, o);
    }
    if (lane == 0) {
        if (err != nullptr && errs != 0) atomicAdd(err, (unsigned long long)errs);
        if (XH && det != nullptr && dets != 0) atomicAdd(det, (unsigned long long)dets);
    }
}

template <int N_, int SYN, int T, int S, int G, int INPLACE, bool XH = false, bool LUT = false>
cudaError_t launch_stream_variant(const StreamVariant &v, const uint32_t *in, uint64_t nchunks, uint32_t *out,
                                  void *syn, unsigned long long *err, uint32_t *status, cudaStream_t st,
                                  unsigned long long *det, const uint16_t *lut, bool pdl);

// Per-device configuration of a kernel (dynamic shared memory opt-in and the
// number of resident CTAs per SM).
int stream_blocks_per_sm(const void *kernel, int threads, uint32_t smem);

template <int N_, int SYN, int T, int S, int G, int INPLACE, bool XH, bool LUT>
cudaError_t launch_stream_variant(const StreamVariant &v, const uint32_t *in, uint64_t nchunks, uint32_t *out,
                                  void *syn, unsigned long long *err, uint32_t *status, cudaStream_t st,
                                  unsigned long long *det, const uint16_t *lut, bool pdl)
{
    using Cfg = StreamCfg<N_, SYN, T, S, G, INPLACE, XH, LUT>;
    if (LUT && lut == nullptr) return cudaErrorInvalidValue;
    auto kern = k_decode_stream<N_, SYN, T, S, G, INPLACE, XH, LUT>;
    const int bps = stream_blocks_per_sm(reinterpret_cast<const void *>(kern), T, Cfg::smem);
    if (bps <= 0) return cudaErrorInvalidConfiguration;
    const uint64_t cap = (uint64_t)num_sms() * (uint64_t)bps;
    const uint64_t want = (nchunks + Cfg::WARPS - 1) / Cfg::WARPS;
    const int grid = decode_grid(want, cap);
    // with pdl the launch may overlap the kernel ahead of it (the counters'
    // clear, or a decode's drain); the kernel waits for it before its first
    // access to global memory
    return launch_kernel(kern, dim3((unsigned)grid), dim3(T), Cfg::smem, st, pdl, in, out,
                         static_cast<uint8_t *>(syn), err, status, nchunks, det, lut);
}

template <int N_, int SYN, int T, int S, int G, int INPLACE, bool XH = false, bool LUT = false>
StreamVariant make_variant()
{
    using Cfg = StreamCfg<N_, SYN, T, S, G, INPLACE, XH, LUT>;
    static_assert(Cfg::fits, "shared memory per CTA");
    StreamVariant v;
    v.n = N_;
    v.syn = SYN;
    v.G = G;
    v.T = T;
    v.S = S;
    v.inplace = INPLACE;
    v.smem = Cfg::smem;
    v.chunk_cw = (uint64_t)32 * G;
    v.launch = &launch_stream_variant<N_, SYN, T, S, G, INPLACE, XH, LUT>;
    v.kernel = reinterpret_cast<const void *>(k_decode_stream<N_, SYN, T, S, G, INPLACE, XH, LUT>);
    v.xh = XH ? 1 : 0;
    v.lut = LUT ? 1 : 0;
    return v;
}

// Every syndrome type of one configuration whose shared memory fits a CTA.
template <int N_, int SYN, int T, int S, int G, int INPLACE, bool XH, bool LUT>
void add_variant_if_fits(std::vector<StreamVariant> &out)
{
    if constexpr (StreamCfg<N_, SYN, T, S, G, INPLACE, XH, LUT>::fits)
        out.push_back(make_variant<N_, SYN, T, S, G, INPLACE, XH, LUT>());
}

template <int N_, int T, int S, int G, int INPLACE, bool XH = false, bool LUT = false>
void add_variants(std::vector<StreamVariant> &out)
{
    static_assert(StreamCfg<N_, 0, T, S, G, INPLACE, XH, LUT>::fits, "shared memory per CTA");
    add_variant_if_fits<N_, 0, T, S, G, INPLACE, XH, LUT>(out);
    add_variant_if_fits<N_, 1, T, S, G, INPLACE, XH, LUT>(out);
    add_variant_if_fits<N_, 2, T, S, G, INPLACE, XH, LUT>(out);
}

}  // namespace hd
