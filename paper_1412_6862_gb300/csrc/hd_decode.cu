// hd_decode.cu -- streaming decoder for long single-n streams on sm_103a.
//
// Persistent CTAs walk the stream in chunks of T thread tiles (32*T
// codewords, T*n input words, T*k output words).  One elected thread streams
// the input chunks into an S-stage shared-memory ring with 1-D bulk copies
// (cp.async.bulk, completing on an mbarrier per stage); every thread decodes
// its own 32-codeword tile out of shared memory (stride n words between
// threads, conflict-free because n is odd); the decoded words and syndromes
// go to a double-buffered shared staging area that the elected thread writes
// back with bulk stores.  HBM sees exactly one read of every input byte and
// one write of every output byte.
#include <cstdint>

#include "hd_device.cuh"
#include "hd_internal.h"
#include "hd_tile.cuh"

namespace hd {
namespace {

__device__ uint32_t g_status_decode;

template <int N_, int SYN, int T, int S>
struct StreamCfg {
    using C = Code<N_>;
    static constexpr int SB = SYN == 2 ? 2 : 1;
    static constexpr uint32_t in_bytes = T * N_ * 4;
    static constexpr uint32_t out_bytes = T * C::k * 4;
    static constexpr uint32_t syn_bytes = SYN ? T * 32 * SB : 0;
    static constexpr uint32_t off_in = 128;
    static constexpr uint32_t off_out = off_in + S * in_bytes;
    static constexpr uint32_t off_syn = off_out + 2 * out_bytes;
    static constexpr uint32_t smem = off_syn + 2 * syn_bytes;
    static constexpr int V = (C::k % 4 == 0) ? 4 : (C::k % 2 == 0) ? 2 : 1;
    static_assert(in_bytes % 16 == 0 && out_bytes % 16 == 0 && syn_bytes % 16 == 0, "bulk copies need 16B sizes");
};

template <int N_, int SYN, int T, int S>
__global__ void __launch_bounds__(T)
    k_decode_stream(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, uint8_t *__restrict__ syn,
                    unsigned long long *__restrict__ err, uint64_t nchunks)
{
    using Cfg = StreamCfg<N_, SYN, T, S>;
    constexpr int K = Code<N_>::k;
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    uint32_t *s_in = reinterpret_cast<uint32_t *>(smem + Cfg::off_in);
    uint32_t *s_out = reinterpret_cast<uint32_t *>(smem + Cfg::off_out);
    uint8_t *s_syn = smem + Cfg::off_syn;
    const int tid = threadIdx.x;

    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const uint64_t c = blockIdx.x + (uint64_t)s * gridDim.x;
            if (c < nchunks) {
                mbar_arrive_expect_tx(&bar[s], Cfg::in_bytes);
                bulk_g2s(s_in + s * T * N_, in + c * (uint64_t)(T * N_), Cfg::in_bytes, &bar[s]);
            }
        }
    }

    uint32_t errs = 0;
    uint32_t it = 0;
    bool aborted = false;
    for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x, ++it) {
        const int s = (int)(it % S);
        const uint32_t parity = (it / S) & 1u;
        const int ob = (int)(it & 1u);
        const bool ok = mbar_wait_bounded(&bar[s], parity);
        if (tid == 0) bulk_wait_read<1>();  // staging buffer ob is no longer read by the store of it-2
        if (__syncthreads_or(!ok)) {
            aborted = true;
            break;
        }
        {
            uint32_t r[N_];
            const uint32_t *src = s_in + s * T * N_ + tid * N_;
#pragma unroll
            for (int w = 0; w < N_; ++w) r[w] = src[w];
            OutPacker<Cfg::V> op(s_out + ob * T * K + tid * K);
            SynPacker<Cfg::SB, SYN != 0> sp(s_syn + ob * Cfg::syn_bytes + tid * 32 * Cfg::SB);
            decode_thread_tile<N_>(r, op, sp);
            errs += sp.nonzero();
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            bulk_s2g(out + c * (uint64_t)(T * K), s_out + ob * T * K, Cfg::out_bytes);
            if constexpr (SYN != 0)
                bulk_s2g(syn + c * (uint64_t)Cfg::syn_bytes, s_syn + ob * Cfg::syn_bytes, Cfg::syn_bytes);
            bulk_commit();
            const uint64_t cn = c + (uint64_t)S * gridDim.x;
            if (cn < nchunks) {
                mbar_arrive_expect_tx(&bar[s], Cfg::in_bytes);
                bulk_g2s(s_in + s * T * N_, in + cn * (uint64_t)(T * N_), Cfg::in_bytes, &bar[s]);
            }
        }
    }
    if (aborted && tid == 0) {
        atomicOr(&g_status_decode, (uint32_t)HD_ERR_TIMEOUT);
        // Wait (bounded) for every load still in flight into this CTA's ring.
        for (uint32_t j = it; j < it + S; ++j) {
            const uint64_t cj = blockIdx.x + (uint64_t)j * gridDim.x;
            if (cj < nchunks) (void)mbar_wait_bounded(&bar[j % S], (j / S) & 1u);
        }
    }
    if (tid == 0) bulk_wait_all<0>();
    if (err != nullptr) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) errs += __shfl_xor_sync(0xFFFFFFFFu, errs, o);
        if ((tid & 31) == 0 && errs != 0) atomicAdd(err, (unsigned long long)errs);
    }
}

template <int N_, int SYN, int T, int S>
cudaError_t launch_stream(const uint32_t *in, uint64_t num_cw, uint32_t *out, void *syn, unsigned long long *err,
                          cudaStream_t st, uint64_t *covered)
{
    using Cfg = StreamCfg<N_, SYN, T, S>;
    const uint64_t nchunks = num_cw / (32ull * T);
    *covered = nchunks * 32ull * T;
    if (nchunks == 0) return cudaSuccess;
    auto kern = k_decode_stream<N_, SYN, T, S>;
    static int configured_dev = -1;
    static int blocks_per_sm = 1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::smem);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, T, Cfg::smem);
        if (e != cudaSuccess) return e;
        if (blocks_per_sm < 1) blocks_per_sm = 1;
        configured_dev = dev;
    }
    const uint64_t cap = (uint64_t)num_sms() * blocks_per_sm;
    const int grid = (int)(nchunks < cap ? nchunks : cap);
    kern<<<grid, T, Cfg::smem, st>>>(in, out, static_cast<uint8_t *>(syn), err, nchunks);
    count_launch();
    return cudaGetLastError();
}

template <int N_, int T, int S>
cudaError_t launch_stream_syn(const uint32_t *in, uint64_t num_cw, uint32_t *out, void *syn, int syn_type,
                              unsigned long long *err, cudaStream_t st, uint64_t *covered)
{
    switch (syn_type) {
        case 1: return launch_stream<N_, 1, T, S>(in, num_cw, out, syn, err, st, covered);
        case 2: return launch_stream<N_, 2, T, S>(in, num_cw, out, syn, err, st, covered);
        default: return launch_stream<N_, 0, T, S>(in, num_cw, out, syn, err, st, covered);
    }
}

}  // namespace

cudaError_t launch_decode_fast(const uint32_t *in, uint32_t n, uint64_t num_cw, uint32_t *out, void *syn,
                               int syn_type, unsigned long long *err, cudaStream_t st, uint64_t *covered)
{
    *covered = 0;
    switch (n) {
        case 7: return launch_stream_syn<7, 256, 4>(in, num_cw, out, syn, syn_type, err, st, covered);
        case 15: return launch_stream_syn<15, 256, 4>(in, num_cw, out, syn, syn_type, err, st, covered);
        case 31: return launch_stream_syn<31, 128, 4>(in, num_cw, out, syn, syn_type, err, st, covered);
        case 63: return launch_stream_syn<63, 64, 4>(in, num_cw, out, syn, syn_type, err, st, covered);
        default: return cudaSuccess;
    }
}

uint32_t read_clear_status_decode()
{
    uint32_t v = 0, zero = 0;
    cudaMemcpyFromSymbol(&v, g_status_decode, sizeof(v));
    cudaMemcpyToSymbol(g_status_decode, &zero, sizeof(zero));
    return v;
}

}  // namespace hd
