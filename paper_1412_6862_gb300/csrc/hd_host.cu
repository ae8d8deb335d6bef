// hd_host.cu -- decode from and to host memory with overlapped transfers.
//
// The paper's asynchronous data transfer (Sec. III-B, Fig. 5, Eq. 1): instead
// of copying a whole packet to the device, decoding it and copying it back in
// sequence, the stream is cut into chunks and each chunk's host-to-device
// copy, decode and device-to-host copy are queued on one of `depth` CUDA
// streams, so that while chunk i is decoded, chunk i+1 is arriving and chunk
// i-1 is leaving (copies in both directions and kernels proceed concurrently).
// Device staging buffers are cached per device and grown on demand.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "hd_internal.h"

namespace hd {
namespace {

constexpr uint32_t kMaxDepth = 8;

struct HostPipe {
    bool init = false;
    uint32_t depth = 0;
    cudaStream_t st[kMaxDepth] = {};
    cudaEvent_t done[kMaxDepth] = {};
    char *dev[kMaxDepth] = {};  // per stream: input | output | syndromes
    size_t cap = 0;             // bytes per stream
    unsigned long long *d_err = nullptr;
    unsigned long long *h_err = nullptr;  // pinned
    size_t err_cap = 0;                   // chunks
};

std::mutex g_pipe_mu;
HostPipe g_pipe[64];

void free_buffers(HostPipe &p)
{
    for (uint32_t s = 0; s < kMaxDepth; ++s) {
        if (p.dev[s]) cudaFree(p.dev[s]);
        p.dev[s] = nullptr;
    }
    p.cap = 0;
}

hd_status ensure(HostPipe &p, uint32_t depth, size_t per_stream, size_t chunks)
{
    if (!p.init) {
        for (uint32_t s = 0; s < kMaxDepth; ++s) {
            if (cudaStreamCreateWithFlags(&p.st[s], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&p.done[s], cudaEventDisableTiming) != cudaSuccess)
                return HD_ERR_CUDA;
        }
        p.init = true;
    }
    if (per_stream > p.cap || depth > p.depth) {
        for (uint32_t s = 0; s < kMaxDepth; ++s) cudaStreamSynchronize(p.st[s]);
        free_buffers(p);
        for (uint32_t s = 0; s < depth; ++s)
            if (cudaMalloc(&p.dev[s], per_stream) != cudaSuccess) return HD_ERR_CUDA;
        p.cap = per_stream;
        p.depth = depth;
    }
    if (chunks > p.err_cap) {
        if (p.d_err) cudaFree(p.d_err);
        if (p.h_err) cudaFreeHost(p.h_err);
        p.d_err = nullptr;
        p.h_err = nullptr;
        if (cudaMalloc(&p.d_err, chunks * sizeof(unsigned long long)) != cudaSuccess ||
            cudaMallocHost(&p.h_err, chunks * sizeof(unsigned long long)) != cudaSuccess)
            return HD_ERR_CUDA;
        p.err_cap = chunks;
    }
    return HD_OK;
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace
}  // namespace hd

using namespace hd;

extern "C" hd_status hd_decode_host(const uint32_t *host_stream, uint64_t in_bits, uint32_t n, uint64_t num_codewords,
                                    uint32_t *host_out, void *host_syndromes, hd_syn_type syn_type,
                                    unsigned long long *host_err_count, uint64_t chunk_codewords, uint32_t depth)
{
    const int m = code_m(n);
    if (m == 0) return HD_ERR_INVALID_N;
    if (syn_type != HD_SYN_NONE && syn_type != HD_SYN_U8 && syn_type != HD_SYN_U16) return HD_ERR_INVALID_ARG;
    if (num_codewords > (1ull << 40)) return HD_ERR_SIZE;
    if (in_bits != (uint64_t)n * num_codewords) return HD_ERR_SIZE;
    if (chunk_codewords == 0) chunk_codewords = 1ull << 20;
    if (depth == 0) depth = 4;
    // chunks start on 16-byte boundaries of both the input and the output
    if (chunk_codewords % 128 != 0 || depth > kMaxDepth) return HD_ERR_INVALID_ARG;
    if (num_codewords == 0) {
        if (host_err_count) *host_err_count = 0;
        return HD_OK;
    }
    if (!host_stream || !host_out) return HD_ERR_NULL;
    if (syn_type != HD_SYN_NONE && !host_syndromes) return HD_ERR_NULL;
    const uint32_t k = n - (uint32_t)m;
    const uint32_t sb = syn_type == HD_SYN_U16 ? 2u : (syn_type == HD_SYN_U8 ? 1u : 0u);
    const uint64_t C = std::min<uint64_t>(chunk_codewords, (num_codewords + 127) / 128 * 128);
    const uint64_t chunks = (num_codewords + C - 1) / C;
    const size_t in_b = round256(words_for_bits(C * n) * 4), out_b = round256(words_for_bits(C * k) * 4),
                 syn_b = round256(C * sb + 16);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return HD_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_pipe_mu);
    HostPipe &p = g_pipe[dev];
    hd_status rc = ensure(p, depth, in_b + out_b + syn_b, chunks);
    if (rc != HD_OK) return rc;
    const uint64_t in_words = words_for_bits(in_bits), out_words = words_for_bits(num_codewords * k);
    for (uint64_t i = 0; i < chunks; ++i) {
        const uint32_t s = (uint32_t)(i % depth);
        cudaStream_t st = p.st[s];
        uint32_t *d_in = reinterpret_cast<uint32_t *>(p.dev[s]);
        uint32_t *d_out = reinterpret_cast<uint32_t *>(p.dev[s] + in_b);
        void *d_syn = sb ? static_cast<void *>(p.dev[s] + in_b + out_b) : nullptr;
        const uint64_t c0 = i * C, cnt = std::min(C, num_codewords - c0);
        const uint64_t w0 = c0 * n / 32, wi = std::min(words_for_bits(cnt * n), in_words - w0);
        const uint64_t o0 = c0 * k / 32, wo = std::min(words_for_bits(cnt * k), out_words - o0);
        if (cudaMemcpyAsync(d_in, host_stream + w0, wi * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return HD_ERR_CUDA;
        rc = hd_decode(d_in, cnt * n, n, cnt, d_out, d_syn, sb ? syn_type : HD_SYN_NONE, p.d_err + i, st);
        if (rc != HD_OK) return rc;
        if (cudaMemcpyAsync(host_out + o0, d_out, wo * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return HD_ERR_CUDA;
        if (sb && cudaMemcpyAsync(static_cast<uint8_t *>(host_syndromes) + c0 * sb, d_syn, cnt * sb,
                                  cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return HD_ERR_CUDA;
    }
    // gather the per-chunk error counts once every stream has finished
    for (uint32_t s = 0; s < depth; ++s) {
        cudaEventRecord(p.done[s], p.st[s]);
        cudaStreamWaitEvent(p.st[0], p.done[s], 0);
    }
    if (cudaMemcpyAsync(p.h_err, p.d_err, chunks * sizeof(unsigned long long), cudaMemcpyDeviceToHost, p.st[0]) !=
        cudaSuccess)
        return HD_ERR_CUDA;
    if (cudaStreamSynchronize(p.st[0]) != cudaSuccess) return HD_ERR_CUDA;
    unsigned long long total = 0;
    for (uint64_t i = 0; i < chunks; ++i) total += p.h_err[i];
    if (host_err_count) *host_err_count = total;
    return HD_OK;
}
