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

namespace hd {
namespace {

struct Chunk {
    uint32_t job;
    uint64_t c0, cnt;  // codewords
};

// The chunk schedule of a batch: every job cut into chunks of C codewords,
// except that the first chunks of the batch ramp up (C/8, C/4, C/2) and the
// last ones ramp down, so the pipeline fills and drains on small copies.
std::vector<Chunk> schedule(const hd_host_job *jobs, uint32_t num, uint64_t C)
{
    std::vector<Chunk> out;
    for (uint32_t j = 0; j < num; ++j)
        for (uint64_t c0 = 0; c0 < jobs[j].num_codewords; c0 += C)
            out.push_back({j, c0, std::min(C, jobs[j].num_codewords - c0)});
    // split the first chunk into pieces of 1/8, 1/4, 1/2 and the rest, and the last chunk into the
    // rest, 1/2, 1/4, 1/8 (multiples of 128 codewords)
    auto ramp = [&](size_t at, bool up) {
        const Chunk big = out[at];
        const uint64_t q[3] = {big.cnt / 8 / 128 * 128, big.cnt / 4 / 128 * 128, big.cnt / 2 / 128 * 128};
        if (q[0] == 0) return;
        const uint64_t rest = big.cnt - q[0] - q[1] - q[2];
        std::vector<Chunk> parts;
        uint64_t c0 = big.c0;
        auto put = [&](uint64_t sz) {
            parts.push_back({big.job, c0, sz});
            c0 += sz;
        };
        if (up) {
            put(q[0]);
            put(q[1]);
            put(q[2]);
            put(rest);
        } else {
            put(rest);
            put(q[2]);
            put(q[1]);
            put(q[0]);
        }
        out.erase(out.begin() + at);
        out.insert(out.begin() + at, parts.begin(), parts.end());
    };
    if (out.size() >= 2) {
        ramp(out.size() - 1, false);
        ramp(0, true);
    }
    return out;
}

}  // namespace
}  // namespace hd

extern "C" hd_status hd_decode_host_batch(const hd_host_job *jobs, uint32_t num_jobs, uint64_t chunk_codewords,
                                          uint32_t depth)
{
    if (num_jobs == 0) return HD_OK;
    if (!jobs) return HD_ERR_NULL;
    if (chunk_codewords == 0) chunk_codewords = 1ull << 22;  // the fastest of 2^19..2^24 on GB300
    if (depth == 0) depth = 4;
    // chunks start on 16-byte boundaries of both the input and the output
    if (chunk_codewords % 128 != 0 || depth > kMaxDepth) return HD_ERR_INVALID_ARG;
    uint64_t C = 0;  // largest chunk any job needs, for the staging size
    size_t in_max = 0, out_max = 0, syn_max = 0;
    for (uint32_t j = 0; j < num_jobs; ++j) {
        const hd_host_job &b = jobs[j];
        const int m = code_m(b.n);
        if (m == 0) return HD_ERR_INVALID_N;
        if (b.syn_type != HD_SYN_NONE && b.syn_type != HD_SYN_U8 && b.syn_type != HD_SYN_U16)
            return HD_ERR_INVALID_ARG;
        if (b.num_codewords > (1ull << 40)) return HD_ERR_SIZE;
        if (b.num_codewords == 0) continue;
        if (!b.host_stream || !b.host_out) return HD_ERR_NULL;
        if (b.syn_type != HD_SYN_NONE && !b.host_syndromes) return HD_ERR_NULL;
        const uint64_t Cj = std::min<uint64_t>(chunk_codewords, (b.num_codewords + 127) / 128 * 128);
        const uint32_t k = b.n - (uint32_t)m, sb = b.syn_type == HD_SYN_U16 ? 2u : (b.syn_type == HD_SYN_U8 ? 1u : 0u);
        in_max = std::max(in_max, round256(words_for_bits(Cj * b.n) * 4));
        out_max = std::max(out_max, round256(words_for_bits(Cj * k) * 4));
        syn_max = std::max(syn_max, round256(Cj * sb + 16));
        C = std::max(C, Cj);
    }
    const std::vector<Chunk> plan = schedule(jobs, num_jobs, chunk_codewords);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return HD_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_pipe_mu);
    HostPipe &p = g_pipe[dev];
    hd_status rc = ensure(p, depth, in_max + out_max + syn_max, std::max<size_t>(plan.size(), 1));
    if (rc != HD_OK) return rc;
    for (size_t i = 0; i < plan.size(); ++i) {
        const Chunk &ch = plan[i];
        const hd_host_job &b = jobs[ch.job];
        const int m = code_m(b.n);
        const uint32_t k = b.n - (uint32_t)m;
        const uint32_t sb = b.syn_type == HD_SYN_U16 ? 2u : (b.syn_type == HD_SYN_U8 ? 1u : 0u);
        const uint32_t s = (uint32_t)(i % depth);
        cudaStream_t st = p.st[s];
        uint32_t *d_in = reinterpret_cast<uint32_t *>(p.dev[s]);
        uint32_t *d_out = reinterpret_cast<uint32_t *>(p.dev[s] + in_max);
        void *d_syn = sb ? static_cast<void *>(p.dev[s] + in_max + out_max) : nullptr;
        const uint64_t in_words = words_for_bits(b.num_codewords * b.n), out_words = words_for_bits(b.num_codewords * k);
        const uint64_t w0 = ch.c0 * b.n / 32, wi = std::min(words_for_bits(ch.cnt * b.n), in_words - w0);
        const uint64_t o0 = ch.c0 * k / 32, wo = std::min(words_for_bits(ch.cnt * k), out_words - o0);
        if (cudaMemcpyAsync(d_in, b.host_stream + w0, wi * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return HD_ERR_CUDA;
        rc = hd_decode(d_in, ch.cnt * b.n, b.n, ch.cnt, d_out, d_syn, sb ? (hd_syn_type)b.syn_type : HD_SYN_NONE,
                       p.d_err + i, st);
        if (rc != HD_OK) return rc;
        if (cudaMemcpyAsync(b.host_out + o0, d_out, wo * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return HD_ERR_CUDA;
        if (sb && cudaMemcpyAsync(static_cast<uint8_t *>(b.host_syndromes) + ch.c0 * sb, d_syn, ch.cnt * sb,
                                  cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return HD_ERR_CUDA;
    }
    // gather the per-chunk error counts once every stream has finished
    for (uint32_t s = 0; s < depth; ++s) {
        cudaEventRecord(p.done[s], p.st[s]);
        cudaStreamWaitEvent(p.st[0], p.done[s], 0);
    }
    if (!plan.empty() && cudaMemcpyAsync(p.h_err, p.d_err, plan.size() * sizeof(unsigned long long),
                                         cudaMemcpyDeviceToHost, p.st[0]) != cudaSuccess)
        return HD_ERR_CUDA;
    if (cudaStreamSynchronize(p.st[0]) != cudaSuccess) return HD_ERR_CUDA;
    for (uint32_t j = 0; j < num_jobs; ++j)
        if (jobs[j].host_err_count) *jobs[j].host_err_count = 0;
    for (size_t i = 0; i < plan.size(); ++i)
        if (jobs[plan[i].job].host_err_count) *jobs[plan[i].job].host_err_count += p.h_err[i];
    return HD_OK;
}

extern "C" hd_status hd_decode_host(const uint32_t *host_stream, uint64_t in_bits, uint32_t n, uint64_t num_codewords,
                                    uint32_t *host_out, void *host_syndromes, hd_syn_type syn_type,
                                    unsigned long long *host_err_count, uint64_t chunk_codewords, uint32_t depth)
{
    if (code_m(n) == 0) return HD_ERR_INVALID_N;
    if (num_codewords > (1ull << 40)) return HD_ERR_SIZE;
    if (in_bits != (uint64_t)n * num_codewords) return HD_ERR_SIZE;
    hd_host_job job;
    job.host_stream = host_stream;
    job.host_out = host_out;
    job.host_syndromes = host_syndromes;
    job.host_err_count = host_err_count;
    job.num_codewords = num_codewords;
    job.n = n;
    job.syn_type = (uint32_t)syn_type;
    if (num_codewords == 0) {
        if (syn_type != HD_SYN_NONE && syn_type != HD_SYN_U8 && syn_type != HD_SYN_U16) return HD_ERR_INVALID_ARG;
        if (chunk_codewords % 128 != 0 || depth > kMaxDepth) return HD_ERR_INVALID_ARG;
        if (host_err_count) *host_err_count = 0;
        return HD_OK;
    }
    return hd_decode_host_batch(&job, 1, chunk_codewords, depth);
}
