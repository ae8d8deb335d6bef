// hd_api.cu -- the C ABI of libhd.so: argument checks and kernel dispatch for
// the single-stream calls.  See include/hd.h for the contract.
#include <algorithm>
#include <cstdint>
#include <mutex>

#include "hd_device.cuh"
#include "hd_internal.h"

namespace hd {

std::atomic<uint64_t> g_launches{0};
std::atomic<uint32_t> g_max_ctas{0};

int num_sms()
{
    static std::mutex mu;
    static int cached[64];
    static bool init = false;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!init) {
        for (int &c : cached) c = 0;
        init = true;
    }
    if (dev < 0 || dev >= 64) dev = 0;
    if (cached[dev] == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 1;
    }
    return cached[dev];
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

namespace {

// Lets the next kernel of the stream launch at once, waits for the kernel
// ahead of it (when it was launched as its programmatic dependent, that
// kernel may still be running and adding to these very counters), then
// clears the counters.
__global__ void k_zero_counts(unsigned long long *a, unsigned long long *b)
{
    grid_dep_launch_dependents();
    grid_dep_wait();
    if (threadIdx.x == 0) {
        if (a) *a = 0ull;
        if (b) *b = 0ull;
    }
}

// Up to kMaxStreamJobs counters, cleared by one thread each.
constexpr uint32_t kMaxStreamJobs = 32;
struct ZeroList {
    unsigned long long *p[kMaxStreamJobs];
    uint32_t count;
};

__global__ void k_zero_list(ZeroList z)
{
    if (threadIdx.x < z.count) *z.p[threadIdx.x] = 0ull;
}

// Streams and events of hd_decode_streams(), per device, created on its first call.
constexpr int kPoolStreams = 8;
constexpr int kMaxDevices = 64;
struct JobPool {
    std::mutex mu;
    bool ready = false;
    cudaStream_t s[kPoolStreams] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kPoolStreams] = {};
};
JobPool g_job_pools[kMaxDevices];

hd_status check_decode_args(const uint32_t *stream, uint64_t in_bits, uint32_t n, uint64_t num_codewords,
                            uint32_t *out_bits, void *syndromes, hd_syn_type syn_type)
{
    const int m = code_m(n);
    if (m == 0) return HD_ERR_INVALID_N;
    if (syn_type != HD_SYN_NONE && syn_type != HD_SYN_U8 && syn_type != HD_SYN_U16) return HD_ERR_INVALID_ARG;
    if (num_codewords > (1ull << 40)) return HD_ERR_SIZE;
    if (in_bits != (uint64_t)n * num_codewords) return HD_ERR_SIZE;
    if (num_codewords == 0) return HD_OK;
    if (!stream || !out_bits) return HD_ERR_NULL;
    if (syn_type != HD_SYN_NONE && !syndromes) return HD_ERR_NULL;
    if (!aligned16(stream) || !aligned16(out_bits) || (syndromes && !aligned16(syndromes))) return HD_ERR_ALIGN;
    return HD_OK;
}

// The decode of one checked stream (num_codewords > 0) on `st`, counters
// already cleared; pdl: the streaming kernel is the programmatic dependent of
// the clear just enqueued on `st`.
hd_status enqueue_decode(const uint32_t *stream, uint64_t in_bits, uint32_t n, uint64_t num_codewords,
                         uint32_t *out_bits, void *syndromes, hd_syn_type syn_type, unsigned long long *err_count,
                         cudaStream_t st, bool pdl)
{
    const uint32_t k = n - (uint32_t)code_m(n);
    const uint64_t in_words = words_for_bits(in_bits);
    const uint64_t out_words = words_for_bits(num_codewords * k);
    const int syn = syndromes ? (int)syn_type : 0;
    uint64_t covered = 0;
    if (launch_decode_fast(stream, n, num_codewords, out_bits, syndromes, syn, err_count, st, &covered, pdl) !=
        cudaSuccess)
        return HD_ERR_CUDA;
    if (covered < num_codewords) {
        const uint64_t tile_begin = covered / 32, tile_end = (num_codewords + 31) / 32;
        if (launch_decode_generic(stream, in_words, n, num_codewords, tile_begin, tile_end, out_bits, out_words,
                                  syndromes, syn, err_count, st) != cudaSuccess)
            return HD_ERR_CUDA;
    }
    return HD_OK;
}

}  // namespace

cudaError_t launch_zero_counts(unsigned long long *a, unsigned long long *b, cudaStream_t st, bool chained)
{
    return launch_kernel(k_zero_counts, dim3(1), dim3(32), 0, st, chained, a, b);
}

}  // namespace hd

using namespace hd;

extern "C" {

int hd_version(void) { return 100; }

uint64_t hd_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

hd_status hd_set_max_ctas(uint32_t max_ctas)
{
    g_max_ctas.store(max_ctas, std::memory_order_relaxed);
    return HD_OK;
}

uint32_t hd_get_max_ctas(void) { return g_max_ctas.load(std::memory_order_relaxed); }

const char *hd_status_string(hd_status status)
{
    switch (status) {
        case HD_OK: return "HD_OK";
        case HD_ERR_INVALID_N: return "HD_ERR_INVALID_N: n must be 2^m-1 with 2<=m<=8";
        case HD_ERR_NULL: return "HD_ERR_NULL: a required pointer is NULL";
        case HD_ERR_SIZE: return "HD_ERR_SIZE: sizes do not match";
        case HD_ERR_ALIGN: return "HD_ERR_ALIGN: buffer not 16-byte aligned";
        case HD_ERR_CAPACITY: return "HD_ERR_CAPACITY: capacity exceeded";
        case HD_ERR_TIMEOUT: return "HD_ERR_TIMEOUT: a bounded device wait ran out";
        case HD_ERR_CUDA: return "HD_ERR_CUDA: CUDA runtime error";
        case HD_ERR_INVALID_ARG: return "HD_ERR_INVALID_ARG: invalid argument";
    }
    return "unknown hd_status";
}

hd_status hd_device_status(uint32_t *status)
{
    if (!status) return HD_ERR_NULL;
    if (cudaDeviceSynchronize() != cudaSuccess) return HD_ERR_CUDA;
    *status = read_clear_status_decode();
    return cudaGetLastError() == cudaSuccess ? HD_OK : HD_ERR_CUDA;
}

hd_status hd_decode(const uint32_t *stream, uint64_t in_bits, uint32_t n, uint64_t num_codewords,
                    uint32_t *out_bits, void *syndromes, hd_syn_type syn_type, unsigned long long *err_count,
                    void *cuda_stream)
{
    hd_status rc = check_decode_args(stream, in_bits, n, num_codewords, out_bits, syndromes, syn_type);
    if (rc != HD_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (num_codewords == 0) {
        if (err_count && cudaMemsetAsync(err_count, 0, sizeof(*err_count), st) != cudaSuccess) return HD_ERR_CUDA;
        return HD_OK;
    }
    // the clear and the decode both chained (programmatic dependent launch):
    // the clear may start while the kernel ahead drains and waits for it
    // before writing; the decode waits for the clear before touching memory
    if (err_count && launch_zero_counts(err_count, nullptr, st, true) != cudaSuccess) return HD_ERR_CUDA;
    return enqueue_decode(stream, in_bits, n, num_codewords, out_bits, syndromes, syn_type, err_count, st, true);
}

hd_status hd_decode_streams(const hd_stream_job *jobs, uint32_t num_jobs, void *cuda_stream)
{
    if (num_jobs > 0 && jobs == nullptr) return HD_ERR_NULL;
    if (num_jobs > kMaxStreamJobs) return HD_ERR_CAPACITY;
    for (uint32_t i = 0; i < num_jobs; ++i) {
        const hd_stream_job &j = jobs[i];
        const hd_status rc = check_decode_args(j.stream, (uint64_t)j.n * j.num_codewords, j.n, j.num_codewords,
                                               j.out_bits, j.syndromes, static_cast<hd_syn_type>(j.syn_type));
        if (rc != HD_OK) return rc;
    }
    if (num_jobs == 0) return HD_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HD_ERR_CUDA;
    JobPool &pool = g_job_pools[dev];
    std::lock_guard<std::mutex> lk(pool.mu);
    if (!pool.ready) {
        for (int i = 0; i < kPoolStreams; ++i)
            if (cudaStreamCreateWithFlags(&pool.s[i], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&pool.join[i], cudaEventDisableTiming) != cudaSuccess)
                return HD_ERR_CUDA;
        if (cudaEventCreateWithFlags(&pool.fork, cudaEventDisableTiming) != cudaSuccess) return HD_ERR_CUDA;
        pool.ready = true;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // every counter cleared by one kernel on the caller's stream, before the fork
    ZeroList zl{};
    for (uint32_t i = 0; i < num_jobs; ++i)
        if (jobs[i].err_count) zl.p[zl.count++] = jobs[i].err_count;
    if (zl.count) {
        k_zero_list<<<1, 32, 0, st>>>(zl);
        count_launch();
        if (cudaGetLastError() != cudaSuccess) return HD_ERR_CUDA;
    }
    if (cudaEventRecord(pool.fork, st) != cudaSuccess) return HD_ERR_CUDA;
    const int used = (int)std::min<uint32_t>(num_jobs, kPoolStreams);
    for (int i = 0; i < used; ++i)
        if (cudaStreamWaitEvent(pool.s[i], pool.fork, 0) != cudaSuccess) return HD_ERR_CUDA;
    // the largest streams first, so that the shorter ones fill in around them
    uint32_t order[kMaxStreamJobs];
    for (uint32_t i = 0; i < num_jobs; ++i) order[i] = i;
    std::sort(order, order + num_jobs, [&](uint32_t x, uint32_t y) {
        return (uint64_t)jobs[x].n * jobs[x].num_codewords > (uint64_t)jobs[y].n * jobs[y].num_codewords;
    });
    for (uint32_t r = 0; r < num_jobs; ++r) {
        const hd_stream_job &j = jobs[order[r]];
        if (j.num_codewords == 0) continue;
        const hd_status rc = enqueue_decode(j.stream, (uint64_t)j.n * j.num_codewords, j.n, j.num_codewords,
                                            j.out_bits, j.syndromes, static_cast<hd_syn_type>(j.syn_type),
                                            j.err_count, pool.s[r % kPoolStreams], false);
        if (rc != HD_OK) return rc;
    }
    for (int i = 0; i < used; ++i)
        if (cudaEventRecord(pool.join[i], pool.s[i]) != cudaSuccess ||
            cudaStreamWaitEvent(st, pool.join[i], 0) != cudaSuccess)
            return HD_ERR_CUDA;
    return HD_OK;
}

hd_status hd_encode(const uint32_t *data_bits, uint32_t n, uint64_t num_codewords, uint32_t *stream,
                    void *cuda_stream)
{
    const int m = code_m(n);
    if (m == 0) return HD_ERR_INVALID_N;
    if (num_codewords > (1ull << 40)) return HD_ERR_SIZE;
    if (num_codewords == 0) return HD_OK;
    if (!data_bits || !stream) return HD_ERR_NULL;
    if (!aligned16(data_bits) || !aligned16(stream)) return HD_ERR_ALIGN;
    const uint32_t k = n - (uint32_t)m;
    if (launch_encode_generic(data_bits, words_for_bits(num_codewords * k), n, num_codewords, stream,
                              words_for_bits(num_codewords * n), static_cast<cudaStream_t>(cuda_stream)) !=
        cudaSuccess)
        return HD_ERR_CUDA;
    return HD_OK;
}

}  // extern "C"
