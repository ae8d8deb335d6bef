// hd_serve.cu -- continuous-batching serving loop for arriving packets.
//
// A scheduler thread owns up to `max_waves` wave slots, each with its own CUDA
// stream, event and device tile table.  Submitted packets (already resident in
// device memory) wait in a bounded FIFO; whenever a slot is free the scheduler
// admits as many waiting packets as the slot's limits and the device-memory
// budget allow, cuts them into tiles and launches one batched decode on the
// slot's stream.  Waves on different slots run concurrently on the GPU, so
// packets that arrive while others are being decoded join the next free slot
// instead of waiting for the whole device to drain.  Completion is detected by
// polling the slot's event; the packet's error count comes back through a
// pinned host buffer copied on the same stream.
//
// This applies the paper's asynchronous pipelining idea (Sec. III-B: overlap
// the independent work of successive packets) to packets that are already in
// device memory: the overlap is between waves of decodes.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "hd_batch_internal.h"
#include "hd_internal.h"

namespace hd {
namespace {

using Clock = std::chrono::steady_clock;

uint64_t now_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Algorithmic bytes of one packet (input + output + syndromes) and its tile count.
bool packet_cost(const hd_packet &q, uint64_t *bytes, uint64_t *tiles, hd_status *err)
{
    const int m = code_m(q.n);
    if (m == 0) return *err = HD_ERR_INVALID_N, false;
    if (q.syn_type > 2) return *err = HD_ERR_INVALID_ARG, false;
    if (q.num_codewords > (1ull << 40)) return *err = HD_ERR_SIZE, false;
    if (q.num_codewords > 0) {
        if (!q.in || !q.out || (q.syn_type != 0 && !q.syndromes)) return *err = HD_ERR_NULL, false;
        if (!aligned16(q.in) || !aligned16(q.out) || (q.syn_type != 0 && !aligned16(q.syndromes)))
            return *err = HD_ERR_ALIGN, false;
    }
    const uint64_t N = q.num_codewords, k = q.n - (uint32_t)m;
    *bytes = (N * q.n + 7) / 8 + (N * k + 7) / 8 + N * (q.syn_type == 2 ? 2 : (q.syn_type == 1 ? 1 : 0));
    *tiles = packet_tiles(q.n, N);  // exactly as the batch plan cuts it
    return true;
}

struct Req {
    hd_packet pkt;
    uint64_t tag;
    uint64_t t_submit;
    uint64_t bytes;
    uint64_t tiles;
};

struct Wave {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    DevTile *d_tiles = nullptr;
    uint32_t *d_counter = nullptr;
    unsigned long long *d_err = nullptr;
    DevTile *h_tiles = nullptr;            // pinned staging of the tile table
    unsigned long long *h_err = nullptr;   // pinned copy of the error counts
    std::vector<Req> reqs;
    uint64_t bytes = 0;
    uint64_t t_admit = 0;
    bool busy = false;
};

}  // namespace
}  // namespace hd

using namespace hd;

struct hd_server {
    hd_server_config cfg;
    int device = 0;
    std::vector<Wave> waves;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req> pending;
    std::deque<hd_completion> done;
    uint64_t resident = 0;  // bytes of admitted, unfinished packets
    hd_server_stats stats;
    uint64_t wave_packets_sum = 0;
    std::thread worker;
    std::atomic<bool> stop{false};
    std::atomic<int> busy_waves{0};
    hd_status error = HD_OK;
};

namespace {

void release_waves(hd_server *s)
{
    for (Wave &w : s->waves) {
        if (w.st) cudaStreamSynchronize(w.st);
        if (w.ev) cudaEventDestroy(w.ev);
        if (w.st) cudaStreamDestroy(w.st);
        if (w.d_tiles) cudaFree(w.d_tiles);
        if (w.h_tiles) cudaFreeHost(w.h_tiles);
        if (w.h_err) cudaFreeHost(w.h_err);
        w = Wave();
    }
}

// Launch one wave from the requests in w.reqs; false on a CUDA failure.
bool launch_wave(hd_server *s, Wave &w)
{
    std::vector<hd_packet> table;
    table.reserve(w.reqs.size());
    for (const Req &r : w.reqs) table.push_back(r.pkt);
    std::vector<DevTile> tiles;
    if (build_tile_table(table.data(), (uint32_t)table.size(), tiles, nullptr) != HD_OK) return false;
    if (tiles.size() > s->cfg.max_wave_tiles) return false;  // admission bounds the tiles; never reached
    if (!tiles.empty()) std::memcpy(w.h_tiles, tiles.data(), tiles.size() * sizeof(DevTile));
    if (!tiles.empty() &&
        cudaMemcpyAsync(w.d_tiles, w.h_tiles, tiles.size() * sizeof(DevTile), cudaMemcpyHostToDevice, w.st) !=
            cudaSuccess)
        return false;
    if (launch_tile_table(w.d_tiles, (uint32_t)tiles.size(), w.d_counter, w.d_err, (uint32_t)table.size(), w.st) !=
        cudaSuccess)
        return false;
    if (cudaMemcpyAsync(w.h_err, w.d_err, table.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, w.st) !=
        cudaSuccess)
        return false;
    return cudaEventRecord(w.ev, w.st) == cudaSuccess;
}

void scheduler(hd_server *s)
{
    cudaSetDevice(s->device);
    for (;;) {
        bool progress = false;
        // 1. completions
        for (Wave &w : s->waves) {
            if (!w.busy) continue;
            const cudaError_t q = cudaEventQuery(w.ev);
            if (q == cudaErrorNotReady) continue;
            const uint64_t t = now_ns();
            std::lock_guard<std::mutex> lk(s->mu);
            for (size_t j = 0; j < w.reqs.size(); ++j) {
                hd_completion c;
                c.tag = w.reqs[j].tag;
                c.err_count = q == cudaSuccess ? w.h_err[j] : 0;
                c.t_submit_ns = w.reqs[j].t_submit;
                c.t_admit_ns = w.t_admit;
                c.t_done_ns = t;
                c.status = q == cudaSuccess ? HD_OK : HD_ERR_CUDA;
                s->done.push_back(c);
            }
            if (q != cudaSuccess) s->error = HD_ERR_CUDA;
            s->stats.completed += w.reqs.size();
            s->resident -= w.bytes;
            w.reqs.clear();
            w.bytes = 0;
            w.busy = false;
            s->busy_waves.fetch_sub(1);
            progress = true;
        }
        // 2. admission: fill every free slot from the FIFO, within the budget
        for (Wave &w : s->waves) {
            if (w.busy) continue;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                uint64_t tiles = 0;
                while (!s->pending.empty() && w.reqs.size() < s->cfg.max_wave_packets) {
                    const Req &r = s->pending.front();
                    if (s->resident + w.bytes + r.bytes > s->cfg.mem_cap_bytes) break;
                    if (!w.reqs.empty() && tiles + r.tiles > s->cfg.max_wave_tiles) break;
                    tiles += r.tiles;
                    w.bytes += r.bytes;
                    w.reqs.push_back(r);
                    s->pending.pop_front();
                }
                if (w.reqs.empty()) break;
                s->resident += w.bytes;
                s->stats.max_resident_bytes = std::max(s->stats.max_resident_bytes, s->resident);
                s->stats.waves += 1;
                s->wave_packets_sum += w.reqs.size();
                // busy before the lock is released: hd_server_drain() must never see these
                // requests neither pending nor in a busy wave
                w.busy = true;
                s->busy_waves.fetch_add(1);
            }
            w.t_admit = now_ns();
            if (!launch_wave(s, w)) {
                std::lock_guard<std::mutex> lk(s->mu);
                s->error = HD_ERR_CUDA;
            }
            progress = true;
        }
        if (progress) continue;
        if (s->busy_waves.load() > 0) {
            std::this_thread::yield();  // a wave is on the GPU: poll its event again soon
            continue;
        }
        std::unique_lock<std::mutex> lk(s->mu);
        if (s->stop.load() && s->pending.empty()) break;
        s->cv.wait_for(lk, std::chrono::milliseconds(5), [&] { return s->stop.load() || !s->pending.empty(); });
    }
}

}  // namespace

extern "C" {

hd_status hd_server_create(const hd_server_config *cfg, hd_server **out)
{
    if (!cfg || !out) return HD_ERR_NULL;
    *out = nullptr;
    if (cfg->max_waves == 0 || cfg->max_waves > 64 || cfg->max_wave_packets == 0 || cfg->max_wave_tiles == 0 ||
        cfg->queue_capacity == 0 || cfg->mem_cap_bytes == 0)
        return HD_ERR_INVALID_ARG;
    hd_server *s = new (std::nothrow) hd_server();
    if (!s) return HD_ERR_CAPACITY;
    s->cfg = *cfg;
    std::memset(&s->stats, 0, sizeof(s->stats));
    cudaGetDevice(&s->device);
    s->waves.resize(cfg->max_waves);
    for (Wave &w : s->waves) {
        const size_t tb = (size_t)cfg->max_wave_tiles * sizeof(DevTile);
        const size_t eb = (size_t)cfg->max_wave_packets * sizeof(unsigned long long);
        char *d = nullptr;
        if (cudaStreamCreateWithFlags(&w.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&w.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaMalloc(&d, tb + 256 + eb) != cudaSuccess ||
            cudaMallocHost(&w.h_tiles, tb) != cudaSuccess || cudaMallocHost(&w.h_err, eb) != cudaSuccess) {
            if (d) cudaFree(d);
            release_waves(s);
            delete s;
            return HD_ERR_CUDA;
        }
        w.d_tiles = reinterpret_cast<DevTile *>(d);
        w.d_counter = reinterpret_cast<uint32_t *>(d + tb);
        w.d_err = reinterpret_cast<unsigned long long *>(d + tb + 256);
    }
    s->worker = std::thread(scheduler, s);
    *out = s;
    return HD_OK;
}

hd_status hd_server_submit(hd_server *s, const hd_packet *pkt, uint64_t tag)
{
    if (!s || !pkt) return HD_ERR_NULL;
    Req r;
    hd_status err = HD_OK;
    if (!packet_cost(*pkt, &r.bytes, &r.tiles, &err)) return err;
    if (r.bytes > s->cfg.mem_cap_bytes || r.tiles > s->cfg.max_wave_tiles) return HD_ERR_CAPACITY;
    r.pkt = *pkt;
    if (!pkt->syndromes) r.pkt.syn_type = HD_SYN_NONE;
    r.tag = tag;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->error != HD_OK) return s->error;
        if (s->pending.size() >= s->cfg.queue_capacity) {
            s->stats.rejected += 1;
            return HD_ERR_CAPACITY;
        }
        r.t_submit = now_ns();
        s->pending.push_back(r);
        s->stats.submitted += 1;
    }
    s->cv.notify_one();
    return HD_OK;
}

hd_status hd_server_poll(hd_server *s, hd_completion *out, uint32_t max, uint32_t *count)
{
    if (!s || !count || (max > 0 && !out)) return HD_ERR_NULL;
    std::lock_guard<std::mutex> lk(s->mu);
    uint32_t c = 0;
    while (c < max && !s->done.empty()) {
        out[c++] = s->done.front();
        s->done.pop_front();
    }
    *count = c;
    return s->error;
}

hd_status hd_server_drain(hd_server *s, uint64_t timeout_ns)
{
    if (!s) return HD_ERR_NULL;
    const uint64_t t0 = now_ns();
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->error != HD_OK) return s->error;
            if (s->pending.empty() && s->busy_waves.load() == 0) return HD_OK;
        }
        if (now_ns() - t0 > timeout_ns) return HD_ERR_TIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

hd_status hd_server_get_stats(hd_server *s, hd_server_stats *stats)
{
    if (!s || !stats) return HD_ERR_NULL;
    std::lock_guard<std::mutex> lk(s->mu);
    *stats = s->stats;
    stats->mean_wave_packets = s->stats.waves ? (double)s->wave_packets_sum / (double)s->stats.waves : 0.0;
    return HD_OK;
}

void hd_server_destroy(hd_server *s)
{
    if (!s) return;
    s->stop.store(true);
    s->cv.notify_all();
    // let the scheduler finish what was admitted and submitted
    if (s->worker.joinable()) s->worker.join();
    release_waves(s);
    delete s;
}

hd_status hd_serve_trace(const hd_server_config *cfg, const hd_packet *pkts, const double *arrival_s, uint32_t num,
                         hd_completion *completions, hd_server_stats *stats)
{
    if (!cfg || (num > 0 && (!pkts || !arrival_s || !completions)) || !stats) return HD_ERR_NULL;
    for (uint32_t j = 1; j < num; ++j)
        if (arrival_s[j] < arrival_s[j - 1]) return HD_ERR_INVALID_ARG;
    hd_server *s = nullptr;
    hd_status rc = hd_server_create(cfg, &s);
    if (rc != HD_OK) return rc;
    std::vector<uint64_t> scheduled(num);
    std::vector<hd_completion> buf(4096);
    uint32_t got = 0;
    auto collect = [&]() {
        uint32_t c = 0;
        hd_status e = hd_server_poll(s, buf.data(), (uint32_t)buf.size(), &c);
        for (uint32_t i = 0; i < c; ++i) {
            const uint64_t tag = buf[i].tag;
            if (tag < num) completions[tag] = buf[i];
        }
        got += c;
        return e;
    };
    const uint64_t t0 = now_ns() + 1000000;  // first arrival 1 ms from now
    uint64_t backpressure = 0;
    for (uint32_t j = 0; j < num && rc == HD_OK; ++j) {
        scheduled[j] = t0 + (uint64_t)(arrival_s[j] * 1e9);
        // wait for the arrival time: sleep through long gaps, spin the last stretch
        for (;;) {
            const uint64_t t = now_ns();
            if (t >= scheduled[j]) break;
            if (scheduled[j] - t > 300000) std::this_thread::sleep_for(std::chrono::microseconds(100));
            else std::this_thread::yield();
        }
        for (;;) {
            const hd_status e = hd_server_submit(s, &pkts[j], j);
            if (e == HD_OK) break;
            if (e != HD_ERR_CAPACITY) {
                rc = e;
                break;
            }
            ++backpressure;  // queue full: the arrival waits for room
            collect();
            std::this_thread::yield();
        }
        if ((j & 255) == 0) collect();
    }
    if (rc == HD_OK) rc = hd_server_drain(s, 600ull * 1000000000ull);
    while (got < num && rc == HD_OK) {
        const uint32_t before = got;
        rc = collect();
        if (got == before) break;
    }
    hd_server_get_stats(s, stats);
    hd_server_destroy(s);
    if (rc != HD_OK) return rc;
    if (got != num) return HD_ERR_CUDA;
    // latency from the scheduled arrival to the host observing completion
    std::vector<double> lat(num);
    uint64_t first = num ? scheduled[0] : 0, last = 0;
    for (uint32_t j = 0; j < num; ++j) {
        lat[j] = (double)(completions[j].t_done_ns - scheduled[j]) * 1e-3;
        last = std::max(last, completions[j].t_done_ns);
    }
    auto pct = [&](double p) {
        if (lat.empty()) return 0.0;
        size_t i = (size_t)std::min<double>((double)lat.size() - 1, p * (double)(lat.size() - 1) + 0.5);
        std::nth_element(lat.begin(), lat.begin() + (long)i, lat.end());
        return lat[i];
    };
    stats->p50_latency_us = pct(0.50);
    stats->p99_latency_us = pct(0.99);
    stats->max_latency_us = num ? *std::max_element(lat.begin(), lat.end()) : 0.0;
    stats->duration_s = num ? (double)(last - first) * 1e-9 : 0.0;
    stats->backpressure_waits = backpressure;
    return HD_OK;
}

}  // extern "C"
