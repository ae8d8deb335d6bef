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
// polling the slot's event; the packets' error counts and the wave's own
// device status word come back through a pinned host buffer copied on the
// same stream.
//
// Packets can also be submitted from pinned host memory (an SDR receive path
// gets its packets there).  A wave that carries such packets gathers them into
// the slot's device staging with one copy kernel (T_PS), decodes (T_DKE) and
// scatters data bits and syndromes back into the caller's host buffers with a
// second copy kernel (T_PR), all on the slot's stream; events between the
// stages time them.  Waves on different slots overlap, so one wave's
// transfers run beside another's decode: the paper's asynchronous data
// transfer (Sec. III-B, Fig. 5, Eq. 1) applied to a stream of arriving
// packets.
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
    hd_packet pkt;   // as submitted (host pointers for a host packet)
    uint64_t tag;
    uint64_t t_submit;
    uint64_t bytes;  // algorithmic bytes (input + output + syndromes)
    uint64_t tiles;
    bool host = false;
    // host packets: device-accessible addresses of the caller's pinned buffers,
    // their exact sizes, and the staging they take (each part 16-byte rounded)
    const void *dev_in = nullptr;
    void *dev_out = nullptr, *dev_syn = nullptr;
    uint64_t in_b = 0, out_b = 0, syn_b = 0, stage_b = 0;
};

inline uint64_t round16(uint64_t b) { return (b + 15) & ~15ull; }

// A wave's table region, in device memory and in its pinned upload image
// alike: the status word (offset 0) and the claim counter (offset 16), the
// packets' error counts (offset 32), the tiles (64-byte aligned) and the copy
// pieces.  Status, counter and counts are zero in the image, so that one copy
// uploads the tables and clears everything the kernels accumulate into.
constexpr size_t kOffCounter = 16, kOffErr = 32;
inline size_t tiles_offset(size_t packets) { return (kOffErr + packets * 8 + 63) & ~size_t(63); }

// Stage times are taken (four timing events) on one host wave in this many.
constexpr uint64_t kTimeEvery = 4;

struct Wave {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;                // completion
    cudaEvent_t t0 = nullptr, t1 = nullptr;  // stage timing of sampled host waves: before and after the gather,
    cudaEvent_t t2 = nullptr, t3 = nullptr;  // after the decode and after the scatter
    char *dmem = nullptr;                    // the table region, then the staging of host packets
    unsigned char *d_stage = nullptr;
    char *h_up = nullptr;                    // pinned upload image of the table region
    char *h_back = nullptr;                  // pinned: status word, counter, error counts
    std::vector<Req> reqs;
    uint64_t bytes = 0;
    uint64_t stage_used = 0;
    uint64_t t_admit = 0;
    bool busy = false;
    bool host = false;                       // carries host packets
    bool timed = false;                      // its stages are timed
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
    std::atomic<uint32_t> inject_failures{0};  // test hook: wave launches to fail on the host
    hd_status error = HD_OK;
    uint64_t pieces_cap = 0;                    // copy pieces per wave
    size_t table_cap = 0;                       // bytes of a wave's table region
    uint64_t host_launched = 0;                 // host waves launched (every kTimeEvery-th is timed)
    uint64_t timed_waves = 0;
    double t_in_us = 0, t_dec_us = 0, t_out_us = 0;  // summed stage times of the timed host waves
};

namespace {

void release_waves(hd_server *s)
{
    for (Wave &w : s->waves) {
        if (w.st) cudaStreamSynchronize(w.st);
        for (cudaEvent_t e : {w.ev, w.t0, w.t1, w.t2, w.t3})
            if (e) cudaEventDestroy(e);
        if (w.st) cudaStreamDestroy(w.st);
        if (w.dmem) cudaFree(w.dmem);
        if (w.h_up) cudaFreeHost(w.h_up);
        if (w.h_back) cudaFreeHost(w.h_back);
        w = Wave();
    }
}

// Launch one wave from the requests in w.reqs; false on a CUDA failure.
bool launch_wave(hd_server *s, Wave &w)
{
    // test hook: fail as a launch error would, before anything is enqueued
    for (uint32_t f = s->inject_failures.load(); f > 0;)
        if (s->inject_failures.compare_exchange_weak(f, f - 1)) return false;
    // the batch table: device packets as submitted, host packets pointed at
    // their part of the slot's staging; copy pieces for the host packets
    std::vector<hd_packet> table;
    table.reserve(w.reqs.size());
    std::vector<CopyPiece> gin, gout;
    uint64_t off = 0;
    for (const Req &r : w.reqs) {
        hd_packet q = r.pkt;
        if (r.host) {
            unsigned char *din = w.d_stage + off;
            unsigned char *dout = din + round16(r.in_b);
            unsigned char *dsyn = dout + round16(r.out_b);
            off += r.stage_b;
            add_copy_pieces(gin, r.dev_in, din, r.in_b);
            add_copy_pieces(gout, dout, r.dev_out, r.out_b);
            if (r.syn_b) add_copy_pieces(gout, dsyn, r.dev_syn, r.syn_b);
            q.in = reinterpret_cast<const uint32_t *>(din);
            q.out = reinterpret_cast<uint32_t *>(dout);
            q.syndromes = r.syn_b ? dsyn : nullptr;
            if (!r.syn_b) q.syn_type = HD_SYN_NONE;
        }
        table.push_back(q);
    }
    std::vector<DevTile> tiles;
    if (build_tile_table(table.data(), (uint32_t)table.size(), tiles, nullptr) != HD_OK) return false;
    if (tiles.size() > s->cfg.max_wave_tiles) return false;  // admission bounds the tiles; never reached
    if (gin.size() + gout.size() > s->pieces_cap) return false;  // bounded by the staging; never reached
    // the upload image: zeroed status, counter and counts, then tiles and pieces
    const size_t toff = tiles_offset(table.size());
    const size_t poff = toff + tiles.size() * sizeof(DevTile);
    const size_t used = poff + (gin.size() + gout.size()) * sizeof(CopyPiece);
    std::memset(w.h_up, 0, toff);
    if (!tiles.empty()) std::memcpy(w.h_up + toff, tiles.data(), tiles.size() * sizeof(DevTile));
    if (!gin.empty()) std::memcpy(w.h_up + poff, gin.data(), gin.size() * sizeof(CopyPiece));
    if (!gout.empty())
        std::memcpy(w.h_up + poff + gin.size() * sizeof(CopyPiece), gout.data(), gout.size() * sizeof(CopyPiece));
    if (cudaMemcpyAsync(w.dmem, w.h_up, used, cudaMemcpyHostToDevice, w.st) != cudaSuccess) return false;
    uint32_t *d_status = reinterpret_cast<uint32_t *>(w.dmem);
    const CopyPiece *d_pieces = reinterpret_cast<const CopyPiece *>(w.dmem + poff);
    w.host = !gin.empty();
    w.timed = w.host && (s->host_launched++ % kTimeEvery) == 0;
    if (w.host) {
        if ((w.timed && cudaEventRecord(w.t0, w.st) != cudaSuccess) ||
            launch_copy_pieces(d_pieces, (uint32_t)gin.size(), w.st) != cudaSuccess ||
            (w.timed && cudaEventRecord(w.t1, w.st) != cudaSuccess))
            return false;
    }
    if (launch_tile_table(reinterpret_cast<const DevTile *>(w.dmem + toff), (uint32_t)tiles.size(),
                          reinterpret_cast<uint32_t *>(w.dmem + kOffCounter),
                          reinterpret_cast<unsigned long long *>(w.dmem + kOffErr), (uint32_t)table.size(), w.st,
                          d_status, false) != cudaSuccess)
        return false;
    if (w.host) {
        if ((w.timed && cudaEventRecord(w.t2, w.st) != cudaSuccess) ||
            launch_copy_pieces(d_pieces + gin.size(), (uint32_t)gout.size(), w.st) != cudaSuccess ||
            (w.timed && cudaEventRecord(w.t3, w.st) != cudaSuccess))
            return false;
    }
    // the status word and the packets' error counts in one copy
    if (cudaMemcpyAsync(w.h_back, w.dmem, kOffErr + table.size() * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, w.st) != cudaSuccess)
        return false;
    return cudaEventRecord(w.ev, w.st) == cudaSuccess;
}

// Hand the wave's packets back with `status` (the counts only when HD_OK or a
// timeout) and free its slot and budget.  Called with s->mu held.
void complete_wave(hd_server *s, Wave &w, hd_status status, uint64_t t)
{
    const unsigned long long *cnt = reinterpret_cast<const unsigned long long *>(w.h_back + kOffErr);
    for (size_t j = 0; j < w.reqs.size(); ++j) {
        hd_completion c;
        c.tag = w.reqs[j].tag;
        c.err_count = status == HD_OK ? cnt[j] : 0;
        c.t_submit_ns = w.reqs[j].t_submit;
        c.t_admit_ns = w.t_admit;
        c.t_done_ns = t;
        c.status = status;
        s->done.push_back(c);
    }
    s->stats.completed += w.reqs.size();
    s->resident -= w.bytes;
    w.reqs.clear();
    w.bytes = 0;
    w.stage_used = 0;
    w.host = false;
    w.timed = false;
    w.busy = false;
    s->busy_waves.fetch_sub(1);
}

// After a CUDA failure the server stops admitting: every packet still
// waiting completes with the server's error.  Called with s->mu held.
void fail_pending(hd_server *s, uint64_t t)
{
    while (!s->pending.empty()) {
        const Req &r = s->pending.front();
        hd_completion c;
        c.tag = r.tag;
        c.err_count = 0;
        c.t_submit_ns = r.t_submit;
        c.t_admit_ns = 0;
        c.t_done_ns = t;
        c.status = s->error;
        s->done.push_back(c);
        s->stats.completed += 1;
        s->pending.pop_front();
    }
}

void scheduler(hd_server *s)
{
    cudaSetDevice(s->device);
    // after the last activity, poll for this long before sleeping on the
    // condition variable, so that an arrival shortly after a completion does
    // not pay a thread wake-up
    constexpr uint64_t kSpinNs = 200000;
    uint64_t last_active = now_ns();
    for (;;) {
        bool progress = false;
        // 1. completions
        for (Wave &w : s->waves) {
            if (!w.busy) continue;
            const cudaError_t q = cudaEventQuery(w.ev);
            if (q == cudaErrorNotReady) continue;
            const uint64_t t = now_ns();
            float a = 0.f, b = 0.f, c = 0.f;
            const bool timed = q == cudaSuccess && w.timed && cudaEventElapsedTime(&a, w.t0, w.t1) == cudaSuccess &&
                               cudaEventElapsedTime(&b, w.t1, w.t2) == cudaSuccess &&
                               cudaEventElapsedTime(&c, w.t2, w.t3) == cudaSuccess;
            std::lock_guard<std::mutex> lk(s->mu);
            hd_status st = HD_OK;
            if (q != cudaSuccess) {
                st = HD_ERR_CUDA;
                s->error = HD_ERR_CUDA;
            } else if (*reinterpret_cast<const uint32_t *>(w.h_back) != 0) {
                st = HD_ERR_TIMEOUT;  // a bounded wait of this wave's kernel ran out
            }
            if (w.host) s->stats.host_waves += 1;
            if (timed) {
                s->timed_waves += 1;
                s->t_in_us += 1000.0 * a;
                s->t_dec_us += 1000.0 * b;
                s->t_out_us += 1000.0 * c;
            }
            complete_wave(s, w, st, t);
            if (s->error != HD_OK) fail_pending(s, t);
            progress = true;
        }
        // 2. admission: fill every free slot from the FIFO, within the budget
        for (Wave &w : s->waves) {
            if (w.busy) continue;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                if (s->error != HD_OK) break;
                uint64_t tiles = 0;
                while (!s->pending.empty() && w.reqs.size() < s->cfg.max_wave_packets) {
                    const Req &r = s->pending.front();
                    if (s->resident + w.bytes + r.bytes > s->cfg.mem_cap_bytes) break;
                    if (!w.reqs.empty() && tiles + r.tiles > s->cfg.max_wave_tiles) break;
                    if (r.host && w.stage_used + r.stage_b > s->cfg.host_staging_bytes) break;
                    tiles += r.tiles;
                    w.bytes += r.bytes;
                    if (r.host) w.stage_used += r.stage_b;
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
                // nothing of this wave is trusted: its packets fail now, and so does
                // every packet still waiting (the server keeps the error)
                const uint64_t t = now_ns();
                std::lock_guard<std::mutex> lk(s->mu);
                s->error = HD_ERR_CUDA;
                complete_wave(s, w, HD_ERR_CUDA, t);
                fail_pending(s, t);
            }
            progress = true;
        }
        const uint64_t now = now_ns();
        if (progress) {
            last_active = now;
            continue;
        }
        if (s->busy_waves.load() > 0 || now - last_active < kSpinNs) {
            std::this_thread::yield();  // a wave is on the GPU, or an arrival may be near: poll again soon
            continue;
        }
        std::unique_lock<std::mutex> lk(s->mu);
        if (s->stop.load() && s->pending.empty()) break;
        s->cv.wait_for(lk, std::chrono::milliseconds(5), [&] { return s->stop.load() || !s->pending.empty(); });
        last_active = now_ns();
    }
}

// Validate a host packet: its buffers must be pinned host memory that kernels
// can reach (cudaPointerGetAttributes gives their device-accessible address).
hd_status host_buffer(const void *p, const void **dev)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return HD_ERR_INVALID_ARG;
    }
    if (a.type != cudaMemoryTypeHost || a.devicePointer == nullptr) return HD_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(a.devicePointer) & 15u) != 0) return HD_ERR_ALIGN;
    *dev = a.devicePointer;
    return HD_OK;
}

hd_status enqueue_req(hd_server *s, Req &r)
{
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

hd_status serve_trace(const hd_server_config *cfg, const hd_packet *pkts, const double *arrival_s, uint32_t num,
                      hd_completion *completions, hd_server_stats *stats, bool host)
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
            const hd_status e = host ? hd_server_submit_host(s, &pkts[j], j) : hd_server_submit(s, &pkts[j], j);
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
    // how late the generator itself submitted (a sleeping thread woken late by
    // the operating system), to tell such delays from the server's
    double lag = 0.0;
    for (uint32_t j = 0; j < num; ++j)
        lag = std::max(lag, (double)((int64_t)completions[j].t_submit_ns - (int64_t)scheduled[j]) * 1e-3);
    stats->max_submit_lag_us = lag;
    stats->max_latency_us = num ? *std::max_element(lat.begin(), lat.end()) : 0.0;
    stats->p50_latency_us = pct(0.50);
    stats->p99_latency_us = pct(0.99);
    stats->p999_latency_us = pct(0.999);
    stats->duration_s = num ? (double)(last - first) * 1e-9 : 0.0;
    stats->backpressure_waits = backpressure;
    return HD_OK;
}

}  // namespace

extern "C" {

hd_status hd_server_create(const hd_server_config *cfg, hd_server **out)
{
    if (!cfg || !out) return HD_ERR_NULL;
    *out = nullptr;
    if (cfg->max_waves == 0 || cfg->max_waves > 64 || cfg->max_wave_packets == 0 || cfg->max_wave_tiles == 0 ||
        cfg->queue_capacity == 0 || cfg->mem_cap_bytes == 0 || cfg->host_staging_bytes > (1ull << 40))
        return HD_ERR_INVALID_ARG;
    hd_server *s = new (std::nothrow) hd_server();
    if (!s) return HD_ERR_CAPACITY;
    s->cfg = *cfg;
    std::memset(&s->stats, 0, sizeof(s->stats));
    cudaGetDevice(&s->device);
    // pieces of a wave: at most one per kPieceBytes of staging plus three
    // partial ones (input, output, syndromes) per packet
    s->pieces_cap = cfg->host_staging_bytes ? cfg->host_staging_bytes / kPieceBytes + 3ull * cfg->max_wave_packets : 0;
    s->table_cap = tiles_offset(cfg->max_wave_packets) + (size_t)cfg->max_wave_tiles * sizeof(DevTile) +
                   (size_t)s->pieces_cap * sizeof(CopyPiece);
    const size_t tr = (s->table_cap + 255) / 256 * 256;
    const size_t sb = (size_t)((cfg->host_staging_bytes + 255) / 256 * 256);
    const size_t bb = kOffErr + (size_t)cfg->max_wave_packets * sizeof(unsigned long long);
    s->waves.resize(cfg->max_waves);
    bool ok = true;
    for (Wave &w : s->waves) {
        ok = cudaStreamCreateWithFlags(&w.st, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&w.ev, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreate(&w.t0) == cudaSuccess && cudaEventCreate(&w.t1) == cudaSuccess &&
             cudaEventCreate(&w.t2) == cudaSuccess && cudaEventCreate(&w.t3) == cudaSuccess &&
             cudaMalloc(&w.dmem, tr + sb) == cudaSuccess && cudaMallocHost(&w.h_up, s->table_cap) == cudaSuccess &&
             cudaMallocHost(&w.h_back, bb) == cudaSuccess;
        if (!ok) break;
        w.d_stage = reinterpret_cast<unsigned char *>(w.dmem + tr);
        // one-time set-up of the batch kernel (attributes, occupancy, the n = 7
        // table) now, so that the first wave pays none of it
        ok = launch_tile_table(reinterpret_cast<const DevTile *>(w.dmem + tiles_offset(0)), 0,
                               reinterpret_cast<uint32_t *>(w.dmem + kOffCounter), nullptr, 0, w.st,
                               reinterpret_cast<uint32_t *>(w.dmem)) == cudaSuccess &&
             cudaStreamSynchronize(w.st) == cudaSuccess;
        if (!ok) break;
    }
    if (!ok) {
        release_waves(s);
        delete s;
        return HD_ERR_CUDA;
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
    return enqueue_req(s, r);
}

hd_status hd_server_submit_host(hd_server *s, const hd_packet *pkt, uint64_t tag)
{
    if (!s || !pkt) return HD_ERR_NULL;
    if (s->cfg.host_staging_bytes == 0) return HD_ERR_INVALID_ARG;
    Req r;
    hd_status err = HD_OK;
    if (!packet_cost(*pkt, &r.bytes, &r.tiles, &err)) return err;
    r.pkt = *pkt;
    if (!pkt->syndromes) r.pkt.syn_type = HD_SYN_NONE;
    r.tag = tag;
    r.host = true;
    const uint64_t N = pkt->num_codewords, m = (uint64_t)code_m(pkt->n), k = pkt->n - m;
    r.in_b = words_for_bits(N * pkt->n) * 4;
    r.out_b = words_for_bits(N * k) * 4;
    r.syn_b = N * (r.pkt.syn_type == HD_SYN_U16 ? 2u : (r.pkt.syn_type == HD_SYN_U8 ? 1u : 0u));
    r.stage_b = round16(r.in_b) + round16(r.out_b) + round16(r.syn_b);
    if (N > 0) {
        void *dv = nullptr;
        if ((err = host_buffer(pkt->in, &r.dev_in)) != HD_OK) return err;
        if ((err = host_buffer(pkt->out, const_cast<const void **>(&dv))) != HD_OK) return err;
        r.dev_out = dv;
        if (r.syn_b) {
            if ((err = host_buffer(pkt->syndromes, const_cast<const void **>(&dv))) != HD_OK) return err;
            r.dev_syn = dv;
        }
    }
    if (r.bytes > s->cfg.mem_cap_bytes || r.tiles > s->cfg.max_wave_tiles || r.stage_b > s->cfg.host_staging_bytes)
        return HD_ERR_CAPACITY;
    return enqueue_req(s, r);
}

hd_status hd_server_inject_launch_failures(hd_server *s, uint32_t count)
{
    if (!s) return HD_ERR_NULL;
    s->inject_failures.store(count);
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
    const double hw = (double)s->timed_waves;
    stats->mean_t_in_us = hw > 0 ? s->t_in_us / hw : 0.0;
    stats->mean_t_decode_us = hw > 0 ? s->t_dec_us / hw : 0.0;
    stats->mean_t_out_us = hw > 0 ? s->t_out_us / hw : 0.0;
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
    return serve_trace(cfg, pkts, arrival_s, num, completions, stats, false);
}

hd_status hd_serve_trace_host(const hd_server_config *cfg, const hd_packet *pkts, const double *arrival_s,
                              uint32_t num, hd_completion *completions, hd_server_stats *stats)
{
    return serve_trace(cfg, pkts, arrival_s, num, completions, stats, true);
}

}  // extern "C"
