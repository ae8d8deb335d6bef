// hd_batch_internal.h -- the batched decoder's tile table, shared by the
// batch entry points (hd_batch.cu) and the serving engine (hd_serve.cu).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "hd.h"

namespace hd {

// A self-contained work item: everything a warp needs to decode it, so that
// the warp never chases a second table.
struct DevTile {
    const uint32_t *in;  // packet input (word 0 = codeword 0)
    uint32_t *out;       // packet output
    uint8_t *syn;        // packet syndromes (NULL when syn_type is 0)
    uint64_t num_cw;     // packet length in codewords
    uint64_t c0;         // first codeword of the tile (a multiple of 32)
    uint32_t packet;     // index into err_counts
    uint32_t count;      // codewords, | kFullTile for whole chunks of 32*G decoded by the chunk decoder
    uint32_t bytes;      // bulk-load size of a full tile (0 for a tail)
    uint16_t n;
    uint8_t m;
    uint8_t syn_type;
    uint64_t pad;
};

constexpr uint32_t kFullTile = 0x80000000u;

inline DevTile make_tile(const uint32_t *in, uint32_t *out, uint8_t *syn, uint64_t num_cw, uint32_t n, uint32_t m,
                         uint32_t syn_type, uint32_t packet, uint64_t c0, uint32_t count, uint32_t bytes)
{
    DevTile t;
    t.in = in;
    t.out = out;
    t.syn = syn;
    t.num_cw = num_cw;
    t.c0 = c0;
    t.packet = packet;
    t.count = count;
    t.bytes = bytes;
    t.n = (uint16_t)n;
    t.m = (uint8_t)m;
    t.syn_type = (uint8_t)syn_type;
    t.pad = 0;
    return t;
}

// Exact number of tiles the batch plan cuts a packet of code length n and
// num_codewords codewords into (n must be a supported length).
uint64_t packet_tiles(uint32_t n, uint64_t num_codewords);

// Validate a packet table and cut it into tiles (grouped by n, long codes
// first, each code's ragged tails spread among its full tiles).  Adds the packets' algorithmic
// bytes (input + output + syndromes) to *bytes when not NULL.
hd_status build_tile_table(const hd_packet *table, uint32_t num_packets, std::vector<DevTile> &tiles,
                           uint64_t *bytes);

// Enqueue one batched decode of a device tile table on `st`: clear the claim
// counter and the error counters (when err is not NULL), then launch the batch
// kernel in its default configuration.  Host-side setup (kernel attributes,
// occupancy, status word) happens on the first call per device.  A timeout
// is latched into `status` (device) when not NULL, else into the device's
// status word.  num_tiles = 0 performs only the set-up and the clears.  With
// clear = false the caller has already zeroed the claim counter and the error
// counters (for example in the same copy that uploaded the table).
cudaError_t launch_tile_table(const DevTile *d_tiles, uint32_t num_tiles, uint32_t *d_counter,
                              unsigned long long *d_err, uint32_t num_packets, cudaStream_t st,
                              uint32_t *status = nullptr, bool clear = true);

// A contiguous copy of at most kPieceBytes between two 16-byte aligned
// addresses that kernels can dereference (device memory, or pinned host memory
// through its device-accessible address).
struct CopyPiece {
    const void *src;
    void *dst;
    uint32_t bytes;
    uint32_t pad;
};

constexpr uint32_t kPieceBytes = 8192;

// Cut a copy of `bytes` into pieces appended to `out`.
inline void add_copy_pieces(std::vector<CopyPiece> &out, const void *src, void *dst, uint64_t bytes)
{
    for (uint64_t o = 0; o < bytes; o += kPieceBytes) {
        CopyPiece p;
        p.src = static_cast<const unsigned char *>(src) + o;
        p.dst = static_cast<unsigned char *>(dst) + o;
        p.bytes = (uint32_t)((bytes - o) < kPieceBytes ? (bytes - o) : kPieceBytes);
        p.pad = 0;
        out.push_back(p);
    }
}

// Copy every piece of a device table of `count` pieces (one CTA per piece,
// 16-byte vector loads and stores; the last bytes of a piece that is not a
// multiple of 16 are copied one by one, so nothing past `bytes` is touched).
cudaError_t launch_copy_pieces(const CopyPiece *d_pieces, uint32_t count, cudaStream_t st);

}  // namespace hd
