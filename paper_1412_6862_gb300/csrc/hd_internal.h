// hd_internal.h -- host-side declarations shared by the translation units of
// libhd.so.  Not installed; the public interface is include/hd.h.
#pragma once

#include <atomic>
#include <cstdint>
#include <utility>
#include <cuda_runtime.h>

#include "hd.h"

namespace hd {

// Kernels launched by this library (hd_launch_count()).
extern std::atomic<uint64_t> g_launches;
inline void count_launch(uint64_t c = 1) { g_launches.fetch_add(c, std::memory_order_relaxed); }

// m for n = 2^m - 1 (2 <= m <= 8), else 0.
inline int code_m(uint32_t n)
{
    for (int m = 2; m <= 8; ++m)
        if (n == (1u << m) - 1u) return m;
    return 0;
}

inline uint64_t words_for_bits(uint64_t bits) { return (bits + 31) >> 5; }

// Multiprocessor count of the current device (cached per device).
int num_sms();

// Upper bound on the CTAs of one decode launch (hd_set_max_ctas(); 0 = none).
extern std::atomic<uint32_t> g_max_ctas;

// Grid of a decode launch: `want` CTAs (enough for the work), at most `cap`
// (what the device holds at once) and at most the caller's limit; at least 1.
inline int decode_grid(uint64_t want, uint64_t cap)
{
    uint64_t g = want < cap ? want : cap;
    const uint32_t lim = g_max_ctas.load(std::memory_order_relaxed);
    if (lim != 0 && g > lim) g = lim;
    return (int)(g > 0 ? g : 1);
}

// Generic warp-tile kernels (any supported n).  Warp tile t covers codewords
// [32t, 32t+32); the launch covers warp tiles [tile_begin, tile_end).
cudaError_t launch_decode_generic(const uint32_t *in, uint64_t in_words, uint32_t n, uint64_t num_cw,
                                  uint64_t tile_begin, uint64_t tile_end, uint32_t *out, uint64_t out_words,
                                  void *syn, int syn_type, unsigned long long *err, cudaStream_t st);
cudaError_t launch_encode_generic(const uint32_t *data, uint64_t data_words, uint32_t n, uint64_t num_cw,
                                  uint32_t *stream, uint64_t stream_words, cudaStream_t st);

// Launch `kern` on `st`, as the programmatic dependent of the kernel ahead of
// it in the stream when pdl is set (it may then start before that kernel has
// finished, and must wait for it before touching what that kernel writes).
template <typename... KArgs, typename... Args>
cudaError_t launch_kernel_uncounted(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                    bool pdl, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? &attr : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// launch_kernel_uncounted, counted in hd_launch_count().
template <typename... KArgs, typename... Args>
cudaError_t launch_kernel(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool pdl,
                          Args &&...args)
{
    count_launch();
    return launch_kernel_uncounted(kern, grid, block, smem, st, pdl, std::forward<Args>(args)...);
}

// Clear one or two device counters (either may be NULL) with a one-thread
// kernel that lets the next kernel of the stream start at once (programmatic
// dependent launch): a launch with pdl = true below overlaps it and waits for
// it before touching global memory.  Inside a CUDA graph this costs far less
// than a memset node between two kernels.  chained: the clear is itself
// launched as the programmatic dependent of the kernel ahead of it (it waits
// for that kernel before writing), so that it and the decode behind it can
// start while that kernel drains; only for decodes that wait before their
// first global access.
cudaError_t launch_zero_counts(unsigned long long *a, unsigned long long *b, cudaStream_t st, bool chained = false);

// Specialised streaming decoder.  Decodes the longest prefix of whole chunks
// it supports and returns the number of codewords covered in *covered (0 when
// n has no specialised kernel).  pdl: launched as the programmatic dependent
// of a launch_zero_counts() just enqueued on `st`.
cudaError_t launch_decode_fast(const uint32_t *in, uint32_t n, uint64_t num_cw, uint32_t *out, void *syn,
                               int syn_type, unsigned long long *err, cudaStream_t st, uint64_t *covered,
                               bool pdl = false);

// The SECDED streaming decoder (codewords of n + 1 bits): whole chunks, as
// launch_decode_fast; `det` (or nullptr) receives the detected double errors.
cudaError_t launch_decode_fast_secded(const uint32_t *in, uint32_t n, uint64_t num_cw, uint32_t *out, void *syn,
                                      int syn_type, unsigned long long *err, unsigned long long *det, cudaStream_t st,
                                      uint64_t *covered, bool pdl = false);

// Decode table of n = 7 or 15 (data | s << k per codeword; with xh the SECDED
// table of n + 1 bits, data | s << k | P << (k + m)), filled on `st` on first
// use per device; nullptr for other n, or when the table is not filled yet and
// `st` is capturing.
const uint16_t *lut_ptr(uint32_t n, cudaStream_t st, bool xh = false);

// Device address of the status word that kernels latch HD_ERR_TIMEOUT into
// (per device; nullptr on failure), and its host-side read-and-clear.
uint32_t *status_ptr();
uint32_t read_clear_status_decode();

}  // namespace hd
