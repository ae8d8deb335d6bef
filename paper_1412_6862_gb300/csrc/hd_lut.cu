// hd_lut.cu -- decode tables for the short full-length codes (n = 7, 15) and
// for their SECDED extensions (8 and 16 bits).
//
// For n <= 15 a whole codeword fits a table index: entry y (bit p-1 of y is
// position p) holds the corrected data bits of y and its checksum vector,
// data | s << k (Sec. II: detect, correct, remove the checksum bits; s as the
// XOR of the positions of the set bits, Sec. III-A).  The streaming kernel's
// table variants copy the table into shared memory and decode a codeword with
// one lookup.  The tables live in static device memory and are filled by a
// kernel on first use per device (on the caller's stream, which that first
// call then synchronises; a first call inside a stream capture falls back to
// the arithmetic decoder).
#include <cstdint>
#include <mutex>

#include "hd_internal.h"

namespace hd {
namespace {

__device__ __align__(128) uint16_t g_lut7[1u << 7];
__device__ __align__(128) uint16_t g_lut15[1u << 15];
// SECDED (extended codes of n + 1 bits, overall parity bit at position 0):
// entry y (bit p of y is position p) holds data | s << k | P << (k + m)
__device__ __align__(128) uint16_t g_lut7x[1u << 8];
__device__ __align__(128) uint16_t g_lut15x[1u << 16];

__global__ void k_fill_lut(uint16_t *lut, uint32_t n, uint32_t m)
{
    const uint32_t y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= (1u << n)) return;
    uint32_t s = 0;
    for (uint32_t p = 1; p <= n; ++p)
        if ((y >> (p - 1)) & 1u) s ^= p;
    const uint32_t c = s ? y ^ (1u << (s - 1)) : y;  // flip position s
    uint32_t d = 0, j = 0;
    for (uint32_t p = 1; p <= n; ++p) {
        if ((p & (p - 1)) == 0) continue;  // checksum position
        d |= ((c >> (p - 1)) & 1u) << j;
        ++j;
    }
    lut[y] = (uint16_t)(d | (s << (n - m)));
}

// SECDED: P = parity of all n + 1 bits; P = 1 flips position s (position 0
// when s = 0), P = 0 flips nothing (s != 0 is a detected double error)
__global__ void k_fill_lut_xh(uint16_t *lut, uint32_t n, uint32_t m)
{
    const uint32_t y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= (2u << n)) return;
    uint32_t s = 0, P = 0;
    for (uint32_t p = 0; p <= n; ++p)
        if ((y >> p) & 1u) {
            s ^= p;
            P ^= 1u;
        }
    const uint32_t c = P ? y ^ (1u << s) : y;
    uint32_t d = 0, j = 0;
    for (uint32_t p = 1; p <= n; ++p) {
        if ((p & (p - 1)) == 0) continue;  // checksum position
        d |= ((c >> p) & 1u) << j;
        ++j;
    }
    lut[y] = (uint16_t)(d | (s << (n - m)) | (P << n));
}

std::mutex g_lut_mu;
bool g_lut_ready[64][4];

}  // namespace

const uint16_t *lut_ptr(uint32_t n, cudaStream_t st, bool xh)
{
    const int which = (n == 7 ? 0 : (n == 15 ? 1 : -1));
    if (which < 0) return nullptr;
    const int slot = which + (xh ? 2 : 0);
    static const void *const syms[4] = {&g_lut7, &g_lut15, &g_lut7x, &g_lut15x};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, syms[slot]) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_lut_mu);
    if (!g_lut_ready[dev][slot]) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
        const uint32_t entries = (xh ? 2u : 1u) << n, m = (uint32_t)code_m(n);
        if (xh)
            k_fill_lut_xh<<<(entries + 255) / 256, 256, 0, st>>>(static_cast<uint16_t *>(p), n, m);
        else
            k_fill_lut<<<(entries + 255) / 256, 256, 0, st>>>(static_cast<uint16_t *>(p), n, m);
        count_launch();
        // kernels on other streams may use the table next: wait for it once
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return nullptr;
        g_lut_ready[dev][slot] = true;
    }
    return static_cast<const uint16_t *>(p);
}

}  // namespace hd
