// hd_secded.cu -- SECDED decoding (extended Hamming codes), an extension of the
// paper's single-error decoder that is not in the paper: a full-length code
// n = 2^m - 1 plus an overall parity bit at position 0, so a codeword has
// n + 1 = 2^m bits and 32 codewords fill n + 1 words.  The overall parity P
// of the n + 1 bits decides: P = 1, one error, flip position s (s = 0 is the
// parity bit itself); P = 0 with s != 0, two errors, detected and left as
// received.  Whole chunks go to the streaming kernel compiled with XH (see
// hd_stream_x.cu); the ragged tail to k_secded_tail, one codeword per lane.
#include <algorithm>
#include <cstdint>

#include "hd_device.cuh"
#include "hd_generic.cuh"
#include "hd_internal.h"

namespace hd {
namespace {

constexpr int kTailWarps = 8;

__global__ void __launch_bounds__(kTailWarps * 32)
    k_secded_tail(const uint32_t *__restrict__ in, uint64_t in_words, uint32_t n, uint32_t m, uint64_t cw_begin,
                  uint64_t num_cw, uint32_t *__restrict__ out, uint64_t out_words, void *__restrict__ syn,
                  int syn_type, unsigned long long *__restrict__ err, unsigned long long *__restrict__ det)
{
    __shared__ uint32_t sy[kTailWarps][kWarpSlotWords];
    __shared__ uint32_t sd[kTailWarps][kWarpSlotWords];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    uint32_t *my_y = &sy[wp][lane * kSlot];
    uint32_t *my_d = &sd[wp][lane * kSlot];
    const uint32_t k = n - m, L = n + 1;
    const uint32_t wy = L <= 32 ? 1u : L >> 5;
    const uint64_t t_begin = cw_begin / 32, tiles = (num_cw + 31) / 32;
    uint32_t errs = 0, dets = 0;
    for (uint64_t t = t_begin + (uint64_t)blockIdx.x * kTailWarps + wp; t < tiles;
         t += (uint64_t)gridDim.x * kTailWarps) {
        const uint64_t i = t * 32 + lane;
        const bool valid = i < num_cw;
        // position p of codeword i is stream bit i*(n+1) + p: the words are the position domain
        uint32_t y[8];
#pragma unroll
        for (uint32_t w = 0; w < 8; ++w)
            y[w] = (valid && w < wy) ? load_window(in, in_words, (int64_t)(i * L) + 32 * (int64_t)w) : 0u;
        if (L < 32) y[0] &= (1u << L) - 1u;
        const uint32_t s = syndrome_y(y, wy);
        uint32_t f = 0;
#pragma unroll
        for (uint32_t w = 0; w < 8; ++w) f ^= y[w];
        const uint32_t P = __popc(f) & 1u;
        const uint32_t sf = P ? s : 0xFFFFFFFFu;  // nothing is flipped when P = 0
#pragma unroll
        for (uint32_t w = 0; w < 8; ++w)
            if (w < wy) y[w] ^= shl_clamp(1u, sf - 32u * w);
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            my_y[w] = y[w];
            my_d[w] = 0;
        }
        my_y[8] = 0;
        my_d[8] = 0;
        for (uint32_t j = 1; j < m; ++j)
            copy_bits(my_y, (1u << j) + 1u, my_d, (1u << j) - j - 1u, (1u << j) - 1u);
        __syncwarp();
        for (uint32_t q = lane; q < k; q += 32) {
            const uint64_t g = t * k + q;
            if (g >= out_words) break;
            uint32_t c = (32u * q) / k, o = 32u * q - c * k, v = 0, filled = 0;
            while (filled < 32 && c < 32) {
                const uint32_t avail = k - o, take = avail < 32 - filled ? avail : 32 - filled;
                v |= get_bits(&sd[wp][c * kSlot], o, take) << filled;
                filled += take;
                ++c;
                o = 0;
            }
            out[g] = v;
        }
        const uint32_t val = s | (P << m);
        if (valid) {
            if (syn_type == 1) static_cast<uint8_t *>(syn)[i] = (uint8_t)val;
            if (syn_type == 2) static_cast<uint16_t *>(syn)[i] = (uint16_t)val;
        }
        errs += __popc(__ballot_sync(0xFFFFFFFFu, valid && val != 0));
        dets += __popc(__ballot_sync(0xFFFFFFFFu, valid && P == 0 && s != 0));
        __syncwarp();
    }
    if (lane == 0) {
        if (err && errs) atomicAdd(err, (unsigned long long)errs);
        if (det && dets) atomicAdd(det, (unsigned long long)dets);
    }
}

// One thread per codeword, bit-serial (builds inputs; not timed).  The stream must be zero.
__global__ void k_encode_secded(const uint32_t *__restrict__ data, uint64_t data_words, uint32_t n, uint32_t m,
                                uint64_t num_cw, uint32_t *__restrict__ stream)
{
    const uint32_t k = n - m, L = n + 1;
    for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < num_cw;
         c += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t s = 0, par = 0, d = 0, win = 0;
        for (uint32_t p = 3; p <= n; ++p) {  // checksum vector and parity of the data positions
            if ((p & (p - 1u)) == 0) continue;
            if ((d & 31u) == 0) win = load_window(data, data_words, (int64_t)(c * k + d));
            if ((win >> (d & 31u)) & 1u) {
                s ^= p;
                par ^= 1u;
            }
            ++d;
        }
        par ^= __popc(s) & 1u;  // the checksum bits set to s
        const uint64_t b0 = c * L, b1 = b0 + L;
        uint32_t acc = 0;
        d = 0;
        for (uint32_t p = 0; p <= n; ++p) {
            uint32_t bit;
            if (p == 0) {
                bit = par;
            } else if ((p & (p - 1u)) == 0) {
                bit = (s >> (31u - __clz(p))) & 1u;
            } else {
                if ((d & 31u) == 0) win = load_window(data, data_words, (int64_t)(c * k + d));
                bit = (win >> (d & 31u)) & 1u;
                ++d;
            }
            const uint64_t b = b0 + p;
            acc |= bit << (b & 31u);
            if ((b & 31u) == 31u || p == n) {
                const uint64_t w = b >> 5;
                if ((w << 5) >= b0 && (w << 5) + 32 <= b1)
                    stream[w] = acc;
                else if (acc)
                    atomicOr(&stream[w], acc);
                acc = 0;
            }
        }
    }
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace
}  // namespace hd

using namespace hd;

extern "C" {

hd_status hd_decode_secded(const uint32_t *stream, uint64_t in_bits, uint32_t n, uint64_t num_codewords,
                           uint32_t *out_bits, void *syndromes, hd_syn_type syn_type, unsigned long long *err_count,
                           unsigned long long *detected_count, void *cuda_stream)
{
    const int m = code_m(n);
    if (m == 0) return HD_ERR_INVALID_N;
    if (syn_type != HD_SYN_NONE && syn_type != HD_SYN_U8 && syn_type != HD_SYN_U16) return HD_ERR_INVALID_ARG;
    if (syn_type == HD_SYN_U8 && m == 8) return HD_ERR_INVALID_ARG;  // s | P << 8 needs 9 bits
    if (num_codewords > (1ull << 40)) return HD_ERR_SIZE;
    if (in_bits != (uint64_t)(n + 1u) * num_codewords) return HD_ERR_SIZE;
    if (num_codewords != 0) {
        if (!stream || !out_bits) return HD_ERR_NULL;
        if (syn_type != HD_SYN_NONE && !syndromes) return HD_ERR_NULL;
        if (!aligned16(stream) || !aligned16(out_bits) || (syndromes && !aligned16(syndromes))) return HD_ERR_ALIGN;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const bool counted = err_count != nullptr || detected_count != nullptr;
    if (counted && launch_zero_counts(err_count, detected_count, st, true) != cudaSuccess) return HD_ERR_CUDA;
    if (num_codewords == 0) return HD_OK;
    const uint32_t k = n - (uint32_t)m;
    const int syn = syndromes ? (int)syn_type : 0;
    uint64_t covered = 0;
    if (launch_decode_fast_secded(stream, n, num_codewords, out_bits, syndromes, syn, err_count, detected_count, st,
                                  &covered, true) != cudaSuccess)
        return HD_ERR_CUDA;
    if (covered < num_codewords) {
        const uint64_t tiles = (num_codewords + 31) / 32 - covered / 32;
        const uint64_t want = (tiles + kTailWarps - 1) / kTailWarps, cap = (uint64_t)num_sms() * 8;
        k_secded_tail<<<decode_grid(want, cap), kTailWarps * 32, 0, st>>>(
            stream, words_for_bits(in_bits), n, (uint32_t)m, covered, num_codewords, out_bits,
            words_for_bits(num_codewords * k), syndromes, syn, err_count, detected_count);
        count_launch();
        if (cudaGetLastError() != cudaSuccess) return HD_ERR_CUDA;
    }
    return HD_OK;
}

hd_status hd_encode_secded(const uint32_t *data_bits, uint32_t n, uint64_t num_codewords, uint32_t *stream,
                           void *cuda_stream)
{
    const int m = code_m(n);
    if (m == 0) return HD_ERR_INVALID_N;
    if (num_codewords > (1ull << 40)) return HD_ERR_SIZE;
    if (num_codewords == 0) return HD_OK;
    if (!data_bits || !stream) return HD_ERR_NULL;
    if (!aligned16(data_bits) || !aligned16(stream)) return HD_ERR_ALIGN;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const uint32_t k = n - (uint32_t)m;
    if (cudaMemsetAsync(stream, 0, words_for_bits(num_codewords * (n + 1u)) * 4, st) != cudaSuccess)
        return HD_ERR_CUDA;
    const uint64_t want = (num_codewords + 255) / 256, cap = (uint64_t)num_sms() * 16;
    k_encode_secded<<<(int)std::min(want, cap), 256, 0, st>>>(data_bits, words_for_bits(num_codewords * k), n,
                                                              (uint32_t)m, num_codewords, stream);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? HD_OK : HD_ERR_CUDA;
}

}  // extern "C"
