/*
 * hd_oracle.c -- TEST INFRASTRUCTURE, not part of the decoder product.
 *
 * A plain, slow, bit-by-bit CPU restatement of the Hamming decoder of
 * Islam, Kim and Kim, "Computationally Efficient Implementation of a Hamming
 * Code Decoder using Graphics Processing Unit" (J. Commun. Netw., 2015).
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * load this library.  It shares no source, header or table with the CUDA
 * decoder, and the CUDA decoder never links or calls it.
 *
 * Conventions (the paper fixes the first three, the rest are this
 * repository's stated readings where the paper is silent):
 *  - Positions inside a codeword are 1-indexed, p = 1..n (Sec. III-A lists
 *    the index sets starting at position 1).
 *  - Index set I_j = { p : bit j of p is 1 }; checksum bit j is the modulo-2
 *    sum (XOR) of the received bits at the positions of I_j (Sec. III-A and
 *    Algorithm 1, step 4).  Even parity: a valid codeword has all checksum
 *    bits 0.
 *  - The checksum bits sit at the power-of-two positions 2^j; the remaining
 *    positions carry data, in increasing position order (Sec. II: the
 *    redundancy remover drops the checksum bits).
 *  - Full-length codes n = 2^m - 1, 2 <= m <= 8.
 *  - Stream bit b is bit (b mod 32) of uint32 word b/32 (LSB first); codeword
 *    i occupies stream bits [i*n, (i+1)*n); its data bits go to output bits
 *    [i*k, (i+1)*k), k = n - m.
 *  - A nonzero syndrome s names the position to flip (single error
 *    correction, Sec. II "error correction").  With two errors the decoder
 *    flips position p XOR q, exactly as a plain single-error decoder does.
 *  - err_count = number of codewords with a nonzero syndrome.
 *  - Output pad bits past N*k in the last word are written as 0.
 */
#include <stddef.h>
#include <stdint.h>

#define REF_OK 0
#define REF_ERR_INVALID_N 1
#define REF_ERR_NULL 2
#define REF_ERR_SIZE 3

#define REF_SYN_NONE 0
#define REF_SYN_U8 1
#define REF_SYN_U16 2

static int get_bit(const uint32_t *w, uint64_t b) { return (int)((w[b >> 5] >> (b & 31u)) & 1u); }

static void put_bit(uint32_t *w, uint64_t b, int v)
{
    uint32_t mask = 1u << (b & 31u);
    if (v)
        w[b >> 5] |= mask;
    else
        w[b >> 5] &= ~mask;
}

/* A position is a checksum position iff it is a power of two (Sec. III-A). */
static int is_checksum_position(uint32_t p) { return p != 0 && (p & (p - 1u)) == 0; }

/* Number of checksum bits m for a full-length code n = 2^m - 1; 0 if n is not
 * a supported length. */
int hd_ref_num_checksum_bits(uint32_t n)
{
    for (uint32_t m = 2; m <= 8; ++m)
        if (n == (1u << m) - 1u)
            return (int)m;
    return 0;
}

/* Decode codewords [first, first + count) of `stream`.  Writes their data bits
 * at output bits [i*k, (i+1)*k) one bit at a time (read-modify-write, so the
 * caller may split a stream into ranges whose first codeword is a multiple of
 * 32 and decode them from several threads), their syndromes, and adds the
 * number of nonzero syndromes to *errs.
 *
 * Steps per codeword, in the paper's order (Sec. II and III):
 *   1. read the n received bits, position p from stream bit i*n + p - 1;
 *   2. checksum: s = XOR of p over the positions p whose bit is 1, which is
 *      the same as checksum bit j = XOR of the bits at positions of I_j;
 *   3. error detection: s != 0; error correction: flip the bit at position s;
 *   4. redundancy removal: keep the non-power-of-two positions in order. */
int hd_ref_decode_range(const uint32_t *stream, uint32_t n, uint64_t first, uint64_t count,
                        uint32_t *out_bits, void *syndromes, int syn_type, uint64_t *errs)
{
    int m = hd_ref_num_checksum_bits(n);
    if (m == 0)
        return REF_ERR_INVALID_N;
    if (count == 0)
        return REF_OK;
    if (!stream || !out_bits || !errs)
        return REF_ERR_NULL;
    uint32_t k = n - (uint32_t)m;
    unsigned char bit[256];
    uint64_t e = 0;
    for (uint64_t i = first; i < first + count; ++i) {
        /* 1. received bits */
        for (uint32_t p = 1; p <= n; ++p)
            bit[p] = (unsigned char)get_bit(stream, i * n + p - 1);
        /* 2. checksum (syndrome) */
        uint32_t s = 0;
        for (uint32_t p = 1; p <= n; ++p)
            if (bit[p])
                s ^= p;
        /* 3. detect and correct */
        if (s != 0) {
            if (s <= n)
                bit[s] ^= 1u;
            ++e;
        }
        /* 4. remove the checksum bits, keep data bits in position order */
        uint32_t d = 0;
        for (uint32_t p = 1; p <= n; ++p) {
            if (is_checksum_position(p))
                continue;
            put_bit(out_bits, i * k + d, bit[p]);
            ++d;
        }
        if (syn_type == REF_SYN_U8 && syndromes)
            ((uint8_t *)syndromes)[i] = (uint8_t)s;
        else if (syn_type == REF_SYN_U16 && syndromes)
            ((uint16_t *)syndromes)[i] = (uint16_t)s;
    }
    *errs += e;
    return REF_OK;
}

/* Zero the output bits from bit `from` up to the end of its 32-bit word. */
static void zero_pad(uint32_t *words, uint64_t from)
{
    for (uint64_t b = from; (b & 31u) != 0; ++b)
        put_bit(words, b, 0);
}

/* Whole-stream decode: argument checks, every codeword, then the pad bits. */
int hd_ref_decode(const uint32_t *stream, uint64_t in_bits, uint32_t n, uint64_t num_codewords,
                  uint32_t *out_bits, void *syndromes, int syn_type, uint64_t *err_count)
{
    int m = hd_ref_num_checksum_bits(n);
    if (m == 0)
        return REF_ERR_INVALID_N;
    if (in_bits != (uint64_t)n * num_codewords)
        return REF_ERR_SIZE;
    if (err_count)
        *err_count = 0;
    if (num_codewords == 0)
        return REF_OK;
    uint64_t e = 0;
    int rc = hd_ref_decode_range(stream, n, 0, num_codewords, out_bits, syndromes, syn_type, &e);
    if (rc != REF_OK)
        return rc;
    zero_pad(out_bits, num_codewords * (uint64_t)(n - (uint32_t)m));
    if (err_count)
        *err_count = e;
    return REF_OK;
}

/* ---------------------------------------------------------------------------
 * Shortened codes: any length n >= 3 (the paper's segments of a packet,
 * Sec. II and Sec. IV-A: a packet of M bytes split into t segments, each with
 * its own checksum bits).  r = the smallest number of checksum bits with
 * 2^r >= n + 1; the checksum bits sit at the power-of-two positions <= n.
 * A syndrome s <= n names the position to flip; s > n names no position, so
 * the codeword is flagged as detected-uncorrectable and left as received.
 * ------------------------------------------------------------------------- */
int hd_ref_short_checksum_bits(uint32_t n)
{
    if (n < 3 || n > 65535u) return 0;
    int r = 0;
    while ((1u << r) < n + 1u) ++r;
    return r;
}

/* Decode codewords [first, first + count) of a shortened-code stream, in the
 * steps of hd_ref_decode_range; adds the number of nonzero syndromes to
 * *errs and the number of syndromes past n to *detected. */
int hd_ref_decode_short_range(const uint32_t *stream, uint32_t n, uint64_t first, uint64_t count, uint32_t *out_bits,
                              void *syndromes, int syn_type, uint64_t *errs, uint64_t *detected)
{
    int r = hd_ref_short_checksum_bits(n);
    if (r == 0) return REF_ERR_INVALID_N;
    if (count == 0) return REF_OK;
    if (!stream || !out_bits || !errs || !detected) return REF_ERR_NULL;
    uint32_t k = n - (uint32_t)r;
    static __thread unsigned char bit[65536];
    uint64_t ce = 0, de = 0;
    for (uint64_t i = first; i < first + count; ++i) {
        for (uint32_t p = 1; p <= n; ++p)
            bit[p] = (unsigned char)get_bit(stream, i * n + p - 1);
        uint32_t s = 0;
        for (uint32_t p = 1; p <= n; ++p)
            if (bit[p]) s ^= p;
        if (s != 0) {
            ++ce;
            if (s <= n)
                bit[s] ^= 1u; /* names a position: correct it */
            else
                ++de; /* names no position: detected, left as received */
        }
        uint32_t d = 0;
        for (uint32_t p = 1; p <= n; ++p) {
            if (is_checksum_position(p)) continue;
            put_bit(out_bits, i * k + d, bit[p]);
            ++d;
        }
        if (syn_type == REF_SYN_U8 && syndromes)
            ((uint8_t *)syndromes)[i] = (uint8_t)s;
        else if (syn_type == REF_SYN_U16 && syndromes)
            ((uint16_t *)syndromes)[i] = (uint16_t)s;
    }
    *errs += ce;
    *detected += de;
    return REF_OK;
}

int hd_ref_decode_short(const uint32_t *stream, uint64_t in_bits, uint32_t n, uint64_t num_codewords,
                        uint32_t *out_bits, void *syndromes, int syn_type, uint64_t *err_count, uint64_t *detected)
{
    int r = hd_ref_short_checksum_bits(n);
    if (r == 0) return REF_ERR_INVALID_N;
    if (in_bits != (uint64_t)n * num_codewords) return REF_ERR_SIZE;
    uint64_t ce = 0, de = 0;
    if (num_codewords > 0) {
        int rc = hd_ref_decode_short_range(stream, n, 0, num_codewords, out_bits, syndromes, syn_type, &ce, &de);
        if (rc != REF_OK) return rc;
        zero_pad(out_bits, num_codewords * (uint64_t)(n - (uint32_t)r));
    }
    if (err_count) *err_count = ce;
    if (detected) *detected = de;
    return REF_OK;
}

/* Encoder of the shortened code (test inputs only): as hd_ref_encode, with
 * the checksum bits at the power-of-two positions <= n. */
int hd_ref_encode_short(const uint32_t *data_bits, uint32_t n, uint64_t num_codewords, uint32_t *stream)
{
    int r = hd_ref_short_checksum_bits(n);
    if (r == 0) return REF_ERR_INVALID_N;
    if (num_codewords == 0) return REF_OK;
    if (!data_bits || !stream) return REF_ERR_NULL;
    uint32_t k = n - (uint32_t)r;
    static __thread unsigned char bit[65536];
    for (uint64_t i = 0; i < num_codewords; ++i) {
        uint32_t d = 0;
        for (uint32_t p = 1; p <= n; ++p) {
            if (is_checksum_position(p)) {
                bit[p] = 0;
            } else {
                bit[p] = (unsigned char)get_bit(data_bits, i * k + d);
                ++d;
            }
        }
        uint32_t s = 0;
        for (uint32_t p = 1; p <= n; ++p)
            if (bit[p]) s ^= p;
        for (int j = 0; j < r; ++j)
            bit[1u << j] = (unsigned char)(1u & (s >> j));
        for (uint32_t p = 1; p <= n; ++p)
            put_bit(stream, i * n + p - 1, bit[p]);
    }
    zero_pad(stream, num_codewords * (uint64_t)n);
    return REF_OK;
}

/* ---------------------------------------------------------------------------
 * SECDED (extended Hamming): not in the paper.  A full-length code n = 2^m - 1
 * plus an overall parity bit at position 0, so a codeword has n + 1 = 2^m
 * bits: codeword i occupies stream bits [i*(n+1), (i+1)*(n+1)) with position p
 * (0..n) at bit i*(n+1) + p.  Even parity over all n + 1 bits.
 *   s = XOR of the positions 1..n of the set bits, P = parity of all n + 1 bits.
 *   P = 1: one error; flip position s (s = 0: the overall parity bit itself).
 *   P = 0, s != 0: two errors, detected; the codeword is left as received.
 * The syndrome value is s | P << m; err_count counts nonzero values, detected
 * counts P = 0 with s != 0.
 * ------------------------------------------------------------------------- */
int hd_ref_decode_secded_range(const uint32_t *stream, uint32_t n, uint64_t first, uint64_t count, uint32_t *out_bits,
                               void *syndromes, int syn_type, uint64_t *errs, uint64_t *detected)
{
    int m = hd_ref_num_checksum_bits(n);
    if (m == 0) return REF_ERR_INVALID_N;
    if (count == 0) return REF_OK;
    if (!stream || !out_bits || !errs || !detected) return REF_ERR_NULL;
    uint32_t k = n - (uint32_t)m, len = n + 1u;
    unsigned char bit[256];
    uint64_t ce = 0, de = 0;
    for (uint64_t i = first; i < first + count; ++i) {
        for (uint32_t p = 0; p <= n; ++p)
            bit[p] = (unsigned char)get_bit(stream, i * len + p);
        uint32_t s = 0, par = 0;
        for (uint32_t p = 0; p <= n; ++p) {
            if (bit[p]) {
                s ^= p;
                par ^= 1u;
            }
        }
        uint32_t v = s | (par << m);
        if (v != 0) ++ce;
        if (par)
            bit[s] ^= 1u; /* one error: position s (0 is the overall parity bit) */
        else if (s != 0)
            ++de; /* two errors: detected, not corrected */
        uint32_t d = 0;
        for (uint32_t p = 1; p <= n; ++p) {
            if (is_checksum_position(p)) continue;
            put_bit(out_bits, i * k + d, bit[p]);
            ++d;
        }
        if (syn_type == REF_SYN_U8 && syndromes)
            ((uint8_t *)syndromes)[i] = (uint8_t)v;
        else if (syn_type == REF_SYN_U16 && syndromes)
            ((uint16_t *)syndromes)[i] = (uint16_t)v;
    }
    *errs += ce;
    *detected += de;
    return REF_OK;
}

int hd_ref_decode_secded(const uint32_t *stream, uint64_t in_bits, uint32_t n, uint64_t num_codewords,
                         uint32_t *out_bits, void *syndromes, int syn_type, uint64_t *err_count, uint64_t *detected)
{
    int m = hd_ref_num_checksum_bits(n);
    if (m == 0) return REF_ERR_INVALID_N;
    if (in_bits != (uint64_t)(n + 1u) * num_codewords) return REF_ERR_SIZE;
    uint64_t ce = 0, de = 0;
    if (num_codewords > 0) {
        int rc = hd_ref_decode_secded_range(stream, n, 0, num_codewords, out_bits, syndromes, syn_type, &ce, &de);
        if (rc != REF_OK) return rc;
        zero_pad(out_bits, num_codewords * (uint64_t)(n - (uint32_t)m));
    }
    if (err_count) *err_count = ce;
    if (detected) *detected = de;
    return REF_OK;
}

/* SECDED encoder (test inputs only): the Hamming checksum bits, then the
 * overall parity bit at position 0 makes the parity of all n + 1 bits even. */
int hd_ref_encode_secded(const uint32_t *data_bits, uint32_t n, uint64_t num_codewords, uint32_t *stream)
{
    int m = hd_ref_num_checksum_bits(n);
    if (m == 0) return REF_ERR_INVALID_N;
    if (num_codewords == 0) return REF_OK;
    if (!data_bits || !stream) return REF_ERR_NULL;
    uint32_t k = n - (uint32_t)m, len = n + 1u;
    unsigned char bit[256];
    for (uint64_t i = 0; i < num_codewords; ++i) {
        uint32_t d = 0;
        for (uint32_t p = 1; p <= n; ++p) {
            if (is_checksum_position(p)) {
                bit[p] = 0;
            } else {
                bit[p] = (unsigned char)get_bit(data_bits, i * k + d);
                ++d;
            }
        }
        uint32_t s = 0;
        for (uint32_t p = 1; p <= n; ++p)
            if (bit[p]) s ^= p;
        for (int j = 0; j < m; ++j)
            bit[1u << j] = (unsigned char)(1u & (s >> j) & 1u);
        uint32_t par = 0;
        for (uint32_t p = 1; p <= n; ++p) par ^= bit[p];
        bit[0] = (unsigned char)par;
        for (uint32_t p = 0; p <= n; ++p)
            put_bit(stream, i * len + p, bit[p]);
    }
    zero_pad(stream, num_codewords * (uint64_t)len);
    return REF_OK;
}

/* Encoder, used only to build test inputs (Sec. II: the transmitter adds the
 * checksum bits to the message).  Per codeword: the k data bits go to the
 * non-power-of-two positions in increasing order, the checksum positions start
 * at 0, s is the XOR of the set positions, and checksum bit 2^j is set to bit j
 * of s, which makes the syndrome of the result 0. */
int hd_ref_encode(const uint32_t *data_bits, uint32_t n, uint64_t num_codewords, uint32_t *stream)
{
    int m = hd_ref_num_checksum_bits(n);
    if (m == 0)
        return REF_ERR_INVALID_N;
    if (num_codewords == 0)
        return REF_OK;
    if (!data_bits || !stream)
        return REF_ERR_NULL;
    uint32_t k = n - (uint32_t)m;
    unsigned char bit[256];
    for (uint64_t i = 0; i < num_codewords; ++i) {
        uint32_t d = 0;
        for (uint32_t p = 1; p <= n; ++p) {
            if (is_checksum_position(p)) {
                bit[p] = 0;
            } else {
                bit[p] = (unsigned char)get_bit(data_bits, i * k + d);
                ++d;
            }
        }
        uint32_t s = 0;
        for (uint32_t p = 1; p <= n; ++p)
            if (bit[p])
                s ^= p;
        for (int j = 0; j < m; ++j)
            bit[1u << j] = (unsigned char)((s >> j) & 1u);
        for (uint32_t p = 1; p <= n; ++p)
            put_bit(stream, i * n + p - 1, bit[p]);
    }
    zero_pad(stream, num_codewords * (uint64_t)n);
    return REF_OK;
}
