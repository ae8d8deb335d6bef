/*
 * hd.h -- C ABI of the GB300 Hamming(n,k) decoder (libhd.so).
 *
 * The operation is the decoder of Islam, Kim and Kim, "Computationally
 * Efficient Implementation of a Hamming Code Decoder using Graphics Processing
 * Unit" (J. Commun. Netw., 2015): for each received codeword compute the
 * checksum vector (Sec. III-C, Algorithm 1: checksum bit j is the modulo-2 sum
 * of the bits at the positions of index set I_j, Sec. III-A), detect and
 * correct the error it names, drop the checksum bits and merge the data bits
 * into the decoded packet (Sec. II, Fig. 1; Sec. III, the "error" kernel).
 *
 * Codes: full-length Hamming codes n = 2^m - 1, 2 <= m <= 8 (n = 3..255),
 * k = n - m data bits.  Positions are 1-indexed; the checksum bits sit at the
 * power-of-two positions and use even parity; the data bits are the other
 * positions in increasing order.
 *
 * Bit layout of every stream: bit b is bit (b mod 32) of uint32 word b/32
 * (LSB first).  Codeword i occupies input bits [i*n, (i+1)*n) with position p
 * at bit i*n + p - 1; its data bits go to output bits [i*k, (i+1)*k).
 *
 * Ownership and asynchrony: every buffer is caller-owned DEVICE memory unless
 * a parameter says otherwise.  Calls enqueue work on `cuda_stream` (a
 * cudaStream_t; NULL is the legacy default stream) and return before the work
 * finishes.  The returned status covers argument checks and launch errors;
 * a device-side failure (a bounded wait that ran out) is latched in a device
 * status word that hd_device_status() reads.
 *
 * Alignment: stream, output and syndrome buffers must start on a 16-byte
 * boundary (allocations from cudaMalloc or PyTorch always do).
 */
#ifndef HD_H
#define HD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HD_OK = 0,
    HD_ERR_INVALID_N = 1,   /* n is not 2^m - 1 with 2 <= m <= 8 */
    HD_ERR_NULL = 2,        /* a required pointer is NULL */
    HD_ERR_SIZE = 3,        /* in_bits != n * num_codewords, or a size is out of range */
    HD_ERR_ALIGN = 4,       /* a buffer is not 16-byte aligned */
    HD_ERR_CAPACITY = 5,    /* a fixed capacity would be exceeded */
    HD_ERR_TIMEOUT = 6,     /* a bounded device-side wait ran out */
    HD_ERR_CUDA = 7,        /* the CUDA runtime reported an error */
    HD_ERR_INVALID_ARG = 8  /* any other invalid argument */
} hd_status;

typedef enum {
    HD_SYN_NONE = 0,  /* do not store syndromes */
    HD_SYN_U8 = 1,    /* one uint8_t per codeword (valid for every supported n) */
    HD_SYN_U16 = 2    /* one uint16_t per codeword */
} hd_syn_type;

/* Decode `num_codewords` back-to-back codewords of length n.
 *
 * stream        device, ceil(in_bits/32) words; pad bits past in_bits are ignored.
 * in_bits       must equal n * num_codewords (HD_ERR_SIZE otherwise).
 * out_bits      device, ceil(num_codewords*k/32) words; receives the data bits of
 *               codeword i at bits [i*k, (i+1)*k); pad bits past num_codewords*k
 *               in the last word are written as 0.
 * syndromes     device, num_codewords elements of the width `syn_type` names, or
 *               NULL with HD_SYN_NONE.  Element i is the checksum vector of codeword
 *               i read as an integer (bit j = checksum bit j): 0 for a valid word,
 *               otherwise the position that was flipped.
 * err_count     device, one unsigned long long, or NULL: overwritten with the
 *               number of codewords whose syndrome is nonzero.
 * Two errors in one codeword give syndrome p XOR q and the decoder flips that
 * third position, as any single-error-correcting Hamming decoder does.
 * num_codewords == 0 is HD_OK; it only zeroes *err_count.
 * For n = 7 and 15 the chosen configuration may decode through a table of
 * 2^n entries (data bits and syndrome per codeword value) kept in static
 * device memory; the first such call on a device fills it with a kernel on
 * `cuda_stream` and synchronises that stream (a first call inside a stream
 * capture uses the arithmetic decoder instead). */
hd_status hd_decode(const uint32_t *stream, uint64_t in_bits, uint32_t n, uint64_t num_codewords,
                    uint32_t *out_bits, void *syndromes, hd_syn_type syn_type,
                    unsigned long long *err_count, void *cuda_stream);

/* Several independent streams decoded concurrently.  Each job is one
 * hd_decode() call (arguments, layout, results and errors as there, with
 * in_bits = n * num_codewords).  The jobs' counters are cleared by one kernel
 * on `cuda_stream`, then the decodes run as concurrent branches forked from
 * `cuda_stream` onto library-owned streams (8 per device, created by the
 * first call on a device, which should come before any stream capture) and
 * joined back into it, largest stream first: work enqueued on `cuda_stream`
 * after this call waits for every job.  Decoding the streams side by side lets
 * one decode's ramp-up and drain overlap another's steady state, the
 * pipelining of independent packets the paper applies to its transfers
 * (Sec. III-B).  At most 32 jobs per call (HD_ERR_CAPACITY); the jobs' output
 * buffers must not overlap.  Calls from several host threads are serialised. */
typedef struct {
    const uint32_t *stream;
    uint32_t *out_bits;
    void *syndromes;
    unsigned long long *err_count;
    uint64_t num_codewords;
    uint32_t n;
    uint32_t syn_type; /* an hd_syn_type */
} hd_stream_job;

hd_status hd_decode_streams(const hd_stream_job *jobs, uint32_t num_jobs, void *cuda_stream);

/* Decode from and to HOST memory with overlapped transfers -- the paper's
 * asynchronous data transfer (Sec. III-B, Fig. 5, Eq. 1).  The stream is cut
 * into chunks of `chunk_codewords` (a multiple of 128; 0 = 2^22) and each
 * chunk's host-to-device copy, decode and device-to-host copy run on one of
 * `depth` CUDA streams (0 = 4, at most 8), so copies in both directions
 * overlap with the decoding of neighbouring chunks.  Arguments and results are
 * as in hd_decode(), but host_stream, host_out, host_syndromes and
 * host_err_count are host memory; pinned (page-locked) buffers are needed for
 * the copies to overlap, pageable ones work but serialise.  The call is
 * synchronous: it returns when every result is in host memory.  Device
 * staging buffers are cached per device and grown on demand; concurrent calls
 * on one device are serialised. */
hd_status hd_decode_host(const uint32_t *host_stream, uint64_t in_bits, uint32_t n, uint64_t num_codewords,
                         uint32_t *host_out, void *host_syndromes, hd_syn_type syn_type,
                         unsigned long long *host_err_count, uint64_t chunk_codewords, uint32_t depth);

/* Several host-buffer decodes in one pipeline (the same asynchronous data
 * transfer as hd_decode_host, without a fill and drain per stream).  Each job
 * names a host stream of num_codewords codewords of length n and its host
 * outputs, as the arguments of hd_decode_host (pinned memory for overlap);
 * *host_err_count (or NULL) receives the job's number of nonzero syndromes.
 * All jobs' chunks (chunk_codewords, a multiple of 128; 0 = 2^22) go through
 * `depth` rotating CUDA streams (0 = 4, at most 8); the first chunks of the
 * batch ramp up from chunk/8 and the last ones ramp down, so the pipeline
 * fills and drains on small copies.  Synchronous; errors as hd_decode_host. */
typedef struct {
    const uint32_t *host_stream;
    uint32_t *host_out;
    void *host_syndromes;
    unsigned long long *host_err_count;
    uint64_t num_codewords;
    uint32_t n;
    uint32_t syn_type; /* an hd_syn_type */
} hd_host_job;

hd_status hd_decode_host_batch(const hd_host_job *jobs, uint32_t num_jobs, uint64_t chunk_codewords, uint32_t depth);

/* Encode `num_codewords` messages (the transmitter side of Sec. II: the
 * checksum bits are added to the message).  data_bits holds message i at bits
 * [i*k, (i+1)*k) (device, ceil(num_codewords*k/32) words); stream receives
 * codeword i at bits [i*n, (i+1)*n) with even parity (device,
 * ceil(num_codewords*n/32) words, pad bits written as 0). */
hd_status hd_encode(const uint32_t *data_bits, uint32_t n, uint64_t num_codewords, uint32_t *stream,
                    void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Shortened codes: segments of any length (Sec. II, Fig. 1: the splitter cuts
 * a packet of M bytes into t segments, each with its own checksum bits; the
 * evaluation of Sec. IV-A uses M = 400..2000 bytes and t = 2..6).
 *
 * A segment of length n, 3 <= n <= 32767, carries r checksum bits, r the
 * smallest count with 2^r >= n + 1, at the power-of-two positions 1..2^(r-1),
 * and k = n - r data bits at the other positions in increasing order; the
 * full-length codes n = 2^m - 1 are the special case with no unused syndrome
 * values.  Stream layout, parity sense and ownership are those of hd_decode().
 * ------------------------------------------------------------------------- */

/* r and k of the shortened code of length n (host only; HD_ERR_INVALID_N
 * outside 3..32767).  Either output pointer may be NULL. */
hd_status hd_short_params(uint32_t n, uint32_t *r, uint32_t *k);

/* The paper's splitter sizing (Sec. II): a packet of packet_bytes bytes cut
 * into t segments gives segments of k = ceil(8 * packet_bytes / t) data bits
 * and r checksum bits, r the smallest count with 2^r >= k + r + 1, so
 * n = k + r.  The packet's message is the first 8 * packet_bytes of its t * k
 * data bits; the rest is zero padding.  HD_ERR_INVALID_ARG for t == 0 or
 * t > 8 * packet_bytes, HD_ERR_SIZE when n would exceed 32767.  Host only. */
hd_status hd_segment_params(uint32_t packet_bytes, uint32_t t, uint32_t *n, uint32_t *k, uint32_t *r);

/* Decode `num_codewords` back-to-back segments of length n (a batch of
 * packets of one size and segment count is one such stream: packet p holds
 * segments [p*t, (p+1)*t)).
 *
 * Arguments as hd_decode(), with n in 3..32767.  Syndrome element i is the
 * checksum vector of segment i (HD_SYN_U8 is accepted only for n <= 255).
 * A syndrome s with 1 <= s <= n flips position s; a syndrome s > n names no
 * position: the segment is left as received and counted in *detected_count
 * (device, one unsigned long long, or NULL).  *err_count (device or NULL)
 * counts every nonzero syndrome, detected ones included.  Both counters are
 * overwritten.  num_codewords == 0 is HD_OK and only zeroes the counters. */
hd_status hd_decode_short(const uint32_t *stream, uint64_t in_bits, uint32_t n, uint64_t num_codewords,
                          uint32_t *out_bits, void *syndromes, hd_syn_type syn_type,
                          unsigned long long *err_count, unsigned long long *detected_count, void *cuda_stream);

/* Encode `num_codewords` messages of k bits into segments of length n (the
 * inverse of hd_decode_short; arguments as hd_encode(), n in 3..32767).  The
 * stream's pad bits past num_codewords * n are written as 0. */
hd_status hd_encode_short(const uint32_t *data_bits, uint32_t n, uint64_t num_codewords, uint32_t *stream,
                          void *cuda_stream);

/* Segments with k >= 64 are decoded by a tiled kernel that reads a per-length
 * output-word table (about 2 * (k + 2200) bytes of device memory).
 * hd_decode_short() keeps these tables in a per-device cache: the first call
 * for a length n builds its table (cudaMalloc plus a synchronous copy); up to
 * 32 lengths are kept per device, and evicting the least recently used one
 * waits only for that table's last use (an event on the stream that used it).
 * A call on a capturing stream for a length not in the cache returns
 * HD_ERR_INVALID_ARG and enqueues nothing, and a table used inside a capture
 * is never evicted.  The allocation-free path is a plan: */
typedef struct hd_short_plan hd_short_plan;

/* Build the tables for segments of length n (3..32767) on the current device:
 * the library's only allocation for that length (synchronous).  The plan is
 * owned by the caller and freed by hd_short_plan_destroy(). */
hd_status hd_short_plan_create(uint32_t n, hd_short_plan **plan);

/* hd_decode_short() for the plan's length: arguments, results and errors as
 * there (in_bits must equal n * num_codewords), HD_ERR_INVALID_ARG when the
 * current device is not the plan's.  Enqueues the counters' clears and the
 * decode on `cuda_stream` and nothing else: no allocation, no
 * synchronisation, so it can run inside a stream capture. */
hd_status hd_decode_short_plan(const hd_short_plan *plan, const uint32_t *stream, uint64_t in_bits,
                               uint64_t num_codewords, uint32_t *out_bits, void *syndromes, hd_syn_type syn_type,
                               unsigned long long *err_count, unsigned long long *detected_count,
                               void *cuda_stream);

/* Free a plan's tables (after the work that reads them has finished). */
void hd_short_plan_destroy(hd_short_plan *plan);

/* The tiled kernel is compiled in several configurations (warps per CTA,
 * pipeline stages, stage bytes).
 * hd_short_variant_select() pins one configuration for every length on the
 * current device (ordinal < 0 removes the pin); hd_short_autotune() times
 * every configuration on `num_codewords` all-zero segments of length n (reps
 * launches each, 0 = 5; it allocates its own scratch buffers and synchronises
 * `cuda_stream`) and keeps the fastest for n on the current device, returned
 * in *chosen (-1 when n has a single kernel, k < 64).  A configuration never
 * changes the result, only the speed. */
hd_status hd_short_variant_count(uint32_t *count);
hd_status hd_short_variant_select(int32_t ordinal);
hd_status hd_short_autotune(uint32_t n, uint64_t num_codewords, uint32_t reps, void *cuda_stream, int32_t *chosen);

/* ---------------------------------------------------------------------------
 * SECDED (extended Hamming codes).  Not in the paper: an extension of its
 * single-error decoder that detects double errors instead of miscorrecting
 * them.  A full-length code n = 2^m - 1 (n = 7..255) plus an overall parity
 * bit at position 0: codeword i occupies stream bits [i*(n+1), (i+1)*(n+1))
 * with position p (0..n) at bit i*(n+1) + p; even parity over all n + 1 bits;
 * the n - m data bits are the non-power-of-two positions as in hd_decode().
 * ------------------------------------------------------------------------- */

/* Decode `num_codewords` SECDED codewords.  in_bits must equal
 * (n + 1) * num_codewords.  With s the checksum vector of positions 1..n and
 * P the parity of all n + 1 bits: P = 1 flips position s (s = 0: the parity
 * bit itself, the data are intact); P = 0 with s != 0 is a detected double
 * error, left as received and counted in *detected_count.  Syndrome element i
 * is s | P << m (HD_SYN_U8 only for n <= 127); *err_count counts nonzero
 * elements.  Other arguments, layout, counters and errors as hd_decode().
 * n = 7 and 15 decode with a table (512 B / 128 KB of device memory) that the
 * first such call on a device fills on `cuda_stream` and then synchronises it;
 * a first call while the stream is capturing decodes arithmetically. */
hd_status hd_decode_secded(const uint32_t *stream, uint64_t in_bits, uint32_t n, uint64_t num_codewords,
                           uint32_t *out_bits, void *syndromes, hd_syn_type syn_type,
                           unsigned long long *err_count, unsigned long long *detected_count, void *cuda_stream);

/* Encode `num_codewords` messages of n - m bits into SECDED codewords (as
 * hd_encode(), with the overall parity bit at position 0; stream pad bits are
 * written as 0). */
hd_status hd_encode_secded(const uint32_t *data_bits, uint32_t n, uint64_t num_codewords, uint32_t *stream,
                           void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Kernel configurations and the autotuner.
 *
 * Long streams are decoded by a streaming kernel compiled in several
 * configurations per (n, syn_type): codewords per thread, threads per CTA,
 * pipeline depth and whether decoded words overwrite the input stage.  A
 * built-in choice measured on GB300 is used until hd_autotune() times every
 * configuration on the current device and keeps the fastest, or
 * hd_variant_select() pins one.  Choices are per device and per process.
 * The configuration never changes the result, only the speed.
 * ------------------------------------------------------------------------- */
typedef struct {
    uint32_t index;                /* ordinal among the configurations of (n, syn_type) */
    uint32_t n;
    uint32_t syn_type;
    uint32_t codewords_per_thread; /* 8, 16 or 32 */
    uint32_t threads;              /* threads per CTA */
    uint32_t stages;               /* input pipeline depth (shared-memory stages) */
    uint32_t inplace;              /* 1: decoded words overwrite their input stage */
    uint32_t smem_bytes;           /* dynamic shared memory per CTA */
    uint64_t chunk_codewords;      /* codewords per CTA iteration */
    int32_t blocks_per_sm;         /* resident CTAs per SM on the current device */
    float measured_us;             /* autotuner time of the request, -1 when not measured */
    uint32_t table_lookup;         /* 1: decodes by one shared-memory table lookup per codeword (n = 7, 15);
                                      the table (2^n 16-bit entries) is filled on first use, see hd_decode() */
} hd_variant_info;

/* Number of compiled configurations for (n, syn_type).  Host only. */
hd_status hd_variant_count(uint32_t n, hd_syn_type syn_type, uint32_t *count);

/* Describe configuration `ordinal` (0 .. count-1) of (n, syn_type). */
hd_status hd_variant_info_get(uint32_t n, hd_syn_type syn_type, uint32_t ordinal, hd_variant_info *info);

/* Pin configuration `ordinal` for (n, syn_type) on the current device;
 * ordinal < 0 restores the built-in choice. */
hd_status hd_variant_select(uint32_t n, hd_syn_type syn_type, int32_t ordinal);

/* The configuration hd_decode() uses now for (n, syn_type). */
hd_status hd_variant_current(uint32_t n, hd_syn_type syn_type, hd_variant_info *info);

/* Time every configuration of (n, syn_type) on `num_codewords` codewords of
 * random scratch data (allocated and freed here: enough buffer sets, at most
 * 8, that one pass over them streams twice the L2 size) on `cuda_stream`;
 * `reps` rounds (0 = 5) launch every configuration once per round over all
 * sets, and a configuration's time is its median round.  The fastest is kept
 * for this device, except that the built-in choice stays unless it is more
 * than 2 % slower; the choice is reported in *chosen (may be NULL).
 * Synchronises the stream. */
hd_status hd_autotune(uint32_t n, hd_syn_type syn_type, uint64_t num_codewords, uint32_t reps, void *cuda_stream,
                      hd_variant_info *chosen);

/* SECDED configurations.  hd_decode_secded() decodes whole chunks with one
 * streaming configuration per (n, syn_type) and, for n = 7 and 15, a second
 * one that decodes through the SECDED table; by default the table one is used
 * once its table is filled.  hd_secded_variant_select() pins configuration
 * `ordinal` (< count) for (n, syn_type) on the current device (ordinal < 0
 * restores the default); a table configuration pinned while its table cannot
 * be filled (a first call inside a stream capture) decodes arithmetically.
 * The configuration never changes the result, only the speed.  Host only. */
hd_status hd_secded_variant_count(uint32_t n, hd_syn_type syn_type, uint32_t *count);
hd_status hd_secded_variant_info_get(uint32_t n, hd_syn_type syn_type, uint32_t ordinal, hd_variant_info *info);
hd_status hd_secded_variant_select(uint32_t n, hd_syn_type syn_type, int32_t ordinal);

/* ---------------------------------------------------------------------------
 * Batched decode: many packets of mixed n and length in one persistent launch.
 *
 * Each packet is an independent stream (its own input, output and syndrome
 * buffers, all device memory, each starting on a 16-byte boundary), decoded
 * exactly as hd_decode() would decode it.  This is the paper's splitter /
 * decoder / merger of Sec. II applied to many segments at once: the segments
 * are independent, so the GPU processes them in parallel (Sec. IV-A).
 * ------------------------------------------------------------------------- */
typedef struct {
    const uint32_t *in;     /* device, ceil(num_codewords*n/32) words */
    uint32_t *out;          /* device, ceil(num_codewords*k/32) words */
    void *syndromes;        /* device, num_codewords elements, or NULL */
    uint64_t num_codewords; /* 0 is allowed (the packet is skipped, its count is 0) */
    uint32_t n;             /* 2^m - 1, 2 <= m <= 8 */
    uint32_t syn_type;      /* hd_syn_type; HD_SYN_NONE requires nothing, other types a syndromes buffer */
} hd_packet;

/* A plan: the packet table turned into a device tile table, owned by the
 * library (allocated by hd_plan_create, freed by hd_plan_destroy).  The
 * buffers the packets point to must stay valid while the plan is launched.
 * A plan is not thread-safe: launch it from one host thread at a time. */
typedef struct hd_plan hd_plan;

/* A plan decodes with one of num_variants configurations: variants
 * 0 .. num_variants - 3 launch one persistent kernel that decodes tiles of
 * every n; variant num_variants - 2 (the split configuration) launches one
 * kernel per code length present, each compiled for that n alone, as
 * concurrent branches forked from and joined back into the launching stream
 * (its n = 15 kernel holds the n = 15 decode table once that is filled); the
 * last one (the stream-group configuration) runs the streaming decoder's
 * chunk geometry over each (n, syndrome type) group of packets, one
 * concurrent branch per group, each warp decoding an equal contiguous share
 * of the group's whole chunks and ragged tails (n = 3 packets go to the tile
 * kernel in a branch of their own; with 2^22 - 1 packets or more this
 * configuration gives way to variant 0). */
typedef struct {
    uint32_t num_packets;
    uint32_t num_tiles;     /* warp work items: full chunks plus ragged tails */
    uint32_t full_tiles;
    uint32_t warps_per_cta; /* batch-kernel configuration in use (split: that of the kernels without a table;
                               stream groups: the longest code's kernel) */
    uint32_t stages;
    uint32_t smem_bytes;
    uint32_t variant;       /* index of the configuration, < num_variants */
    uint32_t num_variants;
    uint64_t codewords;     /* over all packets */
    uint64_t in_bytes, out_bytes, syn_bytes;
    float measured_us;      /* hd_plan_autotune's time for the best configuration, -1 if not tuned */
    uint32_t table_lookup;  /* decode tables the configuration uses: bit 0 n = 7 (256 B per CTA),
                               bit 1 n = 15 (64 KB per CTA); each is filled on the launching stream on
                               first use per device (that call synchronises the stream; a launch whose
                               stream is capturing before then decodes without the table) */
} hd_plan_info;

/* Validate the table (HD_ERR_INVALID_N / NULL / ALIGN / SIZE for the first bad
 * packet) and build the plan; synchronous.  The table itself (host memory) is
 * not referenced after the call. */
hd_status hd_plan_create(const hd_packet *table, uint32_t num_packets, hd_plan **plan);

/* Decode every packet of the plan on `cuda_stream`.  err_counts: device array
 * of num_packets elements, or NULL; element i is overwritten with packet i's
 * number of nonzero syndromes.  The first launch (and any launch with a
 * different err_counts pointer) records the launch as a CUDA graph; later
 * launches replay it.  n = 7 packets decode with a 256-byte table that the
 * first batched decode on a device fills on `cuda_stream` and then
 * synchronises it (a launch whose stream is capturing before that decodes
 * n = 7 arithmetically). */
hd_status hd_plan_launch(hd_plan *plan, unsigned long long *err_counts, void *cuda_stream);

/* Time every batch-kernel configuration on the plan's own packets as
 * hd_plan_launch() runs it (recorded as a CUDA graph, then `reps` replays,
 * 0 = 3; output buffers are overwritten, inputs only read), keep the fastest
 * and report it.  The next hd_plan_launch() records its graph anew.
 * Synchronises the stream. */
hd_status hd_plan_autotune(hd_plan *plan, uint32_t reps, void *cuda_stream, hd_plan_info *chosen);

/* Pin batch-kernel configuration `variant` (< hd_plan_info.num_variants). */
hd_status hd_plan_select(hd_plan *plan, uint32_t variant);

hd_status hd_plan_get_info(const hd_plan *plan, hd_plan_info *info);

void hd_plan_destroy(hd_plan *plan);

/* One-shot batched decode: builds the device tables in stream-ordered memory
 * (cudaMallocAsync, freed with cudaFreeAsync after the launch), decodes and
 * overwrites err_counts (device, num_packets elements, or NULL).  The n = 7
 * table is filled on first use as for hd_plan_launch(). */
hd_status hd_decode_batch(const hd_packet *table, uint32_t num_packets, unsigned long long *err_counts,
                          void *cuda_stream);

/* Batched decode that allocates nothing.  The paper has no counterpart; this
 * entry point exists for callers that cannot allocate device memory: a process
 * that budgets all device memory up front, an application whose allocator
 * hooks forbid allocations from inside libraries, or a latency-critical
 * receive path where an allocation could stall or fail.  It decodes exactly
 * like hd_decode_batch(), but its tile table (one 64-byte descriptor per
 * tile) and claim counter live in one fixed 1 MiB array compiled into libhd.so; every device that
 * loads the library holds that array until the process exits.
 *
 * Limits: at most 4096 packets and 16,380 tiles (a tile is one to four chunks of 128 to
 * 1024 codewords, at most 4 KB of input, or a packet's tail); larger batches
 * return HD_ERR_CAPACITY before anything is enqueued.  This path decodes n = 7
 * without the decode table, so it never fills or synchronises anything.
 * First call on a device: performs a one-time set-up (it looks up the array's
 * device address and the kernel's launch attributes); make that first call
 * before any stream capture.
 * Every call reuses the same array, which keeps the previous call's tables:
 * the claim counter is cleared on `cuda_stream` at the start of each call,
 * and two calls that overlap on the GPU (for example on two streams) race on
 * the array, so order them on one stream or synchronise between them.  The
 * tile table reaches the array through small upload kernels that carry up to
 * 480 tiles each in their launch parameters, so the call needs no host-side
 * staging and returns without waiting for the GPU.  Calls from several host
 * threads are serialised.  err_counts is overwritten as in hd_decode_batch(). */
hd_status hd_decode_batch_noalloc(const hd_packet *table, uint32_t num_packets, unsigned long long *err_counts,
                                  void *cuda_stream);

/* Number of tiles (the batch kernel's work items) the packets of `table` are
 * cut into, in *tiles: the unit of hd_decode_batch_noalloc()'s capacity and of
 * hd_server_config.max_wave_tiles.  A packet of N codewords of length n gives
 * ceil(F / c) full tiles of c chunks plus ceil((N - F * chunk) / 1024) tail
 * tiles, where chunk = 1024 codewords for n <= 31, 512 for n = 63, 256 for
 * n = 127 and 128 for n = 255, F = floor(N / chunk) (0 for n = 3), and c = 4
 * for n = 7, 2 for n = 15, else 1.  Host-only: checks n (HD_ERR_INVALID_N),
 * syn_type (HD_ERR_INVALID_ARG) and sizes (HD_ERR_SIZE) but no pointers. */
hd_status hd_batch_tiles(const hd_packet *table, uint32_t num_packets, uint64_t *tiles);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of arriving packets.
 *
 * A server owns a scheduler thread and `max_waves` wave slots (one CUDA
 * stream each).  Packets are submitted from any thread, either resident in
 * device memory (hd_server_submit) or in pinned host memory
 * (hd_server_submit_host); whenever a slot is free the scheduler admits
 * waiting packets in arrival order, as many as the slot's limits and the
 * device-memory budget (in + out + syndrome bytes of admitted, unfinished
 * packets <= mem_cap_bytes) allow, and launches them as one batched decode on
 * that slot's stream.  A wave that carries host packets first gathers their
 * input into the slot's device staging (one copy kernel reading the pinned
 * buffers), and after the decode scatters data bits and syndromes back into
 * the caller's host buffers (a second copy kernel), all on the slot's stream.
 * Waves on different slots overlap on the GPU, so packets arriving while
 * others are being copied or decoded start as soon as a slot and budget free
 * up: the paper's asynchronous pipelining of successive packets (Sec. III-B,
 * Fig. 5, Eq. 1).  Results are exactly those of hd_decode() on each packet
 * alone.
 * ------------------------------------------------------------------------- */
typedef struct hd_server hd_server;

typedef struct {
    uint32_t max_waves;          /* wave slots (concurrent batched launches), 1..64 */
    uint32_t max_wave_packets;   /* packets per wave */
    uint32_t max_wave_tiles;     /* tile-table capacity per wave (a packet of N codewords needs <= N/128 + 1) */
    uint32_t queue_capacity;     /* submitted packets waiting for admission */
    uint64_t mem_cap_bytes;      /* admission budget in bytes (see above) */
    uint64_t host_staging_bytes; /* device staging per slot for host packets (0: hd_server_submit_host is refused);
                                    a host packet takes its input, output and syndrome sizes, each rounded up
                                    to 16 bytes */
} hd_server_config;

typedef struct {
    uint64_t tag;         /* the caller's tag from hd_server_submit */
    uint64_t err_count;   /* nonzero syndromes in the packet (0 unless status is HD_OK or HD_ERR_TIMEOUT) */
    uint64_t t_submit_ns; /* steady-clock times: submitted, admitted into a wave (0 if never), completion seen */
    uint64_t t_admit_ns;
    uint64_t t_done_ns;
    int32_t status;       /* HD_OK; HD_ERR_TIMEOUT if a bounded wait of its wave's kernel ran out (the
                             outputs are then not to be trusted); HD_ERR_CUDA if its wave failed or the
                             server had failed before admitting it */
} hd_completion;

typedef struct {
    uint64_t submitted, completed, rejected; /* rejected: submissions refused because the queue was full */
    uint64_t waves;                          /* batched launches */
    uint64_t max_resident_bytes;             /* high-water mark of the admission budget */
    double mean_wave_packets;
    /* filled by hd_serve_trace / hd_serve_trace_host: latency from scheduled arrival to completion */
    double p50_latency_us, p99_latency_us, max_latency_us;
    double duration_s;           /* first arrival to last completion */
    uint64_t backpressure_waits; /* submissions retried because the queue was full */
    /* waves that carried host packets, and the mean stage times of one in four of them, measured by
       CUDA events on the slot's stream: gather (T_PS), batched decode (T_DKE), scatter (T_PR) */
    uint64_t host_waves;
    double mean_t_in_us, mean_t_decode_us, mean_t_out_us;
    /* filled by the trace replays: the 99.9th latency percentile, and the largest delay between a
       packet's scheduled arrival and its submission (the replaying thread's own lateness) */
    double p999_latency_us, max_submit_lag_us;
} hd_server_stats;

/* Create a server on the current device (allocates its slots: per slot a
 * stream, events, device tile and copy tables, host_staging_bytes of device
 * staging and pinned host staging) and performs the batch kernel's one-time
 * set-up, so that the first wave pays none of it. */
hd_status hd_server_create(const hd_server_config *cfg, hd_server **server);

/* Queue one packet (device buffers as in hd_packet; they must stay valid until
 * its completion is polled).  Thread-safe.  HD_ERR_CAPACITY when the queue is
 * full or the packet alone exceeds the budget or a wave's tile capacity; the
 * server's error once it has failed. */
hd_status hd_server_submit(hd_server *server, const hd_packet *packet, uint64_t tag);

/* Queue one packet whose in, out and syndromes buffers are pinned HOST memory
 * (cudaMallocHost, cudaHostAlloc or cudaHostRegister; 16-byte aligned; sizes
 * as in hd_packet).  The input is read and the results written by the
 * packet's wave; the buffers must stay valid until its completion is polled.
 * HD_ERR_INVALID_ARG when the server has no host staging or a buffer is not
 * pinned host memory that kernels can reach; HD_ERR_CAPACITY as
 * hd_server_submit, or when the packet alone exceeds host_staging_bytes. */
hd_status hd_server_submit_host(hd_server *server, const hd_packet *packet, uint64_t tag);

/* Move up to `max` completions (in completion order) to `out`; *count gets the
 * number moved.  Returns the server's sticky error, if any. */
hd_status hd_server_poll(hd_server *server, hd_completion *out, uint32_t max, uint32_t *count);

/* Wait until every submitted packet has completed (HD_ERR_TIMEOUT after
 * timeout_ns; the server's error at once if it has failed). */
hd_status hd_server_drain(hd_server *server, uint64_t timeout_ns);

hd_status hd_server_get_stats(hd_server *server, hd_server_stats *stats);

/* Failure injection for tests, on the host: the server's next `count` wave
 * launches fail as a CUDA launch error would, before anything of those waves
 * is enqueued.  A failed wave completes its packets with HD_ERR_CUDA, the
 * server keeps HD_ERR_CUDA as its error, admits nothing more and completes
 * every waiting packet with that error.  No GPU work fails. */
hd_status hd_server_inject_launch_failures(hd_server *server, uint32_t count);

/* Finish the admitted and queued packets, stop the scheduler and free the slots. */
void hd_server_destroy(hd_server *server);

/* Replay an open-loop arrival trace through a fresh server: packet j is
 * submitted at arrival_s[j] seconds (non-decreasing) after the start, with tag
 * j; completions[j] receives its completion.  Fills stats including the
 * p50/p99 latency from scheduled arrival to observed completion. */
hd_status hd_serve_trace(const hd_server_config *cfg, const hd_packet *packets, const double *arrival_s,
                         uint32_t num, hd_completion *completions, hd_server_stats *stats);

/* hd_serve_trace with every packet submitted from pinned host memory
 * (hd_server_submit_host): the latency includes the copies in and out. */
hd_status hd_serve_trace_host(const hd_server_config *cfg, const hd_packet *packets, const double *arrival_s,
                              uint32_t num, hd_completion *completions, hd_server_stats *stats);

/* Human-readable name of a status code (static storage). */
const char *hd_status_string(hd_status status);

/* Reads and clears the device status word of the current device: 0 when no
 * bounded device-side wait has run out since the last call, otherwise a
 * nonzero code (HD_ERR_TIMEOUT).  Synchronises the device. */
hd_status hd_device_status(uint32_t *status);

/* Number of kernels this library has launched in this process (a host-side
 * counter, incremented once per kernel launch it enqueues). */
uint64_t hd_launch_count(void);

/* Cap the number of CTAs (thread blocks) of every decode launch that this
 * library enqueues from now on, on every device: max_ctas = 0 (the default)
 * removes the cap.  The persistent kernels then give each warp more chunks or
 * tiles to walk through; results never change.  Uses: leaving SMs free for
 * other kernels that run beside the decoder, and tests that make every warp's
 * staging ring wrap many times on inputs small enough for the CPU oracle.
 * Launch geometry already recorded in a CUDA graph (a plan's graph, recorded
 * on its first launch) keeps its grid.  Host only; always HD_OK. */
hd_status hd_set_max_ctas(uint32_t max_ctas);

/* The cap set by hd_set_max_ctas() (0 = none). */
uint32_t hd_get_max_ctas(void);

/* Library version, major*10000 + minor*100 + patch. */
int hd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HD_H */
