/*
 * gf.h -- C ABI of the GB300 (sm_103a) GF(2^n) network-coding library.
 *
 * The operations follow the statement of the problem in section II of
 * Guenther, Appel, Carle, "Galois Field Arithmetics for Linear Network Coding
 * using AVX 512 Instruction Set Extensions" (arXiv:1909.02871):
 *
 *   - field GF(q), q = 2^n with n in {1, 2, 4, 8} (GF(2), GF(4), GF(16),
 *     GF(256)); addition is XOR, multiplication the polynomial product
 *     reduced by x^2+x+1, x^4+x+1 and x^8+x^4+x^3+x^2+1 respectively (the
 *     paper fixes no polynomial; these are the library's reading);
 *   - a packet of len bytes holds 8*len/n words; word j of a byte occupies
 *     bits [j*n, (j+1)*n), bit i of a word is the coefficient of x^i
 *     (GF(16) is nibble-packed, GF(4) holds four words per byte);
 *   - coefficients (coding-vector entries) are stored one field element per
 *     byte, valid iff < 2^n.
 *
 * Conventions of every entry point:
 *   - pointers named dst/src/out/payload/coef are DEVICE pointers owned by
 *     the caller, unless stated otherwise; descriptor arrays (gf_gen_t,
 *     gf_dec_t) are HOST arrays that the call reads before it returns;
 *   - all work is enqueued on `stream` (NULL = legacy default stream) and the
 *     call returns without waiting for it, unless stated otherwise;
 *   - the return value is a status: GF_OK (0) or a negative GF_E* code; a
 *     call that returns an error has enqueued nothing;
 *   - no call takes torch or other framework types.
 */
#ifndef GF_GB300_H
#define GF_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t / CUstream; NULL is the legacy default stream. */
typedef struct CUstream_st *gf_stream_t;

/* Status codes. */
#define GF_OK 0
#define GF_EINVAL (-1)    /* bad field, coefficient >= 2^n, negative size, NULL pointer with len > 0 */
#define GF_EOVERLAP (-2)  /* dst and src overlap without being identical */
#define GF_ENOMEM (-3)    /* device or host allocation failed */
#define GF_ERANK (-4)     /* a decode reached rank < n_src (reported by gf_decode_check) */
#define GF_ETIMEOUT (-5)  /* a device-side wait gave up (reported by gf_device_status) */
#define GF_ECUDA (-6)     /* a CUDA runtime call or kernel launch failed */
#define GF_ENOTSUP (-7)   /* the requested path is not available on this device */
#define GF_EBUSY (-8)     /* the result asked for is not ready yet (gf_dec_status without waiting) */

/* Human-readable name of a status code (static string). */
const char *gf_strerror(int status);

/* Library version, major*10000 + minor*100 + patch. */
int gf_version(void);

/* ------------------------------------------------------------------ */
/* Region operations (section II: madd, b := b + c*a)                  */
/* ------------------------------------------------------------------ */

/*
 * gf_region_madd: dst := dst + coef * src over GF(2^field), on every word of
 * the len-byte regions (the madd operation of section II and of Algorithms 1
 * and 2 of section IV; coef 0 is a no-op and coef 1 a plain XOR, the two
 * trivial cases of section IV).
 *   field  bits per word: 1, 2, 4 or 8
 *   dst    device pointer, len bytes, read and written
 *   src    device pointer, len bytes, read; may equal dst (then dst := (1+coef)*dst)
 *   coef   field element, must be < 2^field
 *   len    bytes, any value >= 0, any alignment (16-byte aligned regions with
 *          equal alignment take the vector path)
 * Errors: GF_EINVAL (field, coef, NULL with len > 0), GF_EOVERLAP (regions
 * overlap without being identical), GF_ECUDA (launch failure).
 */
int gf_region_madd(int field, uint8_t *dst, const uint8_t *src, uint8_t coef, size_t len,
                   gf_stream_t stream);

/*
 * gf_region_mul: dst := coef * src over GF(2^field) (coef 0 zero-fills,
 * coef 1 copies).  Needed by decode to normalise a pivot row; the paper's
 * madd with a zero accumulator.  Arguments and errors as gf_region_madd;
 * dst == src multiplies in place.
 */
int gf_region_mul(int field, uint8_t *dst, const uint8_t *src, uint8_t coef, size_t len,
                  gf_stream_t stream);

/* ------------------------------------------------------------------ */
/* Generation encode (section II, Eq. 1 and Eq. 2)                     */
/* ------------------------------------------------------------------ */

/*
 * One generation to encode: the K = n_coded coded packets
 *     out_k = sum_i coef[k][i] * src_i        (Eq. 2, one row of B per packet)
 * of the N = n_src source packets (the columns of A in Eq. 1).
 *   src   device, n_src packets of len bytes, packet i at src + i*len
 *   coef  device, n_coded x n_src coefficients, row-major, one per byte
 *   out   device, n_coded packets of len bytes, packet k at out + k*len;
 *         written (not accumulated); must not overlap src or coef
 */
typedef struct gf_gen {
    int32_t field;     /* 1, 2, 4 or 8 */
    int32_t n_src;     /* N >= 0 */
    int32_t n_coded;   /* K >= 0 */
    int32_t reserved;  /* must be 0 */
    uint64_t len;      /* bytes per packet */
    const uint8_t *src;
    const uint8_t *coef;
    uint8_t *out;
} gf_gen_t;

/* Encode paths. */
#define GF_PATH_AUTO 0       /* autotuned choice per shape bucket */
#define GF_PATH_TABLE 1      /* per-coefficient split tables, prmt lookups, integer ALU */
#define GF_PATH_BITSLICED 2  /* 8x8 GF(2) bit matrices on the tensor cores (E2M1), any field */

/*
 * gf_encode_batched: encode n_gens generations (uneven N, K, len and field
 * allowed) in one persistent launch.  `gens` is a host array of n_gens
 * descriptors, read before the call returns.  Coefficients >= 2^field are
 * not detected here (they give unspecified output bytes but no fault); use
 * gf_encode_validate to check them.  Errors: GF_EINVAL (a descriptor),
 * GF_ENOMEM (library workspace), GF_ECUDA.
 */
int gf_encode_batched(const gf_gen_t *gens, int n_gens, gf_stream_t stream);

/* As gf_encode_batched with an explicit path (GF_PATH_*).  GF_PATH_BITSLICED
 * returns GF_ENOTSUP on a device without sm_103 tensor cores. */
int gf_encode_batched_ex(const gf_gen_t *gens, int n_gens, int path, gf_stream_t stream);

/*
 * gf_encode_validate: synchronously checks every coefficient of every
 * generation against its field; returns GF_OK, GF_EINVAL or GF_ECUDA.
 * Waits for `stream`.
 */
int gf_encode_validate(const gf_gen_t *gens, int n_gens, gf_stream_t stream);

/* ------------------------------------------------------------------ */
/* Decode (Gauss-Jordan elimination; the paper describes no decoder)   */
/* ------------------------------------------------------------------ */

/*
 * One generation to decode from n_recv received coded packets, in arrival
 * order.  Rows are processed in order; each is reduced against the pivots
 * found so far, dropped if it reduces to zero (not innovative), otherwise
 * normalised and used to eliminate its pivot column from the other rows;
 * processing stops when the rank reaches n_src.
 *   coef     device, n_recv x n_src coding vectors, one element per byte
 *   payload  device, n_recv packets of len bytes
 *   out      device, n_src packets of len bytes: decoded source p, or zeros
 *            if source p is not determined by the rows received
 *   rank     device int32: rank reached (== n_src on success)
 *   used     device int32 or NULL: received rows consumed
 *   solved   device, n_src bytes or NULL: 1 where out row p is decoded
 */
/* gf_dec_t.flags: the received packets are mostly sources sent uncoded
 * (systematic coding: unit coding vectors).  The rows of the transform that
 * such packets solve are unit vectors, so the payload phase runs on the
 * table path, which skips zero multipliers: about (unit rows + missing
 * sources x R) x len work instead of N x R x len.  Results are identical
 * with or without the flag. */
#define GF_DEC_SYSTEMATIC 1

typedef struct gf_dec {
    int32_t field;
    int32_t n_src;    /* N, 0 <= N <= 1024 */
    int32_t n_recv;   /* R, 0 <= R <= 4096 */
    int32_t flags;    /* 0 or GF_DEC_SYSTEMATIC; other bits must be 0 */
    uint64_t len;
    const uint8_t *coef;
    const uint8_t *payload;
    uint8_t *out;
    int32_t *rank;
    int32_t *used;
    uint8_t *solved;
} gf_dec_t;

/*
 * gf_decode_batched: decode n_gens generations.  Coefficient elimination runs
 * one CTA per generation (warp-ballot pivot search, row operations as
 * split-table region madds in shared memory); the payloads are then combined
 * by the batched encode with the elimination's transform.  Uses library
 * workspace (device memory, grown on demand).  Rank deficiency is not an
 * error of this call: read `rank`, or call gf_decode_check.
 * Errors: GF_EINVAL, GF_ENOMEM, GF_ECUDA.
 */
int gf_decode_batched(const gf_dec_t *gens, int n_gens, gf_stream_t stream);

/* Waits for `stream`, then returns GF_ERANK if any generation of `gens`
 * reached rank < n_src, else GF_OK (GF_ECUDA on a CUDA error). */
int gf_decode_check(const gf_dec_t *gens, int n_gens, gf_stream_t stream);

/*
 * gf_decode_noalloc: decode ONE generation exactly like gf_decode_batched, but
 * without allocating anything: no cudaMalloc / cudaFree, no growth of the
 * library workspace.  The paper has no counterpart; this entry point exists
 * for callers that cannot let a decode call allocate device memory -- for
 * example a packet data path that decodes each generation as its last packet
 * arrives and must not wait on the allocator, or a process whose device
 * memory is all owned by its own pool.
 *
 * Its scratch (the elimination transform, the descriptors and a work
 * counter) is a fixed array of GF_NOALLOC_SCRATCH_BYTES in the library's
 * device memory, present on every device that loads the library until the
 * process exits.  Limits: n_src * n_recv <= GF_NOALLOC_SCRATCH_BYTES - 1024,
 * and the n_src x (n_src + n_recv) elimination rows must fit one CTA's shared
 * memory (e.g. n_src = 255 with n_recv <= 560 on GB300); larger inputs return
 * GF_EINVAL.  Arguments as in gf_dec_t (device pointers; used and solved may
 * be NULL), enqueued on `stream`.
 *
 * The first call on a device looks up the array's device address (with that
 * device current) and should be made before any stream capture.  Every call
 * shares the one array, which keeps the last call's contents; calls whose
 * work overlaps on the GPU (other streams or threads) race on it.
 * Errors: GF_EINVAL, GF_ECUDA.
 */
#define GF_NOALLOC_SCRATCH_BYTES (256 * 1024)
int gf_decode_noalloc(int field, int n_src, int n_recv, uint64_t len, const uint8_t *coef, const uint8_t *payload,
                      uint8_t *out, int32_t *rank, int32_t *used, uint8_t *solved, gf_stream_t stream);

/* ------------------------------------------------------------------ */
/* Recoding at intermediate nodes                                      */
/* ------------------------------------------------------------------ */

/*
 * A node of a coded network forwards linear combinations of the coded
 * packets it has received (section II).  For one generation it holds n_in
 * coded packets with their coding vectors and makes n_out new ones with
 * fresh coefficients mix (n_out x n_in, one element per byte):
 *   payload_out_k = sum_r mix[k][r] * payload_in_r     (Eq. 2)
 *   coef_out_k    = sum_r mix[k][r] * coef_in_r        (the new packets'
 *                   coding vectors with respect to the original sources)
 *   coef_in      device, n_in x n_src, one element per byte
 *   payload_in   device, n_in x len
 *   mix          device, n_out x n_in
 *   coef_out     device, n_out x n_src
 *   payload_out  device, n_out x len
 * Outputs must not overlap the inputs.
 */
typedef struct gf_recode {
    int32_t field;
    int32_t n_src;    /* N: length of the coding vectors */
    int32_t n_in;     /* R: coded packets held */
    int32_t n_out;    /* coded packets to make */
    uint64_t len;
    const uint8_t *coef_in;
    const uint8_t *payload_in;
    const uint8_t *mix;
    uint8_t *coef_out;
    uint8_t *payload_out;
} gf_recode_t;

/* gf_recode_batched: recode n_gens generations in one batched encode launch
 * (payloads and coding vectors alike, as both are linear combinations with
 * the same coefficients; a coding vector holds one element per byte, which
 * the byte-packed field arithmetic multiplies exactly).  Errors: GF_EINVAL,
 * GF_ENOMEM, GF_ECUDA. */
int gf_recode_batched(const gf_recode_t *gens, int n_gens, gf_stream_t stream);

/* ------------------------------------------------------------------ */
/* Resident decoders: packets arrive over time (serving)               */
/* ------------------------------------------------------------------ */

/*
 * A decoder keeps one generation's received coded packets in device memory
 * that the library owns from gf_dec_open until gf_dec_close, so that a
 * server can append packets as they arrive and decode many partially
 * received generations in one launch.  The paper describes the encoder only
 * and has no counterpart; the decode itself is gf_decode_batched's
 * (progressive Gauss-Jordan in arrival order, stop at rank n_src).  A
 * decoder is used from one host thread at a time; different decoders are
 * independent.
 */
typedef struct gf_decoder gf_decoder_t;

/* Allocates a decoder for a generation of n_src packets of len bytes in
 * GF(2^field) that can hold up to max_recv received packets: device buffers
 * for the coding vectors (max_recv x n_src bytes), the payloads
 * (max_recv x len) and the decoded packets (n_src x len), from a
 * library-private stream-ordered pool of the current device that keeps freed
 * memory for reuse, and a rank word in mapped host memory.  Synchronous.  Errors: GF_EINVAL (field not in
 * {1,2,4,8}, n_src outside 1..1024, max_recv outside 1..4096, dec NULL),
 * GF_ENOMEM, GF_ECUDA. */
int gf_dec_open(int field, int n_src, int max_recv, uint64_t len, gf_decoder_t **dec);

/* Appends n received packets, in arrival order: coef (n x n_src bytes) and
 * payload (n x len bytes), in host or device memory, copied into the
 * decoder's buffers with one cudaMemcpyAsync each on `stream` (host memory
 * must stay valid until the stream has run the copy; pinned memory keeps it
 * asynchronous).  Coding vectors in host memory are also read on the host
 * for unit vectors (sources a systematic sender sent uncoded): a decoder
 * whose packets are at least half unit vectors is decoded with
 * GF_DEC_SYSTEMATIC by gf_dec_poll.  Errors: GF_EINVAL (NULL pointers with
 * n > 0, n < 0, or more than max_recv packets in total), GF_ECUDA. */
int gf_dec_push(gf_decoder_t *dec, const uint8_t *coef, const uint8_t *payload, int n, gf_stream_t stream);

/* Enqueues on `stream` ONE batched decode over every decoder in decs[0..n)
 * that holds at least n_src packets and has received packets since its
 * previous attempt; the others are left alone.  The decoded packets overwrite
 * the decoder's output buffer.  *n_launched (host, may be NULL) receives the
 * number of decoders attempted.  Asynchronous.  Packets may be pushed (on any
 * stream) while an attempt runs: they fill rows the attempt does not read.
 * A decoder must not be polled again before its previous attempt is
 * complete (gf_dec_status reports it).
 * Errors: GF_EINVAL, GF_ENOMEM (library workspace), GF_ECUDA. */
int gf_dec_poll(gf_decoder_t *const *decs, int n, gf_stream_t stream, int *n_launched);

/* Result of the decoder's latest attempt.  With wait != 0 it waits for that
 * attempt; with wait == 0 it returns GF_EBUSY while the attempt is still
 * running.  rank: rank reached (-1 if never attempted); received: packets
 * pushed so far; out: device address of the n_src x len decoded packets
 * (complete when rank == n_src, valid until gf_dec_close).  Any of the
 * three may be NULL.  Errors: GF_EINVAL, GF_EBUSY, GF_ECUDA. */
int gf_dec_status(gf_decoder_t *dec, int wait, int *rank, int *received, const uint8_t **out);

/* Enqueues on `stream` a copy of the decoder's n_src x len decoded packets
 * (as left by its latest attempt) into dst, host (pinned for asynchrony) or
 * device memory.  Errors: GF_EINVAL, GF_ECUDA. */
int gf_dec_read(gf_decoder_t *dec, uint8_t *dst, gf_stream_t stream);

/* Frees the decoder (NULL is a no-op): waits for its latest attempt, then
 * releases the buffers in stream order after the last push, poll and read
 * enqueued on any stream, without waiting for those. */
int gf_dec_close(gf_decoder_t *dec);

/* ------------------------------------------------------------------ */
/* Plans: pre-uploaded batches for CUDA graph capture                  */
/* ------------------------------------------------------------------ */

typedef struct gf_plan gf_plan_t;

/*
 * gf_encode_plan_create: uploads the descriptors and the tile work list of
 * an encode batch into library-owned device memory and fixes the path
 * (GF_PATH_AUTO consults the autotuner).  Synchronous.  The caller's device
 * buffers must stay valid while the plan is used.
 */
int gf_encode_plan_create(const gf_gen_t *gens, int n_gens, int path, gf_plan_t **plan);

/* gf_decode_plan_create: the same for a decode batch. */
int gf_decode_plan_create(const gf_dec_t *gens, int n_gens, gf_plan_t **plan);

/* A plan of gf_recode_batched's work for gens (same arguments). */
int gf_recode_plan_create(const gf_recode_t *gens, int n_gens, gf_plan_t **plan);

/* gf_plan_launch: enqueues the plan's kernels on `stream` (no allocation, no
 * host-device copy: safe inside stream capture). */
int gf_plan_launch(gf_plan_t *plan, gf_stream_t stream);

/* Number of kernel launches gf_plan_launch enqueues. */
int gf_plan_kernel_count(const gf_plan_t *plan);

/* Releases a plan (waits for the device first). NULL is ignored. */
int gf_plan_destroy(gf_plan_t *plan);

/* ------------------------------------------------------------------ */
/* Autotuner (encode tile shapes and path per shape bucket)            */
/* ------------------------------------------------------------------ */

/*
 * A shape bucket is (field, ceil(log2 n_src), ceil(log2 n_coded),
 * ceil(log2 len)).  gf_autotune_encode allocates n_gens generations of that
 * shape (device memory, freed before it returns), times every candidate --
 * the bit-sliced path where it applies and each table-path tile shape --
 * on `stream`, and records the fastest for the bucket; GF_PATH_AUTO then uses
 * it for every generation in the bucket.  Synchronous.  *path / *variant
 * (may be NULL) receive the choice.  Errors: GF_EINVAL, GF_ENOMEM, GF_ECUDA.
 */
int gf_autotune_encode(int field, int n_src, int n_coded, uint64_t len, int n_gens, gf_stream_t stream,
                       int *path, int *variant);

/* gf_autotune_last: the candidates timed by this thread's last
 * gf_autotune_encode call, in the order timed, with the mean device time of
 * one batched encode (ms, three timed runs after a warm-up run) under each:
 * up to `cap` entries into paths / variants / ms (any may be NULL); *n is
 * set to the number of candidates.  The tuner's recorded choice is the
 * candidate with the least time.  Errors: GF_EINVAL (cap < 0, n NULL). */
int gf_autotune_last(int cap, int *paths, int *variants, float *ms, int *n);

/* Record a choice for a bucket without timing (path GF_PATH_TABLE or
 * GF_PATH_BITSLICED, variant 0..3 = table tile shape). */
int gf_autotune_set(int field, int n_src, int n_coded, uint64_t len, int path, int variant);

/* The choice GF_PATH_AUTO makes for a shape (recorded, else the heuristic). */
int gf_autotune_query(int field, int n_src, int n_coded, uint64_t len, int *path, int *variant);

/* Forget every recorded choice. */
int gf_autotune_clear(void);

/* Save / load recorded choices as text lines
 * "field log2N log2K log2len path variant" (host file path). */
int gf_autotune_save(const char *path);
int gf_autotune_load(const char *path);

/* ------------------------------------------------------------------ */
/* Device status                                                       */
/* ------------------------------------------------------------------ */

/* Waits for the current device, returns and clears the library's device-side
 * error word: GF_OK, or GF_ETIMEOUT if a bounded wait inside a kernel gave up. */
int gf_device_status(void);

/* Self-test of the device-side bounded waits (the paper has no counterpart):
 * enqueues a one-warp kernel that waits on an mbarrier nothing will arrive
 * at -- with abort_first != 0, with the CTA's abort flag already set -- using
 * the same bounded wait as the tensor-core encode.  The wait gives up (after
 * its 1 s limit, or at once when aborting), the kernel records GF_ETIMEOUT in
 * the status word that gf_device_status reports and returns; nothing hangs
 * or faults and the context stays usable.  Errors: GF_ENOMEM, GF_ECUDA. */
int gf_selftest_wait(int abort_first, gf_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* GF_GB300_H */
