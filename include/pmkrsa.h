/*
 * pmkrsa.h -- C ABI of the GB300 (sm_103a) PMKRSA library.
 *
 * PMKRSA ("A Variant RSA Acceleration with Parallelization", arXiv
 * 2111.11924) splits a message into chunks and binds chunk t to one of K RSA
 * key pairs; every chunk is then an independent modular exponentiation
 * (Section 3.1, Algorithm 1).  This library runs that hot path on one GPU:
 * split, encrypt (c = m^e mod N_k), decrypt (m = c^d mod N_k, full d or
 * CRT) and join, as hand-written CUDA kernels on the caller's stream.
 *
 * Conventions shared by every call:
 *   - Return value: PMK_OK (0) or a negative PMK_E* code.  Nothing aborts.
 *   - d_* pointers are DEVICE pointers on the context's device, owned by the
 *     caller (for example torch CUDA tensors); h_* pointers are HOST
 *     pointers owned by the caller (pinned memory gives asynchronous copies).
 *   - Device work is enqueued on `stream` (a cudaStream_t; NULL = legacy
 *     default stream) and returns before it finishes.  Errors detected on
 *     the device (an input chunk >= its modulus) are recorded in the
 *     context and reported by pmk_sync_status().
 *   - Chunk buffers hold n_chunks x nbits/32 little-endian uint32 limbs,
 *     chunk-major ("limb buffer"), and must be 16-byte aligned (EINVAL).
 *     Chunk t is bound to key t mod K, the row-per-key reshape of the i x j
 *     plaintext matrix (Section 3.1), unless the call takes explicit key
 *     indices (pmk_encrypt_chunks, pmk_decrypt_chunks).  A call takes fewer
 *     than 2^32 chunks (EINVAL otherwise).
 *   - Calls on one context are not thread-safe; use one context per thread.
 */
#ifndef PMKRSA_H
#define PMKRSA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PMK_OK 0
#define PMK_EINVAL (-1)       /* null pointer, size mismatch, unsupported width, K = 0, even e ... */
#define PMK_ERANGE (-2)       /* an input chunk was >= its modulus (device-detected) */
#define PMK_ENOMEM (-3)       /* a device or host allocation failed */
#define PMK_ECUDA (-4)        /* a CUDA runtime call failed */
#define PMK_EUNSUPPORTED (-5) /* key width not compiled into this build */
#define PMK_ETOOLARGE (-6)    /* request exceeds the fixed capacity of the allocation-free call */
#define PMK_ENOINV (-7)       /* a blinding value shares a factor with its modulus (device-detected) */
#define PMK_EKEYINDEX (-8)    /* an explicit key index was >= K (device-detected) */

typedef struct pmk_ctx pmk_ctx;         /* one GPU: device status word, staging buffers */
typedef struct pmk_keyset pmk_keyset;   /* K key pairs: host copy + device-resident tables */

/* Create a context bound to CUDA device `cuda_device`.  Allocates a small
 * device status word.  *out is set only on success. */
int pmk_create(pmk_ctx **out, int cuda_device);
/* Release the context and its device memory.  NULL is ignored. */
void pmk_destroy(pmk_ctx *ctx);

/*
 * Key initialisation (Section 1.1 steps 1a-1c; Algorithm 1 "Initialization").
 * For each of K keys: primes p != q of exactly nbits/2 bits (two top bits
 * set), N = pq, d = e^-1 mod (p-1)(q-1), plus the CRT values dp = d mod (p-1),
 * dq = d mod (q-1), qinv = q^-1 mod p.  Randomness is SplitMix64 seeded with
 * `seed`; candidates pass trial division by the odd primes below 2000,
 * gcd(e, p-1) = 1 and 40 Miller-Rabin rounds with bases (splitmix64()>>1)+2.
 * Runs on the host; then uploads the key tables to the context's device.
 *   K: 1..16383 keys.
 *   nbits: 128..8192, a multiple of 128 (EUNSUPPORTED if not built).
 *   e: odd, 3 <= e < 2^32.
 * EINVAL for a NULL ctx or out, or K, nbits or e out of range; ENOMEM or
 * ECUDA if the upload fails.  *out is set only on success.
 */
int pmk_keygen(pmk_ctx *ctx, uint32_t K, uint32_t nbits, uint64_t e, uint64_t seed, pmk_keyset **out);

/*
 * Multi-prime key initialisation (Section 2.1, multi-prime RSA): each key
 * has nprimes distinct primes r_0 .. r_{b-1} of exactly nbits/nprimes bits,
 * N = r_0 ... r_{b-1} of exactly nbits bits, d = e^-1 mod prod (r_i - 1).
 * Key k draws r_0, r_1, ... in order from its own SplitMix64 stream exactly
 * as pmk_keygen draws p and q; a candidate is also redrawn while its top
 * byte is below the least T with T^b >= 2^(8b - 1), and a prime equal to an
 * earlier one is redrawn.  nprimes = 2 gives pmk_keygen's keys.
 * pmk_decrypt_chunks with use_crt then computes one residue per prime and
 * recombines them (the Chinese remainder theorem of Section 2.1);
 * encryption and full-d decryption are unchanged.
 *   nprimes: 2..4;  nbits: a multiple of 128 and of 64 nprimes, <= 8192
 *   (EINVAL otherwise; EUNSUPPORTED if nbits/(32 nprimes) limbs are not built).
 */
int pmk_keygen_multiprime(pmk_ctx *ctx, uint32_t K, uint32_t nbits, uint32_t nprimes, uint64_t e, uint64_t seed,
                          pmk_keyset **out);

/*
 * pmk_keygen_multiprime on the host only, with the output layout of
 * pmk_keyset_export_fields (N, d) and pmk_keyset_export_primes (primes, dexp,
 * coef).  Any output pointer may be NULL.
 */
int pmk_keygen_host_multiprime(uint32_t K, uint32_t nbits, uint32_t nprimes, uint64_t e, uint64_t seed, uint32_t *N,
                               uint32_t *d, uint32_t *primes, uint32_t *dexp, uint32_t *coef);

/*
 * The same key initialisation as pmk_keygen, on the host only (no device,
 * no context): writes the key material to caller-owned host arrays with the
 * layout of pmk_keyset_export_fields.  Any output pointer may be NULL.
 */
int pmk_keygen_host(uint32_t K, uint32_t nbits, uint64_t e, uint64_t seed, uint32_t *N, uint32_t *d, uint32_t *p,
                    uint32_t *q, uint32_t *dp, uint32_t *dq, uint32_t *qinv);

/*
 * Build a key set from given primes (K x nbits/64 limbs each, key-major,
 * little-endian): derives N, d, dp, dq, qinv and the device tables.  The
 * caller guarantees p, q prime, p != q, each exactly nbits/2 bits with the
 * top two bits set, gcd(e, p-1) = gcd(e, q-1) = 1 (EINVAL if a cheap check fails).
 */
int pmk_keyset_from_primes(pmk_ctx *ctx, uint32_t K, uint32_t nbits, uint64_t e, const uint32_t *p,
                           const uint32_t *q, pmk_keyset **out);

/*
 * Build a multi-prime key set from given primes: K x nprimes x
 * nbits/(32 nprimes) limbs, key-major (the layout of
 * pmk_keyset_export_primes).  Derives N, d, the CRT values and the device
 * tables.  The caller guarantees the primes are prime; EINVAL if a cheap
 * check fails: each odd with exactly nbits/nprimes bits and its top two bits
 * set, gcd(e, r_i - 1) = 1, pairwise distinct, N of exactly nbits bits.
 */
int pmk_keyset_from_primes_multi(pmk_ctx *ctx, uint32_t K, uint32_t nbits, uint32_t nprimes, uint64_t e,
                                 const uint32_t *primes, pmk_keyset **out);

/* Copy the key material out field by field (host arrays, key-major,
 * little-endian limbs): N, d: K x nbits/32;  p, q, dp, dq, qinv: K x nbits/64.
 * Any pointer may be NULL.  For a key set with more than two primes p .. qinv
 * must be NULL (EINVAL): use pmk_keyset_export_primes.  The serialised form
 * of the whole key set is pmk_keyset_export. */
int pmk_keyset_export_fields(const pmk_keyset *ks, uint32_t *N, uint32_t *d, uint32_t *p, uint32_t *q, uint32_t *dp,
                      uint32_t *dq, uint32_t *qinv);
/* The primes of every key and their CRT values, K x b x nbits/(32 b) limbs
 * each (b = pmk_keyset_num_primes): primes r_i, dexp_i = d mod (r_i - 1),
 * coef_0 = r_1^-1 mod r_0, coef_1 = 0, coef_i = (r_0 ... r_{i-1})^-1 mod r_i.
 * Any pointer may be NULL. */
int pmk_keyset_export_primes(const pmk_keyset *ks, uint32_t *primes, uint32_t *dexp, uint32_t *coef);
/*
 * Versioned key-set serialisation: the Initialization output of Algorithm 1
 * (public [E, N] and private [D, N] of every key, Section 3.1) with the
 * primes and CRT values of Section 2.1, for checkpointing a key set and
 * restoring it in another process.  Layout (every integer little-endian,
 * whatever the host's byte order):
 *   bytes 0-3    "PMKK"
 *   bytes 4-7    version (1)
 *   bytes 8-11   K
 *   bytes 12-15  nbits
 *   bytes 16-19  b, primes per modulus (2 for an ordinary key)
 *   bytes 20-23  0 (reserved)
 *   bytes 24-31  e
 *   then for each key, five rows of s = nbits/32 uint32 limbs: N, d,
 *   primes, dexp, coef (the last three as pmk_keyset_export_primes writes
 *   them: b values of s/b limbs each)
 *   last 8 bytes  FNV-1a 64-bit hash of every byte before it.
 * Size: 32 + 20 K s + 8 bytes.
 * pmk_keyset_export: with buf NULL, *len receives the size; otherwise
 * *len is the buffer's size in bytes (EINVAL, with *len set to the size
 * needed, if smaller) and receives the bytes written.  EINVAL for a NULL
 * key set or len.
 * pmk_keyset_import: checks the magic, version, sizes, hash and ranges,
 * derives every key again from its primes exactly as
 * pmk_keyset_from_primes_multi does, and refuses the blob (EINVAL) unless
 * the stored N, d, dexp and coef equal the derived ones.  With a context the
 * key tables are uploaded to its device (EUNSUPPORTED if the width is not
 * built, ENOMEM or ECUDA if the upload fails); with ctx NULL the key set is
 * host-only: it can be exported and queried, and device calls refuse it
 * (EINVAL).  *out is set only on success.
 */
int pmk_keyset_export(const pmk_keyset *ks, void *buf, size_t *len);
int pmk_keyset_import(pmk_ctx *ctx, const void *buf, size_t len, pmk_keyset **out);
/* Key-set properties: primes per modulus (b), key count K, width nbits and
 * public exponent e.  Each returns 0 for NULL. */
uint32_t pmk_keyset_num_primes(const pmk_keyset *ks);
uint32_t pmk_keyset_num_keys(const pmk_keyset *ks);
uint32_t pmk_keyset_nbits(const pmk_keyset *ks);
uint64_t pmk_keyset_e(const pmk_keyset *ks);
/* Release host and device memory of the key set.  NULL is ignored. */
void pmk_keyset_free(pmk_keyset *ks);

/* Plaintext bytes per chunk, nbits/8 - 1 (so every chunk is < N), and the
 * chunk count ceil(msg_len / payload) of a message (Section 3.1 split). */
size_t pmk_payload_bytes(uint32_t nbits);
size_t pmk_num_chunks(size_t msg_len, uint32_t nbits);

/*
 * Split (Section 3.1): chunk t = message bytes [tP, min((t+1)P, L)) read as
 * a little-endian integer, zero-extended to nbits/32 limbs.
 *   d_msg: msg_len bytes (device), any alignment.  d_chunks: n_chunks x
 *   nbits/32 uint32 (device, 16-byte aligned), n_chunks must equal
 *   pmk_num_chunks(msg_len, nbits).
 * EINVAL for a NULL ctx or buffer, nbits outside 128..8192 or not a multiple
 * of 128, a chunk count that does not match, or a misaligned d_chunks.
 */
int pmk_split(pmk_ctx *ctx, uint32_t nbits, const uint8_t *d_msg, size_t msg_len, uint32_t *d_chunks,
              size_t n_chunks, void *stream);

/*
 * Join (the "merge and output" step of Section 3.3): inverse of pmk_split.
 * Writes the low P bytes of every chunk, concatenated and cut to msg_len;
 * nothing outside d_msg[0, msg_len) is written.  Same arguments and errors
 * as pmk_split (d_chunks 16-byte aligned, d_msg any alignment).
 */
int pmk_join(pmk_ctx *ctx, uint32_t nbits, const uint32_t *d_chunks, size_t n_chunks, uint8_t *d_msg,
             size_t msg_len, void *stream);

/*
 * Encryption (Algorithm 1 "Encryption", c = m^e mod N; Algorithm 2 over
 * Algorithm 3 Montgomery products): d_out[t] = d_in[t]^e mod N_k.
 * d_in, d_out: n_chunks limb buffers (device); they may be the same buffer.
 * d_key_idx: NULL binds chunk t to key k = t mod K (the column-by-column
 *   fill of the i x j matrix with one row per key, Section 3.1); otherwise
 *   a device array of n_chunks uint32 (4-byte aligned, fewer than 2^31
 *   chunks), chunk t bound to key d_key_idx[t], any reshape the caller
 *   chose.  The library groups the chunks by key on the device (a count,
 *   an offset scan and a scatter into a key-group table in the context's
 *   stream-ordered staging) so that every block of the exponentiation
 *   kernel serves one key; results go to each chunk's own position.  An
 *   index >= K is reported as PMK_EKEYINDEX by pmk_sync_status() and that
 *   chunk's output is left unwritten.
 * A chunk >= N is reported as PMK_ERANGE by pmk_sync_status().
 */
int pmk_encrypt_chunks(pmk_ctx *ctx, const pmk_keyset *ks, const uint32_t *d_in, uint32_t *d_out,
                       size_t n_chunks, const uint32_t *d_key_idx, void *stream);

/*
 * Decryption (Algorithm 1 "Decryption", m = c^d mod N):
 * d_out[t] = d_in[t]^{d_k} mod N_k, with k = t mod K (d_key_idx NULL) or
 * k = d_key_idx[t], exactly as for pmk_encrypt_chunks.  use_crt = 0: one
 * full-width exponentiation; use_crt = 1: the CRT form of Section 2.1
 * (one exponentiation per prime over nbits/b bits -- two halves for an
 * ordinary key, b for a multi-prime key -- then the CRT recombination
 * sum_i m_i c_i mod N, c_i = (N/r_i) ((N/r_i)^-1 mod r_i)), bit-identical.
 * With use_crt = 0, d_in and d_out may be the same buffer; with use_crt = 1
 * they must not overlap (EINVAL).  EINVAL also for a NULL or misaligned
 * argument or a key set of another device; a chunk >= N is reported as
 * PMK_ERANGE by pmk_sync_status().
 */
int pmk_decrypt_chunks(pmk_ctx *ctx, const pmk_keyset *ks, const uint32_t *d_in, uint32_t *d_out,
                       size_t n_chunks, const uint32_t *d_key_idx, int use_crt, void *stream);

/*
 * The plain GPU formulation, kept as a measured baseline for the kernels
 * above: one thread per chunk, single-thread Montgomery products and
 * Algorithm 2's binary exponentiation, one launch per call.
 * d_out[t] = d_in[t]^E mod N_{t mod K} with E = d (decrypt != 0) or e.
 * Built for 1024- and 2048-bit keys only (PMK_EUNSUPPORTED otherwise).
 */
int pmk_modexp_chunks_baseline(pmk_ctx *ctx, const pmk_keyset *ks, const uint32_t *d_in, uint32_t *d_out,
                               size_t n_chunks, int decrypt, void *stream);

/*
 * PMKRSA encryption with the random matrix R (Algorithm 1 "Encryption",
 * Section 3.1): for every chunk, with k = t mod K,
 *   c_t = m_t^e,  c*_t = c_t r_t^e,  c_r,t = r_t^e   (mod N_k).
 * d_r holds the caller's random values r_t (< N_k, drawn fresh per message),
 * same layout as the chunks.  Outputs d_cstar (C*) and d_cr (C_R); the four
 * buffers must not overlap.  Chunks or r values >= N report PMK_ERANGE.
 */
int pmk_encrypt_blinded(pmk_ctx *ctx, const pmk_keyset *ks, const uint32_t *d_m, const uint32_t *d_r,
                        uint32_t *d_cstar, uint32_t *d_cr, size_t n_chunks, void *stream);

/*
 * PMKRSA decryption with R (Algorithm 1 "Decryption"): the paper computes
 * r' = c_r^d, m* = c*^d, m' = m* r'^-1 (mod N).  This library computes the
 * same residue as m' = (c* c_r^-1)^d: the inverse of c_r comes from one
 * Fermat exponentiation per prime (c_r^(r_i - 2) mod r_i: p and q for an
 * ordinary key) and their CRT recombination, followed by one exponentiation
 * by d (full width, or the Section 2.1 CRT form with use_crt = 1).  A c_r sharing a factor
 * with N reports PMK_ENOINV through pmk_sync_status.  Buffers must not overlap.
 */
int pmk_decrypt_blinded(pmk_ctx *ctx, const pmk_keyset *ks, const uint32_t *d_cstar, const uint32_t *d_cr,
                        uint32_t *d_m, size_t n_chunks, int use_crt, void *stream);

/*
 * Whole-message calls on HOST buffers: copy in, split/encrypt (or
 * decrypt/join) on the device, copy out, synchronise the stream.  The
 * context keeps grow-only device staging buffers between calls, allocated
 * and freed in stream order (cudaMallocAsync / cudaFreeAsync); a call waits
 * on its own stream for the previous call's use of them, whatever stream
 * that was.
 *   h_cipher: n_chunks x nbits/32 uint32 with n_chunks = pmk_num_chunks(msg_len, nbits).
 * Returns the device status as pmk_sync_status() would.  On an error after
 * the copy of the caller's input was queued, the stream is synchronised
 * before the call returns, so no copy from or to the caller's buffers is
 * left in flight.
 */
int pmk_encrypt_message_host(pmk_ctx *ctx, const pmk_keyset *ks, const uint8_t *h_msg, size_t msg_len,
                             uint32_t *h_cipher, size_t n_chunks, void *stream);
int pmk_decrypt_message_host(pmk_ctx *ctx, const pmk_keyset *ks, const uint32_t *h_cipher, size_t n_chunks,
                             uint8_t *h_msg, size_t msg_len, int use_crt, void *stream);

/*
 * Allocation-free variant of pmk_decrypt_message_host.  The paper has no
 * counterpart of this call.  It exists for callers that must not let the
 * library call cudaMalloc: for example a process whose device memory is
 * handed entirely to another allocator under a fixed budget, or a
 * latency-critical path that cannot pay for a device allocation.  The
 * ciphertext, the decrypted chunks and the message bytes are staged in one
 * fixed device array built into the library (32 MiB, reserved on every GPU
 * that loads the library until the process exits); no allocation routine is
 * called.  No context is needed: the key set's device is used.
 *   Capacity: 256 + 2 * round_up_256(n_chunks * nbits/8) + round_up_256(msg_len)
 *   bytes must fit in 32 MiB, else PMK_ETOOLARGE and nothing is enqueued.
 *   The array is committed when the library's module that holds it is
 *   loaded.  Under CUDA's lazy module loading (the default) that happens in
 *   the first call on a device, whose one-time set-up looks up the array's
 *   device address; if the device's memory is already taken by then, that
 *   call fails with PMK_ECUDA.  A call with n_chunks = msg_len = 0 (h_cipher
 *   and h_msg may be NULL) performs only that set-up: make one at start-up,
 *   before another allocator claims the device's memory.
 *   All calls share the array and it keeps the last call's contents: calls
 *   whose GPU work overlaps (other streams, other host threads) race and
 *   corrupt each other's results.
 *   The call ends by synchronising `stream`, so it must not be made while
 *   `stream` is being captured into a CUDA graph.  It runs the built-in
 *   default kernel geometry and odd-power table of each width, not a
 *   context's autotuned ones (it takes no context), so its speed can differ
 *   from pmk_decrypt_message_host's.
 *   Returns PMK_OK, PMK_ERANGE (a chunk >= its modulus), PMK_EINVAL (NULL
 *   key set or buffer, a chunk count that does not match msg_len, or 2^32
 *   chunks or more), PMK_ETOOLARGE or PMK_ECUDA.  On an error after the copy
 *   of h_cipher was queued, the stream is synchronised before the call
 *   returns, so no copy from or to the caller's buffers is left in flight.
 */
int pmk_decrypt_message_host_noalloc(const pmk_keyset *ks, const uint32_t *h_cipher, size_t n_chunks,
                                     uint8_t *h_msg, size_t msg_len, int use_crt, void *stream);

/*
 * Batched, persistent execution (the pipeline of Section 3.3 over many
 * messages at once).  A job is one call's worth of work on a limb buffer:
 *   op = PMK_OP_ENCRYPT (c = m^e), PMK_OP_DECRYPT (m = c^d, full d) or
 *   PMK_OP_DECRYPT_CRT (Section 2.1 CRT form; d_in and d_out must not overlap),
 * over n_chunks chunks, chunk t bound to key t mod K of the job's key set.
 * Jobs may mix key sets and key widths.  pmk_batch_create plans the work:
 *   - in a batch of at most the context's direct-launch limit of jobs with
 *     chunks (pmk_set_batch_direct_max, default 256), every job gets its
 *     own grid launch (the kernel of pmk_*_chunks);
 *   - in a larger batch, a job with at least one GPU-full of
 *     exponentiations (as many as the GPU holds resident at once) gets its
 *     own grid launch, and the others are grouped by exponentiation width
 *     and mode; each group runs as one persistent kernel whose warps take
 *     tasks (up to 32/TPI chunks of one key) from a device queue, longest
 *     tasks first;
 *   - groups and launched jobs run concurrently on internal streams, widest
 *     first;
 *   - range checks, the kernels and CRT recombination are captured once into
 *     a CUDA graph (geometry: the context's current kernel configs).
 * pmk_batch_launch replays that graph on `stream` (asynchronous; errors via
 * pmk_sync_status).  The buffers named by the jobs must stay valid and keep their
 * addresses for the batch's lifetime; their contents may change between
 * launches.  Results are bit-identical to one pmk_*_chunks call per job.
 */
#define PMK_OP_ENCRYPT 0
#define PMK_OP_DECRYPT 1
#define PMK_OP_DECRYPT_CRT 2
typedef struct pmk_job {
  const pmk_keyset *ks;
  const uint32_t *d_in;  /* n_chunks x nbits/32 limbs, 16-byte aligned */
  uint32_t *d_out;       /* same shape */
  size_t n_chunks;
  int op;
} pmk_job;
typedef struct pmk_batch pmk_batch;

int pmk_batch_create(pmk_ctx *ctx, const pmk_job *jobs, size_t n_jobs, pmk_batch **out);
/* The direct-launch limit of the batches this context plans from now on:
 * batches with at most max_jobs jobs with chunks run every job as its own
 * grid launch; 0 sends every job below one GPU-full through the persistent
 * queues.  Default 256 (one launch per job measured faster up to 256 jobs,
 * the queues faster for 1,024 jobs of a few chunks).  EINVAL for a NULL
 * context.  Results do not depend on it. */
int pmk_set_batch_direct_max(pmk_ctx *ctx, size_t max_jobs);
int pmk_batch_launch(pmk_batch *batch, void *stream);
/* Tasks queued for the persistent kernels, and exponentiation kernels per
 * launch (persistent kernels plus the jobs' own grid launches). */
int pmk_batch_info(const pmk_batch *batch, size_t *n_tasks, int *n_kernels);
void pmk_batch_destroy(pmk_batch *batch);

/* Synchronise `stream`, then return (and clear) the device-side errors
 * recorded since the last call, the most specific one: PMK_EKEYINDEX before
 * PMK_ERANGE before PMK_ENOINV; PMK_OK if none; PMK_ECUDA if a CUDA call
 * fails. */
int pmk_sync_status(pmk_ctx *ctx, void *stream);
/* pmk_sync_status, and where: *first_chunk (may be NULL) receives the
 * smallest chunk index that raised a device-side error since the last
 * status call -- the index within its call (within its job for a batch);
 * with several calls between status reads, the smallest over them -- or
 * UINT64_MAX when none did.  Same return values and clearing as
 * pmk_sync_status. */
int pmk_sync_status_detail(pmk_ctx *ctx, void *stream, uint64_t *first_chunk);

/* Static description of an error code. */
const char *pmk_strerror(int code);

/*
 * Integer-pipe peak of this GPU, measured by the library's own
 * dependency-free 32x32->64 multiply-accumulate loop: MACs per clock per SM,
 * the SM clock seen during the loop (MHz) and the SM count.  Used as the
 * roofline denominator of the modular-exponentiation kernels.  Synchronous.
 * EINVAL for a NULL argument; ENOMEM or ECUDA if its buffers or launches
 * fail, or if fewer of its blocks fit on an SM than the loop assumes.
 */
int pmk_measure_int_peak(pmk_ctx *ctx, double *macs_per_clk_per_sm, double *sm_mhz, int *num_sms);

/*
 * INT32 multiply-add issue rate of this GPU, measured the same way with a
 * loop of plain 32-bit multiply-adds (mad.lo, sixteen independent chains per
 * thread): mad.lo per clock per SM, the SM clock seen (MHz) and the SM count.
 * One 32x32->64 MAC is two such operations (low and high halves); this is
 * the denominator of the kernels' "% of INT32 peak".  Like
 * pmk_measure_int_peak: EINVAL for a NULL argument, ENOMEM or ECUDA if its
 * buffers or launches fail.
 */
int pmk_measure_imad_peak(pmk_ctx *ctx, double *mad_lo_per_clk_per_sm, double *sm_mhz, int *num_sms);

/*
 * Launch geometry of the exponentiation kernels for one limb count and mode.
 *   limbs: nbits/32 for the full-width kernels (crt = 0); for the CRT
 *          kernels (crt = 1) the limbs of one prime, nbits/(32 b) for a key
 *          with b primes (nbits/64 for an ordinary key).
 *   tpi:   lanes of a warp that hold one exponentiation (a power of two
 *          dividing 32 and the limb count); 0 restores the built-in default.
 *   form:  Montgomery product form, 0 = one add-with-carry chain per lane and
 *          row, 1 = independent 64-bit column accumulators.
 * Returns EUNSUPPORTED if that geometry is not compiled in.  Results are
 * bit-identical for every geometry; only speed differs.
 */
int pmk_set_kernel_config(pmk_ctx *ctx, uint32_t limbs, int crt, uint32_t tpi, uint32_t form);
/* The geometry the context currently uses for (limbs, crt).  EINVAL for a
 * NULL argument, EUNSUPPORTED if no kernel is compiled for (limbs, crt). */
int pmk_get_kernel_config(const pmk_ctx *ctx, uint32_t limbs, int crt, uint32_t *tpi, uint32_t *form);
/* Compiled geometries for (limbs, crt): writes up to `max` (tpi, form) pairs
 * and returns how many exist (a negative code on bad arguments).  Host only. */
int pmk_list_kernel_configs(uint32_t limbs, int crt, uint32_t *tpi, uint32_t *form, int max);

/*
 * Widest sliding window of the exponentiation kernels for (limbs, crt) (the
 * left-to-right windowed form of Algorithm 2's square-and-multiply).  Each
 * exponentiation keeps a table of odd powers x, x^3, ... in shared memory:
 *   max_window = 5: 16 odd powers (the default);
 *   max_window = 4: 8 odd powers, half the shared memory, so more
 *                   exponentiations are resident per SM.
 * Every key holds a schedule for each; within the bound the host picks, per
 * exponent, the width with the fewest products.  0 restores the default.
 * The small table is compiled for the CRT residue kernels (crt = 1) of the
 * throughput geometries; a geometry without it runs with the full table,
 * and pmk_get_kernel_window reports the bound in effect for the current
 * geometry.  Returns EINVAL for any other width or a NULL context,
 * EUNSUPPORTED if no kernel for (limbs, crt) is compiled with that bound.
 * Results are bit-identical either way; pmk_autotune chooses the bound
 * together with the geometry.
 */
int pmk_set_kernel_window(pmk_ctx *ctx, uint32_t limbs, int crt, uint32_t max_window);
/* The widest window the context currently uses for (limbs, crt), for its
 * current geometry.  EINVAL for a NULL argument, EUNSUPPORTED if no kernel
 * is compiled for (limbs, crt). */
int pmk_get_kernel_window(const pmk_ctx *ctx, uint32_t limbs, int crt, uint32_t *max_window);

/*
 * Autotuner: time every compiled geometry of one exponentiation, with each
 * window bound it is compiled for (5, and 4 for the CRT residue kernels), on
 * `n_chunks` synthetic chunks of this key set
 * (mode 0 = encrypt, 1 = full-d decrypt, 2 = CRT decrypt), `reps` timed
 * launches each after one warm-up, and make the fastest the context's
 * geometry and window for that limb count and mode (as
 * pmk_set_kernel_config and pmk_set_kernel_window would).  Writes the
 * geometry and its best launch time in ms (any output pointer may be NULL);
 * pmk_get_kernel_window reads the window chosen.  Allocates and frees two
 * temporary device buffers and synchronises the device's legacy stream.
 * reps is clamped to 1..20.  EINVAL for a NULL ctx or ks, n_chunks = 0 or a
 * mode outside 0..2; EUNSUPPORTED if no kernel is compiled for the width;
 * ENOMEM or ECUDA if the temporary buffers or a launch fail (the context's
 * geometry is then left unchanged).
 */
int pmk_autotune(pmk_ctx *ctx, const pmk_keyset *ks, size_t n_chunks, int mode, int reps, uint32_t *tpi,
                 uint32_t *form, float *ms);

#ifdef __cplusplus
}
#endif

#endif /* PMKRSA_H */
