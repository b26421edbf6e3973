/*
 * hpdr.h -- C ABI of the GB300 (sm_103a) error-bounded multilevel compressor.
 *
 * The library implements the data-parallel path of the MGARD reduction
 * pipeline of "HPDR: High-Performance Portable Scientific Data Reduction
 * Framework" (Sec. IV-A, Alg. 1: multilevel decomposition with per-level
 * interpolation coefficients and an L2-projection correction computed by a
 * mass-matrix multiply and a tridiagonal solve along every dimension, then
 * level-scaled linear quantization; Sec. IV-B, Alg. 2: histogram, canonical
 * Huffman codebook, encoding and serialization into one bitstream) and its
 * inverse.  Every step runs in hand-written CUDA kernels.
 *
 * Common conventions
 *   - Arrays are row-major with the last dimension contiguous; 1 <= ndim <= 3
 *     and every dims[k] >= 2 (squeeze size-1 dimensions before calling).
 *   - Pointers named d_* are CUDA device pointers on the context's device;
 *     h_* are host pointers; the caller owns every buffer it passes.  The
 *     context owns only its cached plans and workspaces (reused across calls,
 *     grown on demand; the reductions themselves allocate nothing once the
 *     workspace is large enough).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All work is
 *     enqueued on it.  Calls that return a size to the host (compress,
 *     decompress) synchronize that stream once before returning.
 *   - Coefficient streams (decompose/recompose and their adjoints) are
 *     level-major: level 0 (every node of the coarsest grid, row-major), then
 *     for l = 1..L the nodes that are new on level l, in row-major order of
 *     their level-l grid index.  Level l therefore starts at N_{l-1}, the node
 *     count of level l-1.  Element type = dtype.
 *   - Hierarchy: node i of a dimension sits at coordinate i (unit spacing)
 *     unless the *_coords entry points give node coordinates; one coarsening
 *     keeps every other node plus the last one; all dimensions coarsen
 *     together, L = the smallest per-dimension number of coarsenings that
 *     reaches two nodes.
 *   - Node coordinates (Sec. IV-A: MGARD reduces uniform and non-uniform
 *     grids alike): `coords` is a HOST array of dims[0] + ... + dims[ndim-1]
 *     doubles, the coordinates of dimension 0's nodes, then dimension 1's,
 *     and so on, each run finite and strictly increasing (else HPDR_ERR_ARG).
 *     Interpolation weights, mass matrices, the correction solves and the
 *     correction norms behind the bins all follow them.  The library copies
 *     them into its plan cache (keyed by their bytes); the caller keeps
 *     ownership.  NULL means unit spacing, identical to the plain entries.
 *   - No exception crosses the ABI.  Errors are reported by the returned
 *     status; a failing call leaves the output buffer's contents undefined.
 *   - Calls on one context must not overlap in time (one host thread at a
 *     time per context); use one context per host thread.
 */
#ifndef HPDR_H
#define HPDR_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HPDR_OK = 0,
    HPDR_ERR_ARG = -1,       /* invalid argument (dims, dtype, tolerance, null pointer) */
    HPDR_ERR_CUDA = -2,      /* a CUDA runtime call or kernel failed */
    HPDR_ERR_CAPACITY = -3,  /* output buffer too small */
    HPDR_ERR_FORMAT = -4,    /* malformed or corrupted container */
    HPDR_ERR_TIMEOUT = -5,   /* a bounded device-side wait gave up */
    HPDR_ERR_NOMEM = -6      /* device allocation of a workspace failed */
} hpdr_status;

typedef enum { HPDR_F32 = 0, HPDR_F64 = 1 } hpdr_dtype;
/* Norm of the error bound.  LINF: max |u - u~| <= tau.  L2: tau from the RMS
 * of u (REL), with the max-norm bins, so max |u - u~| <= tau as well.
 * L2_STAT: statistical L2 bins (the paper names an L2 mode without a rule):
 * q_l = sqrt(12 tau'^2 T / ((L+1) S_l)), S_l the level-l P1 mass-matrix
 * diagonal summed over the level's new nodes and T its sum over all finest
 * nodes, which bounds the EXPECTED squared L2 error by tau'^2 T (errors
 * uniform and independent; the level components are L2-orthogonal), i.e. an
 * RMS error of about tau or less; no per-field guarantee. */
typedef enum { HPDR_LINF = 0, HPDR_L2 = 1, HPDR_L2_STAT = 2 } hpdr_mode;
typedef enum { HPDR_ABS = 0, HPDR_REL = 1 } hpdr_tol_kind;  /* REL: tol x norm of the input */

typedef struct hpdr_ctx hpdr_ctx;

/* Tunables of the lossless stage (Alg. 2).  dict_size D: quantized codes k
 * with |k| < D/2 become symbols k + D/2; others are escaped (symbol 0, with
 * k written after its codeword); even, 4 <= D <= 65536; default 8192.
 * chunk K: symbols per decode chunk (the chunk table stores the bit offset of
 * every K-th symbol); multiple of 128, 128 <= K <= 32768; default (0): chosen
 * from the field's N values, 1024 for N >= 2^27, 512 for N >= 2^26, else 256
 * (every chunk is one sequential decode, so smaller fields take shorter ones).
 * A zero field selects the default. */
typedef struct {
    uint32_t dict_size;
    uint32_t chunk;
} hpdr_config;

/* Create a context on CUDA device `device`.  *ctx receives the handle.
 * Errors: HPDR_ERR_ARG (null ctx, bad device), HPDR_ERR_CUDA. */
hpdr_status hpdr_ctx_create(hpdr_ctx **ctx, int device);

/* Release the context's workspaces and plans.  Waits for nothing: the caller
 * must make sure no work of this context is still running. */
hpdr_status hpdr_ctx_destroy(hpdr_ctx *ctx);

/* Upper bound of the container size for a field, with the given config (NULL
 * = defaults): header, bins, room for node coordinates, code lengths, chunk table and ceil(log2 D) + 32
 * bits per value (a Huffman code never exceeds the fixed-length code of
 * ceil(log2 D) bits in total; an escape payload takes at most 32 bits while
 * |k| < 2^31).  Only tolerances so small that many codes reach |k| >= 2^31
 * can exceed it; hpdr_compress then returns HPDR_ERR_CAPACITY.  0 on bad
 * arguments. */
size_t hpdr_compress_bound(int ndim, const size_t *dims, hpdr_dtype dtype, const hpdr_config *cfg);

/* Compress a device-resident field (Alg. 1 then Alg. 2).
 *   d_in        device array, ndim/dims as above, element type dtype.
 *   tol, tol_kind, mode: the error bound.  REL: tau = tol * max|u| (LINF) or
 *               tol * rms(u) (L2, L2_STAT); ABS: tau = tol.  With LINF and L2
 *               the reconstruction satisfies max|u - u~| <= tau (which also
 *               bounds the RMS error); with L2_STAT its expected RMS error is
 *               at most about tau (see hpdr_mode).
 *   d_out       device buffer of out_capacity bytes receiving the container
 *               (format v3: 128-byte header, bins, code lengths, chunk table,
 *               bitstream; every section 16-byte aligned).  A code k whose
 *               symbol k + D/2 falls outside [1, D-1] is escaped: symbol 0,
 *               followed in the bitstream by zigzag(k) in W bits, W the
 *               largest bit length among the container's escapes (header).
 *   out_bytes   host pointer receiving the container size.
 * Errors: HPDR_ERR_ARG (including a bound below the data type's precision
 * floor, tau <= 32 (L+1) eps max|u|, or a code with |k| >= 2^62),
 * HPDR_ERR_CAPACITY, HPDR_ERR_NOMEM,
 * HPDR_ERR_CUDA.  Synchronizes `stream` once. */
hpdr_status hpdr_compress(hpdr_ctx *ctx, const void *d_in, hpdr_dtype dtype, int ndim,
                          const size_t *dims, double tol, hpdr_tol_kind tol_kind, hpdr_mode mode,
                          const hpdr_config *cfg, void *d_out, size_t out_capacity,
                          size_t *out_bytes, void *stream);

/* hpdr_compress on a grid with the given node coordinates (host array, see
 * Common conventions; NULL = unit spacing, the same container as
 * hpdr_compress).  With coordinates the container's header word at byte 48
 * carries 0x100 and the coordinates follow the bins as doubles, so
 * hpdr_decompress needs nothing else to invert it. */
hpdr_status hpdr_compress_coords(hpdr_ctx *ctx, const void *d_in, hpdr_dtype dtype, int ndim,
                                 const size_t *dims, const double *coords, double tol, hpdr_tol_kind tol_kind,
                                 hpdr_mode mode, const hpdr_config *cfg, void *d_out, size_t out_capacity,
                                 size_t *out_bytes, void *stream);

/* Decompress a device-resident container into d_out (out_capacity bytes; the
 * field's shape and type are read from the header, see hpdr_inspect; node
 * coordinates too, when the container carries them).
 * Errors: HPDR_ERR_FORMAT, HPDR_ERR_CAPACITY, HPDR_ERR_ARG, HPDR_ERR_CUDA.
 * Synchronizes `stream` once (to read the header). */
hpdr_status hpdr_decompress(hpdr_ctx *ctx, const void *d_in, size_t in_bytes, void *d_out,
                            size_t out_capacity, void *stream);

/* Compression and decompression that never wait on the host, so that a
 * caller can queue many of them back to back (the paper's host-device
 * execution model keeps the device fed, Sec. V-A).  Both return once
 * everything is queued on `stream`; errors found on the host (arguments,
 * allocation) are returned as usual, errors found on the device only through
 * d_result, a device array written when the stream reaches the end of the
 * call: 0 means success, otherwise a device status code that
 * hpdr_device_status maps to an hpdr_status.  A call may synchronize the
 * device once, when its context's workspace has to grow.
 *
 * hpdr_compress_async: as hpdr_compress (unit spacing); d_result holds two
 *   uint64 values, {container bytes, device status}, 8-byte aligned.
 * hpdr_decompress_async: the container at d_in (in_capacity readable bytes)
 *   is decoded with its header parsed on the device.  The caller passes the
 *   dtype, ndim, dims and cfg the container was compressed with; a header that
 *   disagrees with them, fails its CRC, or carries node coordinates gives the
 *   FORMAT status and leaves d_out undefined.  d_result: one uint64 (status).
 *   out_capacity must hold the field (HPDR_ERR_CAPACITY otherwise). */
hpdr_status hpdr_compress_async(hpdr_ctx *ctx, const void *d_in, hpdr_dtype dtype, int ndim, const size_t *dims,
                                double tol, hpdr_tol_kind tol_kind, hpdr_mode mode, const hpdr_config *cfg,
                                void *d_out, size_t out_capacity, uint64_t *d_result, void *stream);
hpdr_status hpdr_decompress_async(hpdr_ctx *ctx, const void *d_in, size_t in_capacity, hpdr_dtype dtype, int ndim,
                                  const size_t *dims, const hpdr_config *cfg, void *d_out, size_t out_capacity,
                                  uint64_t *d_result, void *stream);
/* The hpdr_status of a device status code (d_result of the calls above). */
hpdr_status hpdr_device_status(uint64_t code);

/* Read the shape and type of a container held in host or device memory
 * (detected).  dims receives ndim entries (3 slots must be provided).  The
 * header gets the checks of hpdr_decompress (magic, version, CRC-32, field
 * ranges, positive finite bin widths, sections inside in_bytes); a container
 * that fails one gives HPDR_ERR_FORMAT.  No kernel runs: the header of a
 * device buffer is read with one blocking copy, that of a host buffer in place. */
hpdr_status hpdr_inspect(const void *in, size_t in_bytes, hpdr_dtype *dtype, int *ndim,
                         size_t *dims);

/* Multilevel decomposition (Alg. 1 without quantization): d_coef receives the
 * level-major coefficient stream of d_u (same element count and type). */
hpdr_status hpdr_decompose(hpdr_ctx *ctx, const void *d_u, void *d_coef, hpdr_dtype dtype,
                           int ndim, const size_t *dims, void *stream);

/* Multilevel recomposition, the exact inverse of hpdr_decompose. */
hpdr_status hpdr_recompose(hpdr_ctx *ctx, const void *d_coef, void *d_u, hpdr_dtype dtype,
                           int ndim, const size_t *dims, void *stream);

/* hpdr_decompose / hpdr_recompose on a grid with the given node coordinates
 * (host array, see Common conventions; NULL = unit spacing).  Errors as for
 * the plain entries, plus HPDR_ERR_ARG for coordinates that are not finite
 * and strictly increasing along each dimension. */
hpdr_status hpdr_decompose_coords(hpdr_ctx *ctx, const void *d_u, void *d_coef, hpdr_dtype dtype,
                                  int ndim, const size_t *dims, const double *coords, void *stream);
hpdr_status hpdr_recompose_coords(hpdr_ctx *ctx, const void *d_coef, void *d_u, hpdr_dtype dtype,
                                  int ndim, const size_t *dims, const double *coords, void *stream);

/* Transpose of hpdr_recompose: maps a field-shaped gradient d_grad_u to the
 * gradient with respect to the coefficient stream (no intermediate of the
 * forward pass is needed: the map is linear). */
hpdr_status hpdr_recompose_adjoint(hpdr_ctx *ctx, const void *d_grad_u, void *d_grad_coef,
                                   hpdr_dtype dtype, int ndim, const size_t *dims, void *stream);

/* Transpose of hpdr_decompose: maps a coefficient-stream gradient to a
 * field-shaped gradient. */
hpdr_status hpdr_decompose_adjoint(hpdr_ctx *ctx, const void *d_grad_coef, void *d_grad_u,
                                   hpdr_dtype dtype, int ndim, const size_t *dims, void *stream);

/* The two transposes on a grid with the given node coordinates (host array,
 * see Common conventions; NULL = unit spacing): the transposes of
 * hpdr_recompose_coords and hpdr_decompose_coords on the same grid. */
hpdr_status hpdr_recompose_adjoint_coords(hpdr_ctx *ctx, const void *d_grad_u, void *d_grad_coef, hpdr_dtype dtype,
                                          int ndim, const size_t *dims, const double *coords, void *stream);
hpdr_status hpdr_decompose_adjoint_coords(hpdr_ctx *ctx, const void *d_grad_coef, void *d_grad_u, hpdr_dtype dtype,
                                          int ndim, const size_t *dims, const double *coords, void *stream);

/* Huffman stage alone (Alg. 2) on a device array of N uint16 symbols < D:
 * histogram, code lengths (two-queue rule, leaves sorted by (frequency,
 * symbol)), canonical codewords, encoding.  Outputs (device): d_lengths[D]
 * code length per symbol, d_chunk_bits[ceil(N/K)] bit offset of every K-th
 * symbol, d_words[words_capacity] bitstream (uint32 words, MSB first).
 * *total_bits (host) receives the bitstream length.  Synchronizes `stream`.
 * Errors: HPDR_ERR_ARG, HPDR_ERR_CAPACITY, HPDR_ERR_CUDA. */
hpdr_status hpdr_huffman_encode(hpdr_ctx *ctx, const uint16_t *d_symbols, uint64_t N, uint32_t D,
                                uint32_t K, uint8_t *d_lengths, uint64_t *d_chunk_bits,
                                uint32_t *d_words, uint64_t words_capacity, uint64_t *total_bits,
                                void *stream);

/* Inverse of hpdr_huffman_encode: decodes N symbols from the bitstream of
 * total_bits bits (ceil(total_bits/32) words) with the given code lengths and
 * chunk table (device pointers) into d_symbols.  Every chunk must end exactly
 * where the next one starts and the last one at total_bits.
 * Errors: HPDR_ERR_FORMAT (invalid stream), HPDR_ERR_ARG, HPDR_ERR_CUDA. */
hpdr_status hpdr_huffman_decode(hpdr_ctx *ctx, const uint32_t *d_words, uint64_t total_bits,
                                const uint64_t *d_chunk_bits, uint64_t N, uint32_t D, uint32_t K,
                                const uint8_t *d_lengths, uint16_t *d_symbols, void *stream);

/* One field of a batch. */
typedef struct {
    const void *d_in;        /* device array, 16-byte aligned */
    hpdr_dtype dtype;
    int ndim;
    size_t dims[3];
    double tol;
    hpdr_tol_kind tol_kind;
    hpdr_mode mode;
} hpdr_field;

/* Compress many fields of uneven shapes (each with its own bound) in one
 * replay of a CUDA graph (Sec. III-A's Map&Process over many fields).  The
 * first call with a given batch (fields, pointers, config) captures every
 * field's whole compression into one graph, in four phases over all fields:
 * the norms, bins and large levels of each field forked over K worker
 * streams (fields assigned largest first to the least-loaded stream); the
 * coarse levels of every field in one launch and every codebook in one
 * launch; each field's encoder on the workers; every header (with its size
 * and status) in one launch.  An autotuner captures K = 1, 2, 4, 8, 16, times
 * one replay of each and keeps the fastest.  Later calls with the same batch
 * only replay it (one graph launch, one wait).  Each field's container is
 * byte-identical to hpdr_compress on that field.
 *   d_out          device buffer of out_capacity bytes;
 *   out_offsets    host [nfields+1]: field i's container starts at
 *                  d_out + out_offsets[i] (256-byte aligned slots of
 *                  hpdr_compress_bound bytes); out_offsets[nfields] = bytes used;
 *   out_sizes      host [nfields]: container sizes.
 * A captured graph holds the buffers it was captured with, so a batch over
 * other buffers (inputs or d_out) is captured anew.  The context keeps the
 * four most recently used batches (each with one workspace per field);
 * capturing a fifth destroys the least recently used one.  Synchronous
 * (waits for the replay).  Errors as hpdr_compress. */
hpdr_status hpdr_compress_batched(hpdr_ctx *ctx, int nfields, const hpdr_field *fields, const hpdr_config *cfg,
                                  void *d_out, size_t out_capacity, size_t *out_offsets, size_t *out_sizes,
                                  void *stream);

/* Stream count the autotuner chose for the most recently replayed batch
 * (0: none). */
int hpdr_batched_streams(hpdr_ctx *ctx);
/* Number of captured batches the context holds (at most four). */
int hpdr_batched_cached(hpdr_ctx *ctx);

/* Compression of a host-resident field in slabs along its first dimension
 * (the host-device pipeline of Sec. V: Fig. 7 and Alg. 4 with a fixed slab
 * size).  Host-to-device copies, compression and device-to-host copies run on
 * three streams owned by the context, with two input and two output device
 * buffers; slab i+1 is copied in while slab i is compressed and slab i-1 is
 * copied out.  Every slab is compressed on its own with the given bound
 * (relative bounds use the slab's own norm, never larger than the field's,
 * so the field's bound holds).
 *   h_in        host array (pinned memory gives overlapped copies).
 *   slab_bytes  target slab size (0: 256 MiB); at least two planes per slab.
 *   h_out       host buffer of out_capacity bytes receiving the streamed
 *               container: "HPDS" directory (64 bytes + 32 per slab: first
 *               plane, planes, byte offset, bytes) followed by the slab
 *               containers (format v3) at 16-byte boundaries.
 *   out_bytes   receives the size.
 * Synchronous.  Errors as hpdr_compress. */
hpdr_status hpdr_compress_host_streamed(hpdr_ctx *ctx, const void *h_in, hpdr_dtype dtype, int ndim,
                                        const size_t *dims, double tol, hpdr_tol_kind tol_kind,
                                        hpdr_mode mode, const hpdr_config *cfg, size_t slab_bytes,
                                        void *h_out, size_t out_capacity, size_t *out_bytes);

/* Inverse of hpdr_compress_host_streamed with the same three-stream
 * pipeline: h_out (host, out_capacity bytes) receives the field. */
hpdr_status hpdr_decompress_host_streamed(hpdr_ctx *ctx, const void *h_in, size_t in_bytes, void *h_out,
                                          size_t out_capacity);

/* Lossless compression of keys: the Huffman stage of Sec. IV-B (Alg. 2:
 * histogram, codebook, encode, serialize) on its own, for byte keys
 * (key_bytes = 1, alphabet D = 256) or 16-bit keys (key_bytes = 2,
 * D = 65536).  Container "HPDL" (little endian, device memory):
 *    0 "HPDL"  4 u32 version (1)  8 u32 key_bytes  12 u32 D  16 u32 K
 *   20 u32 0   24 u64 n  32 u64 total_bits  40 u64 chunk-table offset
 *   48 u64 bitstream offset  56 u32 0  60 u32 CRC-32 of bytes [0, 60)
 *   64 code length of every symbol 0..D-1 (u8, 0 = absent)
 *   then the chunk table (u64 bit offset of every K-th key) and the
 *   bitstream (u32 words, codewords MSB first), each at a 16-byte boundary.
 * Codes are the canonical two-queue Huffman code of the keys' histogram
 * (lengths at most 63), the same as hpdr_huffman_encode's. */

/* Capacity that always holds the container of n keys (the code never exceeds
 * 8 or 16 bits per key).  K: chunk size, 0 = automatic.  0 on bad
 * arguments.  Host only. */
size_t hpdr_lossless_bound(uint64_t n, int key_bytes, uint32_t K);

/* Compresses n >= 1 keys at d_keys (device; 16-byte aligned for 16-bit keys)
 * into d_out (device, 16-byte aligned, out_capacity bytes); *out_bytes (host)
 * receives the container size.  K: chunk size (multiple of 128 in
 * [128, 32768]) or 0 for automatic.  Synchronizes stream.  Errors:
 * HPDR_ERR_ARG, HPDR_ERR_CAPACITY, HPDR_ERR_NOMEM, HPDR_ERR_CUDA. */
hpdr_status hpdr_lossless_compress(hpdr_ctx *ctx, const void *d_keys, uint64_t n, int key_bytes, uint32_t K,
                                   void *d_out, size_t out_capacity, size_t *out_bytes, void *stream);

/* Inverse of hpdr_lossless_compress: d_in (device, in_bytes) to d_keys
 * (device, keys_capacity bytes; 16-byte aligned for 16-bit keys).
 * Synchronizes stream (header read and status).  Errors: HPDR_ERR_FORMAT
 * (bad magic, version, CRC, sizes or bitstream), HPDR_ERR_CAPACITY,
 * HPDR_ERR_ARG, HPDR_ERR_CUDA. */
hpdr_status hpdr_lossless_decompress(hpdr_ctx *ctx, const void *d_in, size_t in_bytes, void *d_keys,
                                     size_t keys_capacity, void *stream);

/* Key width and count of an HPDL container (host or device pointer). */
hpdr_status hpdr_lossless_inspect(const void *in, size_t in_bytes, int *key_bytes, uint64_t *n);

/* ---- Fixed-rate ZFP (Alg. 3, Sec. IV-C) --------------------------------
 * A second compressor on its own path: the field is cut into blocks of 4^d
 * values (edge-replicated at the array border), each block aligned to its
 * largest binary exponent and made fixed point (P - 5 fraction bits, P = 32
 * or 64), decorrelated by a two-level integer S-transform per dimension,
 * reordered coarse to fine, mapped to negabinary, and its bit planes coded
 * most significant first with group tests, cut at exactly rate * 4^d bits.
 * Every block has the same size, so compression and decompression are one
 * thread per block with no coordination and no synchronization.
 * Container "HPDZ": a 64-byte header (version 1, dtype, ndim, dims, rate,
 * bits per block, block count, CRC-32 of bytes [0,60)) and the blocks' 32-bit
 * words (bits least significant first).
 *   rate   bits per value, 1..256, with rate * 4^ndim a multiple of 32 (1-D:
 *          multiples of 8; 2-D: even; 3-D: any).
 * hpdr_zfp_bound: the exact container size (0 on bad arguments).
 * hpdr_zfp_compress: d_in device array (dims >= 1, row-major), d_out 16-byte
 *   aligned; *out_bytes = hpdr_zfp_bound(...).  Does not synchronize.
 *   Errors: HPDR_ERR_ARG, HPDR_ERR_CAPACITY, HPDR_ERR_CUDA.  Non-finite
 *   values are not supported (their blocks decode to unspecified values).
 * hpdr_zfp_decompress: d_in (16-byte aligned) holds in_bytes of a container;
 *   reads the header back (synchronizes `stream` once), then decodes into
 *   d_out (out_capacity bytes, aligned to the element size).  Errors: HPDR_ERR_FORMAT,
 *   HPDR_ERR_CAPACITY, HPDR_ERR_ARG, HPDR_ERR_CUDA.
 * hpdr_zfp_inspect: dtype, ndim, dims (3 slots) and rate of a container in
 *   host or device memory. */
size_t hpdr_zfp_bound(int ndim, const size_t *dims, hpdr_dtype dtype, uint32_t rate);
hpdr_status hpdr_zfp_compress(hpdr_ctx *ctx, const void *d_in, hpdr_dtype dtype, int ndim, const size_t *dims,
                              uint32_t rate, void *d_out, size_t out_capacity, size_t *out_bytes, void *stream);
hpdr_status hpdr_zfp_decompress(hpdr_ctx *ctx, const void *d_in, size_t in_bytes, void *d_out, size_t out_capacity,
                                void *stream);
hpdr_status hpdr_zfp_inspect(const void *in, size_t in_bytes, hpdr_dtype *dtype, int *ndim, size_t *dims,
                             uint32_t *rate);

/* Adaptive chunk sizing of the host-device pipeline (Sec. V-C, Alg. 4).
 * Model of the pipeline (all sizes in bytes, throughputs in bytes/s):
 *   Phi(C)   = alpha * C + beta  for C <  c_threshold
 *            = gamma             for C >= c_threshold
 *              compression throughput on a chunk of C bytes;
 *   Theta(t) = t * h2d: bytes the host-to-device copy moves in t seconds.
 * Alg. 4 sizes the next chunk so that its copy takes as long as the
 * compression of the current one:
 *   C_next = min(Theta(C_curr / Phi(C_curr)), C_limit, bytes left). */
typedef struct hpdr_pipeline_model {
    double alpha;        /* 1/s */
    double beta;         /* bytes/s */
    double gamma;        /* bytes/s, saturated throughput */
    double c_threshold;  /* bytes */
    double h2d;          /* bytes/s */
} hpdr_pipeline_model;

/* Fit of Phi from n >= 1 profiled chunks (chunk_bytes[i] > 0, throughput[i]
 * > 0 bytes/s, any order), as Sec. V-C describes: gamma is the throughput of
 * the largest chunk; walking to smaller chunks, a chunk belongs to the
 * saturated range while its throughput is at least (1 - f) * gamma
 * (0 <= f < 1); c_threshold is the smallest chunk of that range; alpha and
 * beta are the least-squares line through the smaller chunks (one smaller
 * chunk: the line through it and (c_threshold, gamma); none: alpha = 0,
 * beta = gamma).  h2d is copied into the model.  Host only, no device work.
 * Errors: HPDR_ERR_ARG. */
hpdr_status hpdr_pipeline_fit(const double *chunk_bytes, const double *throughput, int n, double f, double h2d,
                              hpdr_pipeline_model *model);

/* Chunk plan of Alg. 4 for a field of n0 planes of plane_bytes each, cut
 * along its first dimension: the first chunk holds c_init bytes, every next
 * one min(Theta(C / Phi(C)), c_limit, what is left) for the previous chunk's
 * C (c_limit 0: no limit).  Sizes are rounded down to whole planes, at least
 * two planes per chunk, and a single plane left at the end joins the last
 * chunk.  Writes min(count, cap) plane counts to planes[] and returns the
 * count (0 on bad arguments: n0 < 2, plane_bytes 0, a model with gamma or
 * h2d <= 0).  Host only, no device work. */
size_t hpdr_pipeline_plan(const hpdr_pipeline_model *model, size_t n0, size_t plane_bytes, size_t c_init,
                          size_t c_limit, size_t *planes, size_t cap);

/* Capacity that always holds the streamed container of a field cut into
 * n_chunks chunks of planes[i] planes (sum = dims[0]) along dimension 0.
 * 0 on bad arguments.  Host only. */
size_t hpdr_streamed_bound(int ndim, const size_t *dims, hpdr_dtype dtype, const hpdr_config *cfg,
                           const size_t *planes, size_t n_chunks);

/* Profiling that builds the model on the data itself (Sec. V-C fits Phi
 * per dataset and error bound): the first planes of the host field h_in are
 * copied to the device once (timed: h2d), then device-resident compressions
 * of the first chunk_bytes[i] bytes (whole planes, at least two) are timed
 * with CUDA events, reps times each after one warm-up, keeping the fastest;
 * the pairs are fitted as hpdr_pipeline_fit with f.  Uses the context's
 * pipeline buffers.  Synchronous.  Errors as hpdr_compress, HPDR_ERR_ARG for
 * n < 1 or reps < 1. */
hpdr_status hpdr_pipeline_profile(hpdr_ctx *ctx, const void *h_in, hpdr_dtype dtype, int ndim, const size_t *dims,
                                  double tol, hpdr_tol_kind tol_kind, hpdr_mode mode, const hpdr_config *cfg,
                                  const size_t *chunk_bytes, int n, int reps, double f,
                                  hpdr_pipeline_model *model);

/* hpdr_compress_host_streamed with the chunk plan of hpdr_pipeline_plan
 * (model, c_init, c_limit) instead of equal slabs: Alg. 4.  The container is
 * the same streamed format (hpdr_decompress_host_streamed reads it); each
 * chunk's container equals hpdr_compress of the same planes.  h_out needs
 * hpdr_streamed_bound of the plan.  Synchronous.  Errors as
 * hpdr_compress_host_streamed. */
hpdr_status hpdr_compress_host_adaptive(hpdr_ctx *ctx, const void *h_in, hpdr_dtype dtype, int ndim,
                                        const size_t *dims, double tol, hpdr_tol_kind tol_kind, hpdr_mode mode,
                                        const hpdr_config *cfg, const hpdr_pipeline_model *model, size_t c_init,
                                        size_t c_limit, void *h_out, size_t out_capacity, size_t *out_bytes);

/* Decomposition for callers that cannot allocate device memory on their call
 * path -- for example a service that hands all device memory to its own pool
 * at start-up (a later cudaMalloc fails or is forbidden), or a latency-bound
 * loop that cannot pay for cudaMalloc/cudaFree, which may synchronize the
 * device.  The paper has no counterpart: this is a variant of hpdr_decompose
 * that takes no context and calls no cudaMalloc, cudaFree or other
 * allocating routine.  Its plan tables and level buffers live in one fixed
 * 16 MiB device array inside the library (every GPU that loads the library
 * holds it until the process exits).
 *   d_u, d_coef, dtype, ndim, dims, stream: as for hpdr_decompose, on the
 *   current device; d_u 16-byte aligned.
 * Limit: the tables plus three arrays of the first coarse level (N_{L-1}
 * elements each) must fit in 16 MiB -- FP32 fields up to about 213^3 nodes;
 * larger fields return HPDR_ERR_CAPACITY before any work is queued.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  The
 * tables are copied from a host image that the library keeps, per dtype and
 * shape, until the process exits.  Every call shares the one array and
 * overwrites it: calls that overlap on the GPU (on different streams, or
 * from several host threads) race. */
hpdr_status hpdr_decompose_noalloc(const void *d_u, void *d_coef, hpdr_dtype dtype, int ndim,
                                   const size_t *dims, void *stream);

/* Diagnostics (not part of the reduction; off by default).
 * hpdr_profile_enable: when on, every call of this context records CUDA
 * events around each of its kernel groups on the call's stream.
 * hpdr_profile_read: waits for the recorded events, adds their elapsed times
 * per group name, returns the number of groups (at most cap are written:
 * names[i] static strings owned by the context, ms[i] total milliseconds,
 * count[i] number of recorded intervals) and clears the records.
 * hpdr_launch_count: kernels launched by the library since it was loaded. */
hpdr_status hpdr_profile_enable(hpdr_ctx *ctx, int on);
int hpdr_profile_read(hpdr_ctx *ctx, const char **names, double *ms, long long *count, int cap);
unsigned long long hpdr_launch_count(void);

/* Failure detection (test support; not part of the reduction).  The plane
 * pipelines of the level kernels wait on mbarriers for their bulk copies;
 * every such wait gives up after a number of polls, the kernel records
 * DS_TIMEOUT, waits (with its own, long bound) for the copies it has in
 * flight and returns, and the call returns HPDR_ERR_TIMEOUT.  This sets the
 * number of polls for every later launch in the process (polls >= 0; a
 * negative value only reads it) and returns the previous value.  The
 * default, 2^20, is never reached by a healthy GPU; 0 makes the first wait
 * give up at once, which is how the tests make a wait run out without
 * stalling the GPU.  Not thread-safe against concurrent launches. */
int hpdr_debug_set_wait_limit(int polls);

/* Static description of a status code. */
const char *hpdr_status_string(hpdr_status status);

#ifdef __cplusplus
}
#endif
#endif
