/*
 * hpdr_oracle.h -- plain, slow FP64 CPU oracle for the MGARD-style reduction
 * path (multilevel decomposition, level-scaled quantization, canonical
 * Huffman coding) described in Sec. IV-A (Alg. 1) and Sec. IV-B (Alg. 2) of
 * "HPDR: High-Performance Portable Scientific Data Reduction Framework".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the GPU library; the container format is
 * implemented here independently from its written definition.
 *
 * Conventions
 *   - arrays are row-major, last dimension contiguous, d = 1..3 dimensions,
 *     every n_k >= 2;
 *   - coefficient streams are level-major: level 0 (all coarsest nodes), then
 *     the nodes that are new on level 1, ..., level L; inside a level, nodes
 *     follow the row-major order of their level-grid index;
 *   - every function returns 0 on success and a negative value on a bad
 *     argument or a malformed buffer.
 */
#ifndef HPDR_ORACLE_H
#define HPDR_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Hierarchy: number of levels L and the node count of every dim per level. */
int oracle_levels(int d, const size_t *n, int *L, size_t *m_out /* [3*(L+1)], m_out[k*(L+1)+l] */);

/* Multilevel decomposition / recomposition and their transposes (FP64). */
int oracle_decompose(int d, const size_t *n, const double *u, double *coef);
/* _c variants: coords = NULL (node i at coordinate i) or the node
 * coordinates of every dimension, n[0] + ... + n[d-1] strictly increasing
 * values, dimension 0 first (MGARD's non-uniform grids) */
int oracle_decompose_c(int d, const size_t *n, const double *coords, const double *u, double *coef);
int oracle_recompose_c(int d, const size_t *n, const double *coords, const double *coef, double *u);
int oracle_correction_norms_c(int d, const size_t *n, const double *coords, double *c);
int oracle_recompose_adjoint_c(int d, const size_t *n, const double *coords, const double *g_u, double *g_coef);
int oracle_decompose_adjoint_c(int d, const size_t *n, const double *coords, const double *g_coef, double *g_u);
int oracle_bins_c(int d, const size_t *n, const double *coords, double tau_abs, double norm_inf, double eps,
                  double *q);
/* Statistical L2 bins (mode 2; the paper states no formula, see
 * hierarchy.c): S[l] = sum over the nodes new on level l (every node of level
 * 0) of the diagonal of the level-l tensor P1 mass matrix, and *T the same
 * sum over all finest nodes; q_l = sqrt(12 tau'^2 T / ((L+1) S_l)). */
int oracle_l2s_weights_c(int d, const size_t *n, const double *coords, double *S /* [L+1] */, double *T);
int oracle_bins_l2s_c(int d, const size_t *n, const double *coords, double tau_abs, double norm_inf, double eps,
                      double *q);
/* Fixed-rate ZFP (Alg. 3; the reading is in zfp.c's header).  rate = bits
 * per value (1..256); rate * 4^d must be a multiple of 32.  dtype 0 rounds the input
 * to binary32 first.  Returns 0, -1 (arguments), -3 (capacity), -4 (format). */
uint64_t oracle_zfp_bound(int d, const size_t *n, int dtype, uint32_t rate);
int oracle_zfp_compress(int d, const size_t *n, const double *u, int dtype, uint32_t rate, uint8_t *out,
                        uint64_t cap, uint64_t *out_bytes);
int oracle_zfp_decompress(const uint8_t *in, uint64_t in_bytes, double *u, uint64_t n_cap);
/* its steps, for the pins */
void oracle_zfp_fwd_line(int64_t *a, int stride);
void oracle_zfp_inv_line(int64_t *a, int stride);
void oracle_zfp_order(int d, int *perm);
uint64_t oracle_negabinary(int64_t q, int P);
int64_t oracle_from_negabinary(uint64_t u, int P);
void oracle_zfp_encode_planes(const uint64_t *u, int B, int P, uint32_t *words, uint64_t start, uint64_t end);
void oracle_zfp_decode_planes(uint64_t *u, int B, int P, const uint32_t *words, uint64_t start, uint64_t end);
int oracle_recompose(int d, const size_t *n, const double *coef, double *u);
int oracle_recompose_adjoint(int d, const size_t *n, const double *g_u, double *g_coef);
int oracle_decompose_adjoint(int d, const size_t *n, const double *g_coef, double *g_u);

/* Per-level correction operator norms c_l (l = 1..L; c[0] = 0). */
int oracle_correction_norms(int d, const size_t *n, double *c /* [L+1] */);

/* Level-scaled quantization bins q[0..L] for an absolute bound tau_abs.
 * eps = unit roundoff of the data type (2^-24 or 2^-53). */
int oracle_bins(int d, const size_t *n, double tau_abs, double norm_inf, double eps, double *q);

/* Quantization of a level-major coefficient stream.
 * precision: 32 = decision in binary32, 64 = decision in binary64.
 * Writes symbols[N]; returns the number of outliers through *n_out and
 * their (stream index, integer code) pairs into out_idx/out_k when those
 * pointers are non-NULL (capacity out_cap). */
int oracle_quantize(int d, const size_t *n, const double *coef, const double *q, int precision,
                    uint32_t D, uint16_t *symbols, uint64_t *n_out,
                    uint64_t *out_idx, int64_t *out_k, uint64_t out_cap);
int oracle_dequantize(int d, const size_t *n, const uint16_t *symbols, const double *q, uint32_t D,
                      uint64_t n_out, const uint64_t *out_idx, const int64_t *out_k, double *coef);

/* Huffman stage (Alg. 2). */
int oracle_histogram(const uint16_t *symbols, uint64_t N, uint32_t D, uint64_t *hist);
int oracle_code_lengths(const uint64_t *hist, uint32_t D, uint8_t *len);
int oracle_canonical_codes(const uint8_t *len, uint32_t D, uint64_t *code);
/* Encode: writes the bitstream (uint32 words, MSB first) and the chunk table
 * (bit offset of every K-th symbol).  words must hold ceil(bits/32) words.
 * esc_k: NULL for plain symbols; otherwise symbol 0 is the escape of the
 * quantizer and esc_k holds, in stream order, the integer code of every
 * escape.  Each escape's codeword is followed by its payload: zigzag(k)
 * (k >= 0 -> 2k, k < 0 -> -2k - 1) in esc_width bits (0..63; 0 only for a
 * stream without escapes), which must hold the bit length of every escape's
 * zigzag(k) (|k| < 2^62). */
int oracle_encode(const uint16_t *symbols, uint64_t N, const uint8_t *len, const uint64_t *code,
                  uint32_t K, const int64_t *esc_k, int esc_width, uint32_t *words, uint64_t nwords_cap,
                  uint64_t *chunk_bits, uint64_t *total_bits);
/* Bit length of zigzag(k) of one escape, or -1 when k = 0 or |k| >= 2^62. */
int oracle_escape_bits(int64_t k);
/* Decode; with esc_width > 0 every escape's payload of esc_width bits is read
 * and its code stored into esc_k (stream order, capacity esc_cap), their
 * count in *n_esc. */
int oracle_decode(const uint32_t *words, uint64_t nwords, const uint64_t *chunk_bits, uint64_t N,
                  uint32_t K, const uint8_t *len, uint32_t D, uint16_t *symbols, int esc_width,
                  int64_t *esc_k, uint64_t esc_cap, uint64_t *n_esc);

/* Full container (format v3).  dtype: 0 = binary32 data, 1 = binary64 data
 * (u is always passed as FP64 values).  mode: 0 = L-infinity, 1 = L2 (RMS).
 * tol_kind: 0 = absolute, 1 = relative. */
int oracle_compress(int d, const size_t *n, const double *u, int dtype, double tol, int tol_kind,
                    int mode, uint32_t D, uint32_t K, uint8_t *out, uint64_t cap,
                    uint64_t *out_bytes);
/* oracle_compress with node coordinates (as oracle_decompose_c); the
 * container records them, and oracle_decompress uses them */
int oracle_compress_c(int d, const size_t *n, const double *coords, const double *u, int dtype, double tol,
                      int tol_kind, int mode, uint32_t D, uint32_t K, uint8_t *out, uint64_t cap,
                      uint64_t *out_bytes);
int oracle_decompress(const uint8_t *in, uint64_t in_bytes, double *u, uint64_t cap_elems);
int oracle_inspect(const uint8_t *in, uint64_t in_bytes, int *dtype, int *d, uint64_t *dims);
uint64_t oracle_compress_bound(int d, const size_t *n, uint32_t D, uint32_t K);
uint32_t oracle_crc32(const uint8_t *p, uint64_t n);

#ifdef __cplusplus
}
#endif
#endif
