/*
 * container.c -- oracle of the whole reduction path (Alg. 1 followed by
 * Alg. 2) and of its inverse, written into / read from the self-describing
 * container, format version 3.  TEST INFRASTRUCTURE ONLY (see
 * hpdr_oracle.h).
 *
 * Container v3 (little endian; every section starts on a 16-byte boundary;
 * padding bytes are zero):
 *   0   "HPDR"            4  u32 version (3)     8  u32 dtype (0 f32, 1 f64)
 *   12  u32 ndim          16 u64 dims[3] (unused dims hold 1)
 *   40  u32 L             44 u32 mode (0 Linf, 1 L2, 2 statistical L2)
 *   48  u32 tol kind (0 abs, 1 rel) | 0x100 when the container holds node coordinates
 *   52  u32 D             56 u32 K               60 u32 s_lo
 *   64  f64 tol           72 f64 tau_abs         80 f64 max|u|    88 f64 rms(u)
 *   96  u64 N             104 u64 escapes        112 u64 bitstream bits
 *   120 u16 s_hi          122 u8 escape width W   123 u8 0
 *   124 u32 CRC-32 of bytes [0,124)
 *   128 f64 q[L+1]
 *   with the coordinate flag: f64 node coordinates, dims[0] + ... + dims[ndim-1]
 *                 values, dimension 0 first (directly after q, 8-byte aligned)
 *   code lengths  u8[s_hi - s_lo + 1]  (symbols s_lo..s_hi)
 *   chunk table   u64[ceil(N/K)]       (bit offset of symbol j*K)
 *   bitstream     u32[ceil(bits/32)]
 *
 * Symbol s = k + D/2 carries the quantized code k when 1 <= s <= D-1; every
 * other code is escaped: symbol 0, whose codeword is followed in the
 * bitstream by zigzag(k) in W bits, W the largest bit length of the
 * container's escapes (0 without escapes; see oracle_encode).
 *
 * Tolerance: REL means tol times max|u| (Linf mode) or times rms(u) (both L2
 * modes); ABS means tol itself.  L2 mode uses the same bins, which bound the
 * maximum error and therefore the RMS error too; statistical L2 mode uses the
 * bins of oracle_bins_l2s_c, which bound the expected RMS error.
 */
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include "hpdr_oracle.h"

#define HDR 128

static uint64_t align16(uint64_t x) { return (x + 15) & ~(uint64_t)15; }

uint32_t oracle_crc32(const uint8_t *p, uint64_t n)
{
    uint32_t c = 0xFFFFFFFFu;
    for (uint64_t i = 0; i < n; i++) {
        c ^= p[i];
        for (int b = 0; b < 8; b++) c = (c >> 1) ^ (0xEDB88320u & (0u - (c & 1u)));
    }
    return c ^ 0xFFFFFFFFu;
}

static void put32(uint8_t *p, uint32_t v) { for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i)); }
static void put64(uint8_t *p, uint64_t v) { for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i)); }
static void putf64(uint8_t *p, double v) { uint64_t u; memcpy(&u, &v, 8); put64(p, u); }
static uint32_t get32(const uint8_t *p) { uint32_t v = 0; for (int i = 0; i < 4; i++) v |= (uint32_t)p[i] << (8 * i); return v; }
static uint64_t get64(const uint8_t *p) { uint64_t v = 0; for (int i = 0; i < 8; i++) v |= (uint64_t)p[i] << (8 * i); return v; }
static double getf64(const uint8_t *p) { uint64_t u = get64(p); double v; memcpy(&v, &u, 8); return v; }

uint64_t oracle_compress_bound(int d, const size_t *n, uint32_t D, uint32_t K)
{
    int L;
    if (oracle_levels(d, n, &L, NULL) || K == 0) return 0;
    uint64_t N = 1, nco = 0;
    for (int k = 0; k < d; k++) { N *= n[k]; nco += n[k]; }
    /* room for the node coordinates, present or not */
    uint64_t b = align16(HDR + 8 * (uint64_t)(L + 1) + 8 * nco);
    b = align16(b + D);
    b = align16(b + 8 * ((N + K - 1) / K));
    /* Huffman bits <= N ceil(log2 D) (a fixed-length code is a prefix code);
     * escape payloads <= 32 bits each while |k| < 2^31 */
    uint64_t lg = 0;
    while ((1ULL << lg) < D) lg++;
    b += 4 * ((N * (lg + 32) + 31) / 32);
    return b;
}

int oracle_compress(int d, const size_t *n, const double *u, int dtype, double tol, int tol_kind,
                    int mode, uint32_t D, uint32_t K, uint8_t *out, uint64_t cap,
                    uint64_t *out_bytes)
{
    return oracle_compress_c(d, n, NULL, u, dtype, tol, tol_kind, mode, D, K, out, cap, out_bytes);
}

int oracle_compress_c(int d, const size_t *n, const double *coords, const double *u, int dtype, double tol,
                      int tol_kind, int mode, uint32_t D, uint32_t K, uint8_t *out, uint64_t cap,
                      uint64_t *out_bytes)
{
    int L;
    if (oracle_levels(d, n, &L, NULL)) return -1;
    if ((dtype != 0 && dtype != 1) || mode < 0 || mode > 2 || (tol_kind != 0 && tol_kind != 1))
        return -1;
    if (D < 4 || D > 65536 || (D % 2) || K == 0 || !(tol > 0)) return -1;
    uint64_t N = 1;
    for (int k = 0; k < d; k++) N *= n[k];

    double mx = 0.0, ss = 0.0;
    for (uint64_t i = 0; i < N; i++) { double a = fabs(u[i]); if (a > mx) mx = a; ss += u[i] * u[i]; }
    double rms = sqrt(ss / (double)N);
    double nrm = (mode == 0) ? mx : rms;
    double tau_abs = (tol_kind == 1) ? tol * nrm : tol;
    double eps = (dtype == 0) ? ldexp(1.0, -24) : ldexp(1.0, -53);
    double *q = (double *)malloc((size_t)(L + 1) * sizeof(double));
    int rc = (mode == 2) ? oracle_bins_l2s_c(d, n, coords, tau_abs, mx, eps, q)
                         : oracle_bins_c(d, n, coords, tau_abs, mx, eps, q);
    if (rc) { free(q); return (rc == -2) ? -1 : rc; }

    double *coef = (double *)malloc(N * sizeof(double));
    uint16_t *sym = (uint16_t *)malloc(N * sizeof(uint16_t));
    uint64_t nout = 0;
    if (oracle_decompose_c(d, n, coords, u, coef)) { free(q); free(coef); free(sym); return -1; }
    oracle_quantize(d, n, coef, q, 64, D, sym, &nout, NULL, NULL, 0);
    uint64_t *oidx = (uint64_t *)malloc((nout + 1) * sizeof(uint64_t));
    int64_t *ok = (int64_t *)malloc((nout + 1) * sizeof(int64_t));
    oracle_quantize(d, n, coef, q, 64, D, sym, &nout, oidx, ok, nout);

    uint64_t *hist = (uint64_t *)malloc((size_t)D * sizeof(uint64_t));
    uint8_t *len = (uint8_t *)malloc(D);
    uint64_t *code = (uint64_t *)malloc((size_t)D * sizeof(uint64_t));
    oracle_histogram(sym, N, D, hist);
    rc = oracle_code_lengths(hist, D, len);
    if (rc == 0) oracle_canonical_codes(len, D, code);
    uint32_t slo = 0, shi = 0;
    for (uint32_t s = 0; s < D; s++) if (len[s]) { slo = s; break; }
    for (uint32_t s = D; s-- > 0;) if (len[s]) { shi = s; break; }

    uint64_t nch = (N + K - 1) / K;
    uint64_t nco = 0;
    if (coords) for (int k = 0; k < d; k++) nco += n[k];
    uint64_t off_q = HDR;
    uint64_t off_co = off_q + 8 * (uint64_t)(L + 1);
    uint64_t off_len = align16(off_co + 8 * nco);
    uint64_t off_chunk = align16(off_len + (shi - slo + 1));
    uint64_t off_bits = align16(off_chunk + 8 * nch);
    uint64_t bits = 0;
    for (uint64_t i = 0; i < N && rc == 0; i++) bits += len[sym[i]];
    int ew = 0;
    for (uint64_t j = 0; j < nout && rc == 0; j++) {
        int eb = oracle_escape_bits(ok[j]);
        if (eb < 0) rc = -1;
        else if (eb > ew) ew = eb;
    }
    bits += nout * (uint64_t)ew;
    uint64_t nwords = (bits + 31) / 32;
    uint64_t total = off_bits + 4 * nwords;
    if (rc == 0 && total > cap) rc = -3;
    if (rc == 0) {
        memset(out, 0, total);
        uint64_t *chunk = (uint64_t *)malloc(nch * sizeof(uint64_t));
        uint32_t *words = (uint32_t *)malloc((nwords + 1) * sizeof(uint32_t));
        uint64_t tb = 0;
        rc = oracle_encode(sym, N, len, code, K, nout ? ok : NULL, ew, words, nwords + 1, chunk, &tb);
        if (rc == 0 && tb != bits) rc = -1;
        memcpy(out, "HPDR", 4);
        put32(out + 4, 3);
        put32(out + 8, (uint32_t)dtype);
        put32(out + 12, (uint32_t)d);
        for (int k = 0; k < 3; k++) put64(out + 16 + 8 * k, (k < d) ? (uint64_t)n[k] : 1);
        put32(out + 40, (uint32_t)L);
        put32(out + 44, (uint32_t)mode);
        put32(out + 48, (uint32_t)tol_kind | (coords ? 0x100u : 0u));
        put32(out + 52, D);
        put32(out + 56, K);
        put32(out + 60, slo);
        putf64(out + 64, tol);
        putf64(out + 72, tau_abs);
        putf64(out + 80, mx);
        putf64(out + 88, rms);
        put64(out + 96, N);
        put64(out + 104, nout);
        put64(out + 112, bits);
        put32(out + 120, shi | ((uint32_t)ew << 16));
        put32(out + 124, oracle_crc32(out, 124));
        for (int l = 0; l <= L; l++) putf64(out + off_q + 8 * l, q[l]);
        for (uint64_t i = 0; i < nco; i++) putf64(out + off_co + 8 * i, coords[i]);
        for (uint32_t s = slo; s <= shi; s++) out[off_len + (s - slo)] = len[s];
        for (uint64_t j = 0; j < nch; j++) put64(out + off_chunk + 8 * j, chunk[j]);
        for (uint64_t w = 0; w < nwords; w++) put32(out + off_bits + 4 * w, words[w]);
        *out_bytes = total;
        free(chunk); free(words);
    }
    free(q); free(coef); free(sym); free(oidx); free(ok); free(hist); free(len); free(code);
    return rc;
}

typedef struct {
    int dtype, d, L, mode, tol_kind;
    size_t n[3];
    uint32_t D, K, slo, shi, ew;
    uint64_t N, nout, bits, nch, nwords, nco;
    uint64_t off_q, off_co, off_len, off_chunk, off_bits, total;
} hdr_t;

static int parse(const uint8_t *in, uint64_t in_bytes, hdr_t *h)
{
    if (in_bytes < HDR || memcmp(in, "HPDR", 4) != 0 || get32(in + 4) != 3) return -4;
    if (oracle_crc32(in, 124) != get32(in + 124)) return -4;
    h->dtype = (int)get32(in + 8);
    h->d = (int)get32(in + 12);
    if (h->d < 1 || h->d > 3 || h->dtype > 1) return -4;
    for (int k = 0; k < 3; k++) h->n[k] = (size_t)get64(in + 16 + 8 * k);
    h->L = (int)get32(in + 40);
    h->mode = (int)get32(in + 44);
    const uint32_t tk = get32(in + 48);
    if (tk & ~0x101u) return -4;
    h->tol_kind = (int)(tk & 1u);
    h->D = get32(in + 52);
    h->K = get32(in + 56);
    h->slo = get32(in + 60);
    h->N = get64(in + 96);
    h->nout = get64(in + 104);
    h->bits = get64(in + 112);
    h->shi = get32(in + 120) & 0xFFFFu;
    h->ew = (get32(in + 120) >> 16) & 0xFFu;
    if (get32(in + 120) >> 24) return -4;
    int L;
    if (oracle_levels(h->d, h->n, &L, NULL) || L != h->L) return -4;
    uint64_t N = 1;
    for (int k = 0; k < h->d; k++) N *= h->n[k];
    if (N != h->N || h->K == 0 || h->D < 4 || h->D > 65536 || h->shi >= h->D || h->slo > h->shi)
        return -4;
    if (h->nout > N || h->ew > 63 || (h->nout && h->ew == 0)) return -4;
    h->nch = (N + h->K - 1) / h->K;
    h->nwords = (h->bits + 31) / 32;
    h->nco = 0;
    if (tk & 0x100u) for (int k = 0; k < h->d; k++) h->nco += h->n[k];
    h->off_q = HDR;
    h->off_co = h->off_q + 8 * (uint64_t)(L + 1);
    h->off_len = align16(h->off_co + 8 * h->nco);
    h->off_chunk = align16(h->off_len + (h->shi - h->slo + 1));
    h->off_bits = align16(h->off_chunk + 8 * h->nch);
    h->total = h->off_bits + 4 * h->nwords;
    if (h->total > in_bytes) return -4;
    return 0;
}

int oracle_inspect(const uint8_t *in, uint64_t in_bytes, int *dtype, int *d, uint64_t *dims)
{
    hdr_t h;
    int rc = parse(in, in_bytes, &h);
    if (rc) return rc;
    *dtype = h.dtype;
    *d = h.d;
    for (int k = 0; k < 3; k++) dims[k] = h.n[k];
    return 0;
}

int oracle_decompress(const uint8_t *in, uint64_t in_bytes, double *u, uint64_t cap_elems)
{
    hdr_t h;
    int rc = parse(in, in_bytes, &h);
    if (rc) return rc;
    if (h.N > cap_elems) return -3;
    double *q = (double *)malloc((size_t)(h.L + 1) * sizeof(double));
    for (int l = 0; l <= h.L; l++) q[l] = getf64(in + h.off_q + 8 * l);
    uint8_t *len = (uint8_t *)calloc(h.D, 1);
    for (uint32_t s = h.slo; s <= h.shi; s++) len[s] = in[h.off_len + (s - h.slo)];
    uint64_t *chunk = (uint64_t *)malloc(h.nch * sizeof(uint64_t));
    for (uint64_t j = 0; j < h.nch; j++) chunk[j] = get64(in + h.off_chunk + 8 * j);
    uint64_t *oidx = (uint64_t *)malloc((h.nout + 1) * sizeof(uint64_t));
    int64_t *ok = (int64_t *)malloc((h.nout + 1) * sizeof(int64_t));
    uint32_t *words = (uint32_t *)malloc((h.nwords + 1) * sizeof(uint32_t));
    for (uint64_t w = 0; w < h.nwords; w++) words[w] = get32(in + h.off_bits + 4 * w);
    uint16_t *sym = (uint16_t *)malloc(h.N * sizeof(uint16_t));
    double *coef = (double *)malloc(h.N * sizeof(double));
    uint64_t ne = 0;
    rc = oracle_decode(words, h.nwords, chunk, h.N, h.K, len, h.D, sym, (int)h.ew, ok, h.nout, &ne);
    if (rc == 0 && ne != h.nout) rc = -4;
    for (uint64_t i = 0, j = 0; rc == 0 && i < h.N; i++)
        if (sym[i] == 0) oidx[j++] = i;
    if (rc == 0) rc = oracle_dequantize(h.d, h.n, sym, q, h.D, h.nout, oidx, ok, coef);
    double *co = NULL;
    if (rc == 0 && h.nco) {
        co = (double *)malloc(h.nco * sizeof(double));
        for (uint64_t i = 0; i < h.nco; i++) co[i] = getf64(in + h.off_co + 8 * i);
    }
    if (rc == 0) rc = oracle_recompose_c(h.d, h.n, co, coef, u) ? -4 : 0;
    free(co);
    free(q); free(len); free(chunk); free(oidx); free(ok); free(words); free(sym); free(coef);
    return rc;
}
