/*
 * zfp.c -- FP64/integer oracle of fixed-rate ZFP compression (Alg. 3,
 * Sec. IV-C).  TEST INFRASTRUCTURE ONLY (see hpdr_oracle.h).
 *
 * The paper gives the outline: the field is cut into blocks of 4^d values,
 * each block's values are aligned to the block's largest exponent and made
 * fixed point, a near-orthogonal transform decorrelates them, and the bit
 * planes of the result are serialized, most significant first, truncated at
 * a fixed number of bits per block.  Everything below that outline is a
 * reading fixed here (and written independently in the CUDA path):
 *
 *   blocks      row-major over ceil(n_k / 4) blocks per dimension, values in
 *               a block row-major (last index fastest); a block that runs
 *               past the array edge repeats the last in-range value of each
 *               dimension (edge replication, decoded values there dropped).
 *   exponent    emax = max over the block of e, x = f 2^e with 1/2 <= |f| < 1
 *               (frexp); a block of zeros is flagged and codes nothing else.
 *   fixed point q = trunc(x 2^(P - 5 - emax)), P = 32 (f32) or 64 (f64), so
 *               |q| < 2^(P-5).
 *   transform   per dimension (last index first, then the others in reverse
 *               order), on every line (a0, a1, a2, a3) of the block, a
 *               two-level integer S-transform:
 *                 s0 = floor((a0 + a1) / 2), d0 = a0 - a1,
 *                 s1 = floor((a2 + a3) / 2), d1 = a2 - a3,
 *                 S  = floor((s0 + s1) / 2), D  = s0 - s1,
 *               giving (S, D, d0, d1).  It is exactly invertible (the parity
 *               of a sum equals that of the difference) and each dimension at
 *               most doubles a magnitude, so 3 dimensions stay below 2^(P-2),
 *               inside the range of P negabinary digits (about 2^P / 3 each
 *               way) and of a P-bit signed integer.
 *   order       coefficients sorted by the sum over dimensions of the class
 *               of their index (S: 0, D: 1, d0 and d1: 2), ties by block
 *               index: coarse (smooth) coefficients first.
 *   negabinary  u = (q + M) xor M, M = 0xAA..AA (P bits): base -2 digits, so
 *               dropped low planes err in either direction.
 *   coding      maxbits = rate * 4^d bits per block (rate 1..256; a plane
 *               costs at most 2 * 4^d + 1 bits, so every plane fits once
 *               rate * 4^d >= P (2 * 4^d + 1) + 1 + EB): 1 flag bit (nonzero
 *               block), EB exponent bits (emax + 2^(EB-1); EB = 9 for f32,
 *               12 for f64), then the planes k = P-1 .. 0.  In each plane the
 *               bits of the n coefficients already found significant are
 *               written as they are, then group tests: one bit "is any of
 *               coefficients n.. set in this plane"; after a 1, the bits of
 *               coefficients n, n+1, ... one at a time until a 1 (each makes
 *               n grow); after a 0 the plane ends.  Writing stops when the
 *               block's budget is spent; unused bits are zero.  The decoder
 *               makes the same decisions and leaves unread bits zero.
 *   stream      block b occupies bits [b maxbits, (b+1) maxbits) of an
 *               array of 32-bit words, bit j of the block in word j/32 at bit
 *               position j%32 (maxbits is a multiple of 32).
 *   container   64-byte header "HPDZ" | u32 version 1 | u32 dtype | u32 ndim
 *               | u64 dims[3] (16..40) | u32 rate (40) | u32 maxbits (44) |
 *               u64 blocks (48) | u32 0 (56) | u32 CRC-32 of bytes [0,60)
 *               (60); the block words follow at byte 64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include "hpdr_oracle.h"

#define ZHDR 64

static void zput32(uint8_t *p, uint32_t v) { for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i)); }
static void zput64(uint8_t *p, uint64_t v) { for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i)); }
static uint32_t zget32(const uint8_t *p) { uint32_t v = 0; for (int i = 0; i < 4; i++) v |= (uint32_t)p[i] << (8 * i); return v; }
static uint64_t zget64(const uint8_t *p) { uint64_t v = 0; for (int i = 0; i < 8; i++) v |= (uint64_t)p[i] << (8 * i); return v; }

/* floor(v / 2) for any sign, without relying on the shift of a negative */
static int64_t half_floor(int64_t v) { return (v >= 0) ? v / 2 : -((-v + 1) / 2); }

void oracle_zfp_fwd_line(int64_t *a, int stride)
{
    int64_t a0 = a[0], a1 = a[stride], a2 = a[2 * stride], a3 = a[3 * stride];
    int64_t s0 = half_floor(a0 + a1), d0 = a0 - a1;
    int64_t s1 = half_floor(a2 + a3), d1 = a2 - a3;
    int64_t S = half_floor(s0 + s1), D = s0 - s1;
    a[0] = S; a[stride] = D; a[2 * stride] = d0; a[3 * stride] = d1;
}

/* inverse of one level: from (s, d) back to (x, y) with s = floor((x+y)/2), d = x - y:
 * x + y = 2 s + (d mod 2), so x = s + (d + (d mod 2)) / 2 and y = x - d */
static void inv_pair(int64_t s, int64_t d, int64_t *x, int64_t *y)
{
    int64_t par = d & 1;   /* d mod 2 in {0, 1} for two's complement */
    *x = s + (d + par) / 2;
    *y = *x - d;
}

void oracle_zfp_inv_line(int64_t *a, int stride)
{
    int64_t S = a[0], D = a[stride], d0 = a[2 * stride], d1 = a[3 * stride];
    int64_t s0, s1, a0, a1, a2, a3;
    inv_pair(S, D, &s0, &s1);
    inv_pair(s0, d0, &a0, &a1);
    inv_pair(s1, d1, &a2, &a3);
    a[0] = a0; a[stride] = a1; a[2 * stride] = a2; a[3 * stride] = a3;
}

/* the transform of a whole block: dimension d-1 (stride 1) first */
static void fwd_block(int d, int64_t *blk)
{
    int B = 1 << (2 * d);
    for (int k = d - 1; k >= 0; k--) {
        int stride = 1 << (2 * (d - 1 - k));
        for (int i = 0; i < B; i++)
            if (((i / stride) % 4) == 0) oracle_zfp_fwd_line(blk + i, stride);
    }
}

static void inv_block(int d, int64_t *blk)
{
    int B = 1 << (2 * d);
    for (int k = 0; k < d; k++) {
        int stride = 1 << (2 * (d - 1 - k));
        for (int i = 0; i < B; i++)
            if (((i / stride) % 4) == 0) oracle_zfp_inv_line(blk + i, stride);
    }
}

/* sequency order: perm[r] = block index of the r-th coefficient */
void oracle_zfp_order(int d, int *perm)
{
    static const int cls[4] = {0, 1, 2, 2};
    int B = 1 << (2 * d);
    int key[64];
    for (int i = 0; i < B; i++) {
        int s = 0, r = i;
        for (int k = 0; k < d; k++) { s += cls[r % 4]; r /= 4; }
        key[i] = s;
        perm[i] = i;
    }
    /* insertion sort by (key, index): stable on the index order */
    for (int i = 1; i < B; i++) {
        int p = perm[i], j = i - 1;
        while (j >= 0 && key[perm[j]] > key[p]) { perm[j + 1] = perm[j]; j--; }
        perm[j + 1] = p;
    }
}

uint64_t oracle_negabinary(int64_t q, int P)
{
    uint64_t M = (P == 32) ? 0xAAAAAAAAull : 0xAAAAAAAAAAAAAAAAull;
    uint64_t mask = (P == 32) ? 0xFFFFFFFFull : ~0ull;
    return (((uint64_t)q + M) ^ M) & mask;
}

int64_t oracle_from_negabinary(uint64_t u, int P)
{
    uint64_t M = (P == 32) ? 0xAAAAAAAAull : 0xAAAAAAAAAAAAAAAAull;
    if (P == 32) {
        uint32_t v = (uint32_t)((u ^ M) - M);
        return (int64_t)(int32_t)v;
    }
    return (int64_t)((u ^ M) - M);
}

/* bit writer / reader over one block's budget */
typedef struct { uint32_t *w; uint64_t pos, end; } zbits;

static int put_bit(zbits *b, int v)
{
    if (b->pos >= b->end) return 0;
    if (v) b->w[b->pos >> 5] |= 1u << (b->pos & 31);
    b->pos++;
    return 1;
}

static int get_bit(zbits *b, int *v)
{
    if (b->pos >= b->end) return 0;
    *v = (int)((b->w[b->pos >> 5] >> (b->pos & 31)) & 1u);
    b->pos++;
    return 1;
}

/* embedded coding of B negabinary coefficients (sequency order) */
void oracle_zfp_encode_planes(const uint64_t *u, int B, int P, uint32_t *words, uint64_t start, uint64_t end)
{
    zbits b = {words, start, end};
    int n = 0;
    for (int k = P - 1; k >= 0; k--) {
        for (int i = 0; i < n; i++)
            if (!put_bit(&b, (int)((u[i] >> k) & 1u))) return;
        while (n < B) {
            int any = 0;
            for (int i = n; i < B; i++) if ((u[i] >> k) & 1u) { any = 1; break; }
            if (!put_bit(&b, any)) return;
            if (!any) break;
            for (;;) {
                int bit = (int)((u[n] >> k) & 1u);
                if (!put_bit(&b, bit)) return;
                n++;
                if (bit) break;
            }
        }
    }
}

void oracle_zfp_decode_planes(uint64_t *u, int B, int P, const uint32_t *words, uint64_t start, uint64_t end)
{
    zbits b = {(uint32_t *)words, start, end};
    for (int i = 0; i < B; i++) u[i] = 0;
    int n = 0;
    for (int k = P - 1; k >= 0; k--) {
        int v;
        for (int i = 0; i < n; i++) {
            if (!get_bit(&b, &v)) return;
            u[i] |= (uint64_t)v << k;
        }
        while (n < B) {
            int any;
            if (!get_bit(&b, &any)) return;
            if (!any) break;
            /* a stream that is not this encoder's may promise a set bit that
             * never comes: the scan stops at the block's end */
            while (n < B) {
                if (!get_bit(&b, &v)) return;
                u[n] |= (uint64_t)v << k;
                n++;
                if (v) break;
            }
        }
    }
}

static int zfp_params(int d, int dtype, uint32_t rate, int *P, int *EB, uint32_t *maxbits)
{
    if (d < 1 || d > 3 || (dtype != 0 && dtype != 1) || rate < 1 || rate > 256) return -1;
    *P = dtype == 0 ? 32 : 64;
    *EB = dtype == 0 ? 9 : 12;
    *maxbits = rate << (2 * d);
    if (*maxbits % 32 || *maxbits < (uint32_t)(*EB + 2)) return -1;
    return 0;
}

uint64_t oracle_zfp_bound(int d, const size_t *n, int dtype, uint32_t rate)
{
    int P, EB;
    uint32_t maxbits;
    if (zfp_params(d, dtype, rate, &P, &EB, &maxbits)) return 0;
    uint64_t nb = 1;
    for (int k = 0; k < d; k++) nb *= (n[k] + 3) / 4;
    return ZHDR + nb * (maxbits / 8);
}

/* gather block (b0, b1, b2) with edge replication; strides row-major */
static void gather(int d, const size_t *n, const double *u, const size_t *bi, double *out)
{
    int B = 1 << (2 * d);
    for (int i = 0; i < B; i++) {
        size_t off = 0;
        int r = i;
        size_t idx[3];
        for (int k = d - 1; k >= 0; k--) { idx[k] = (size_t)(r % 4); r /= 4; }
        for (int k = 0; k < d; k++) {
            size_t p = 4 * bi[k] + idx[k];
            if (p >= n[k]) p = n[k] - 1;
            off = off * n[k] + p;
        }
        out[i] = u[off];
    }
}

int oracle_zfp_compress(int d, const size_t *n, const double *u, int dtype, uint32_t rate, uint8_t *out,
                        uint64_t cap, uint64_t *out_bytes)
{
    int P, EB;
    uint32_t maxbits;
    if (zfp_params(d, dtype, rate, &P, &EB, &maxbits)) return -1;
    for (int k = 0; k < d; k++) if (n[k] < 1) return -1;
    uint64_t total = oracle_zfp_bound(d, n, dtype, rate);
    if (total > cap) return -3;
    size_t nbk[3] = {1, 1, 1};
    uint64_t nb = 1;
    for (int k = 0; k < d; k++) { nbk[k] = (n[k] + 3) / 4; nb *= nbk[k]; }
    memset(out, 0, total);
    memcpy(out, "HPDZ", 4);
    zput32(out + 4, 1);
    zput32(out + 8, (uint32_t)dtype);
    zput32(out + 12, (uint32_t)d);
    for (int k = 0; k < 3; k++) zput64(out + 16 + 8 * k, k < d ? (uint64_t)n[k] : 1);
    zput32(out + 40, rate);
    zput32(out + 44, maxbits);
    zput64(out + 48, nb);
    zput32(out + 60, oracle_crc32(out, 60));
    uint32_t *words = (uint32_t *)malloc(nb * (maxbits / 8));
    memset(words, 0, nb * (maxbits / 8));
    int B = 1 << (2 * d), perm[64];
    oracle_zfp_order(d, perm);
    double vals[64];
    int64_t q[64];
    uint64_t un[64];
    for (uint64_t b = 0; b < nb; b++) {
        size_t bi[3], r = (size_t)b;
        for (int k = d - 1; k >= 0; k--) { bi[k] = r % nbk[k]; r /= nbk[k]; }
        gather(d, n, u, bi, vals);
        if (dtype == 0) for (int i = 0; i < B; i++) vals[i] = (double)(float)vals[i];
        int emax = INT32_MIN, nz = 0;
        for (int i = 0; i < B; i++) {
            if (vals[i] != 0.0) {
                int e;
                frexp(vals[i], &e);
                if (e > emax) emax = e;
                nz = 1;
            }
        }
        uint64_t start = b * maxbits;
        zbits hb = {words, start, start + maxbits};
        if (!nz) { put_bit(&hb, 0); continue; }
        put_bit(&hb, 1);
        uint32_t eb = (uint32_t)(emax + (1 << (EB - 1)));
        for (int i = 0; i < EB; i++) put_bit(&hb, (int)((eb >> i) & 1u));
        for (int i = 0; i < B; i++) q[i] = (int64_t)ldexp(vals[i], P - 5 - emax);  /* exact, truncated */
        fwd_block(d, q);
        for (int r2 = 0; r2 < B; r2++) un[r2] = oracle_negabinary(q[perm[r2]], P);
        oracle_zfp_encode_planes(un, B, P, words, hb.pos, start + maxbits);
    }
    memcpy(out + ZHDR, words, nb * (maxbits / 8));
    free(words);
    *out_bytes = total;
    return 0;
}

int oracle_zfp_decompress(const uint8_t *in, uint64_t in_bytes, double *u, uint64_t n_cap)
{
    if (in_bytes < ZHDR || memcmp(in, "HPDZ", 4) || zget32(in + 4) != 1) return -4;
    if (oracle_crc32(in, 60) != zget32(in + 60)) return -4;
    int dtype = (int)zget32(in + 8), d = (int)zget32(in + 12);
    uint32_t rate = zget32(in + 40), maxbits = zget32(in + 44);
    int P, EB;
    uint32_t mb;
    if (zfp_params(d, dtype, rate, &P, &EB, &mb) || mb != maxbits) return -4;
    size_t n[3], nbk[3] = {1, 1, 1};
    uint64_t N = 1, nb = 1;
    for (int k = 0; k < d; k++) {
        n[k] = (size_t)zget64(in + 16 + 8 * k);
        if (n[k] < 1) return -4;
        nbk[k] = (n[k] + 3) / 4;
        N *= n[k];
        nb *= nbk[k];
    }
    if (zget64(in + 48) != nb || ZHDR + nb * (maxbits / 8) > in_bytes) return -4;
    if (N > n_cap) return -3;
    const uint32_t *words = (const uint32_t *)malloc(nb * (maxbits / 8));
    memcpy((void *)words, in + ZHDR, nb * (maxbits / 8));
    int B = 1 << (2 * d), perm[64];
    oracle_zfp_order(d, perm);
    int64_t q[64];
    uint64_t un[64];
    for (uint64_t b = 0; b < nb; b++) {
        size_t bi[3], r = (size_t)b;
        for (int k = d - 1; k >= 0; k--) { bi[k] = r % nbk[k]; r /= nbk[k]; }
        uint64_t start = b * maxbits;
        zbits hb = {(uint32_t *)words, start, start + maxbits};
        int flag = 0, v = 0;
        get_bit(&hb, &flag);
        double vals[64];
        if (!flag) {
            for (int i = 0; i < B; i++) vals[i] = 0.0;
        } else {
            uint32_t eb = 0;
            for (int i = 0; i < EB; i++) { get_bit(&hb, &v); eb |= (uint32_t)v << i; }
            int emax = (int)eb - (1 << (EB - 1));
            oracle_zfp_decode_planes(un, B, P, words, hb.pos, start + maxbits);
            for (int r2 = 0; r2 < B; r2++) q[perm[r2]] = oracle_from_negabinary(un[r2], P);
            inv_block(d, q);
            for (int i = 0; i < B; i++) vals[i] = ldexp((double)q[i], emax - (P - 5));
        }
        /* scatter the in-range values */
        for (int i = 0; i < B; i++) {
            int rr = i;
            size_t idx[3], off = 0;
            int inside = 1;
            for (int k = d - 1; k >= 0; k--) { idx[k] = (size_t)(rr % 4); rr /= 4; }
            for (int k = 0; k < d; k++) {
                size_t p = 4 * bi[k] + idx[k];
                if (p >= n[k]) { inside = 0; break; }
                off = off * n[k] + p;
            }
            if (inside) u[off] = (dtype == 0) ? (double)(float)vals[i] : vals[i];
        }
    }
    free((void *)words);
    return 0;
}
