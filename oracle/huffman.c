/*
 * huffman.c -- FP-free oracle of the Huffman stage of Sec. IV-B (Alg. 2):
 * histogram, sort by frequency, drop zero frequencies, code lengths,
 * canonical codewords, encoding and serialization into one bitstream, and
 * the inverse decoding.  TEST INFRASTRUCTURE ONLY (see hpdr_oracle.h).
 *
 * Readings fixed here (the paper defers the codebook details to its
 * references):
 *   - leaves are the symbols with non-zero frequency, sorted ascending by
 *     (frequency, symbol); a single present symbol gets length 1;
 *   - lengths come from the two-queue Huffman merge: queue A holds the sorted
 *     leaves, queue B the merged nodes in creation order; every pick takes
 *     A's front when its weight is <= B's front weight, else B's front;
 *   - codewords are canonical: symbols ordered by (length, symbol), the first
 *     gets 0, each next one the previous plus one, shifted left by the
 *     growth in length;
 *   - codewords are written most significant bit first into 32-bit words,
 *     filling bit 31 of a word first; the chunk table holds the bit offset of
 *     symbol j*K for every chunk j.
 */
#include <stdlib.h>
#include <string.h>
#include "hpdr_oracle.h"

#define OMAXLEN 63

int oracle_histogram(const uint16_t *symbols, uint64_t N, uint32_t D, uint64_t *hist)
{
    memset(hist, 0, (size_t)D * sizeof(uint64_t));
    for (uint64_t i = 0; i < N; i++) {
        if (symbols[i] >= D) return -1;
        hist[symbols[i]]++;
    }
    return 0;
}

typedef struct { uint64_t f; uint32_t s; } leaf_t;

static int leaf_cmp(const void *a, const void *b)
{
    const leaf_t *x = (const leaf_t *)a, *y = (const leaf_t *)b;
    if (x->f != y->f) return (x->f < y->f) ? -1 : 1;
    return (x->s < y->s) ? -1 : (x->s > y->s);
}

int oracle_code_lengths(const uint64_t *hist, uint32_t D, uint8_t *len)
{
    memset(len, 0, D);
    uint32_t n = 0;
    for (uint32_t s = 0; s < D; s++) if (hist[s]) n++;
    if (n == 0) return 0;
    leaf_t *lv = (leaf_t *)malloc(n * sizeof(leaf_t));
    n = 0;
    for (uint32_t s = 0; s < D; s++) if (hist[s]) { lv[n].f = hist[s]; lv[n].s = s; n++; }
    qsort(lv, n, sizeof(leaf_t), leaf_cmp);                   /* SortByKey + filter */
    if (n == 1) { len[lv[0].s] = 1; free(lv); return 0; }
    uint32_t tot = 2 * n - 1;
    uint64_t *wt = (uint64_t *)malloc(tot * sizeof(uint64_t));
    uint32_t *parent = (uint32_t *)malloc(tot * sizeof(uint32_t));
    uint32_t *depth = (uint32_t *)malloc(tot * sizeof(uint32_t));
    for (uint32_t i = 0; i < n; i++) wt[i] = lv[i].f;
    uint32_t ia = 0, ib = n, next = n;                        /* queue fronts */
    while (next < tot) {
        uint32_t pick[2];
        for (int t = 0; t < 2; t++) {
            if (ia < n && (ib >= next || wt[ia] <= wt[ib])) pick[t] = ia++;
            else pick[t] = ib++;
        }
        wt[next] = wt[pick[0]] + wt[pick[1]];
        parent[pick[0]] = parent[pick[1]] = next;
        next++;
    }
    depth[tot - 1] = 0;                                       /* root */
    for (uint32_t i = tot - 1; i-- > 0;) depth[i] = depth[parent[i]] + 1;
    int rc = 0;
    for (uint32_t i = 0; i < n; i++) {
        if (depth[i] > OMAXLEN) rc = -3;
        len[lv[i].s] = (uint8_t)depth[i];
    }
    free(lv); free(wt); free(parent); free(depth);
    return rc;
}

int oracle_canonical_codes(const uint8_t *len, uint32_t D, uint64_t *code)
{
    memset(code, 0, (size_t)D * sizeof(uint64_t));
    uint64_t c = 0;
    int prev = -1;
    for (int L = 1; L <= OMAXLEN; L++) {
        for (uint32_t s = 0; s < D; s++) {
            if (len[s] != L) continue;
            if (prev < 0) prev = L;
            else if (L > prev) { c <<= (L - prev); prev = L; }
            code[s] = c++;
        }
    }
    return 0;
}

/* zigzag map of an escaped code: k >= 0 -> 2k, k < 0 -> -2k - 1 */
static uint64_t zigzag(int64_t k) { return k >= 0 ? 2 * (uint64_t)k : 2 * (uint64_t)(-(k + 1)) + 1; }
static int64_t unzigzag(uint64_t z) { return (z & 1) ? -(int64_t)(z >> 1) - 1 : (int64_t)(z >> 1); }
static int bitlen(uint64_t z) { int n = 0; while (z) { n++; z >>= 1; } return n; }

int oracle_escape_bits(int64_t k)
{
    if (k == 0 || k >= ((int64_t)1 << 62) || k <= -((int64_t)1 << 62)) return -1;
    return bitlen(zigzag(k));
}

static void put_bits(uint32_t *words, uint64_t *pos, uint64_t v, int nbits)
{
    for (int b = nbits - 1; b >= 0; b--) {
        if ((v >> b) & 1u) words[*pos / 32] |= 1u << (31 - (*pos % 32));
        (*pos)++;
    }
}

int oracle_encode(const uint16_t *symbols, uint64_t N, const uint8_t *len, const uint64_t *code,
                  uint32_t K, const int64_t *esc_k, int esc_width, uint32_t *words, uint64_t nwords_cap,
                  uint64_t *chunk_bits, uint64_t *total_bits)
{
    if (K == 0 || esc_width < 0 || esc_width > 63) return -1;
    uint64_t bits = 0, e = 0;
    for (uint64_t i = 0; i < N; i++) {
        if (len[symbols[i]] == 0) return -1;
        bits += len[symbols[i]];
        if (esc_k && symbols[i] == 0) {
            int eb = oracle_escape_bits(esc_k[e++]);
            if (eb < 0 || eb > esc_width) return -1;
            bits += (uint64_t)esc_width;
        }
    }
    uint64_t nwords = (bits + 31) / 32;
    *total_bits = bits;
    if (nwords > nwords_cap) return -3;
    memset(words, 0, nwords * sizeof(uint32_t));
    uint64_t pos = 0;
    e = 0;
    for (uint64_t i = 0; i < N; i++) {
        if (i % K == 0) chunk_bits[i / K] = pos;
        put_bits(words, &pos, code[symbols[i]], len[symbols[i]]);
        if (esc_k && symbols[i] == 0) put_bits(words, &pos, zigzag(esc_k[e++]), esc_width);
    }
    return 0;
}

static int get_bits(const uint32_t *words, uint64_t nwords, uint64_t *pos, int nbits, uint64_t *v)
{
    *v = 0;
    for (int b = 0; b < nbits; b++) {
        if (*pos / 32 >= nwords) return -4;
        *v = (*v << 1) | ((words[*pos / 32] >> (31 - (*pos % 32))) & 1u);
        (*pos)++;
    }
    return 0;
}

int oracle_decode(const uint32_t *words, uint64_t nwords, const uint64_t *chunk_bits, uint64_t N,
                  uint32_t K, const uint8_t *len, uint32_t D, uint16_t *symbols, int esc_width,
                  int64_t *esc_k, uint64_t esc_cap, uint64_t *n_esc)
{
    if (esc_width < 0 || esc_width > 63) return -4;
    uint64_t ne = 0;
    uint64_t count[OMAXLEN + 2] = {0}, first[OMAXLEN + 2] = {0}, findex[OMAXLEN + 2] = {0};
    uint32_t *sorted = (uint32_t *)malloc((size_t)D * sizeof(uint32_t));
    uint32_t ns = 0;
    for (int L = 1; L <= OMAXLEN; L++)
        for (uint32_t s = 0; s < D; s++)
            if (len[s] == L) { if (!count[L]) findex[L] = ns; count[L]++; sorted[ns++] = s; }
    if (ns == 0) { free(sorted); return -4; }
    /* first canonical code of every length */
    uint64_t c = 0;
    int prev = -1;
    for (int L = 1; L <= OMAXLEN; L++) {
        if (!count[L]) continue;
        if (prev < 0) { c = 0; }
        else { c <<= (L - prev); }
        first[L] = c;
        c += count[L];
        prev = L;
    }
    uint64_t nchunks = (N + K - 1) / K;
    for (uint64_t j = 0; j < nchunks; j++) {
        uint64_t pos = chunk_bits[j];
        uint64_t end = (j + 1) * (uint64_t)K;
        if (end > N) end = N;
        for (uint64_t i = j * (uint64_t)K; i < end; i++) {
            uint64_t v = 0;
            int L = 0, found = 0;
            while (!found) {
                if (pos / 32 >= nwords) { free(sorted); return -4; }
                uint32_t bit = (words[pos / 32] >> (31 - (pos % 32))) & 1u;
                pos++;
                v = (v << 1) | bit;
                L++;
                if (L > OMAXLEN) { free(sorted); return -4; }
                if (count[L] && v >= first[L] && v - first[L] < count[L]) {
                    symbols[i] = (uint16_t)sorted[findex[L] + (v - first[L])];
                    found = 1;
                }
            }
            if (esc_width && symbols[i] == 0) {
                uint64_t z;
                if (get_bits(words, nwords, &pos, esc_width, &z) || ne >= esc_cap) {
                    free(sorted);
                    return -4;
                }
                esc_k[ne++] = unzigzag(z);
            }
        }
    }
    if (n_esc) *n_esc = ne;
    free(sorted);
    return 0;
}
