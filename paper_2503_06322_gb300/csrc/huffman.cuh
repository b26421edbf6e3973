// huffman.cuh -- launchers of the Huffman stage (huffman.cu), Sec. IV-B / Alg. 2.
#pragma once
#include "internal.cuh"

namespace hpdr {

constexpr int kLutBits = 13;    // decoder: first-level table of every 13-bit prefix
constexpr int kSubMax = 10;     // decoder: second-level index bits (codewords of up to 23 bits)
constexpr unsigned kSubCap = 12288;   // decoder: second-level entries (48 KB of shared memory)
constexpr int kMaxCodeLen = 63;

// Escape payload (container format v3): after the codeword of symbol 0,
// zigzag(k) in W bits, W = the container's payload width (the largest bit
// length of zigzag(k) over its escapes, 1..63).
__host__ __device__ inline unsigned long long zigzag(long long k)
{
    return k >= 0 ? 2ULL * (unsigned long long)k : 2ULL * (unsigned long long)(-(k + 1)) + 1ULL;
}
__host__ __device__ inline long long unzigzag(unsigned long long z)
{
    return (z & 1ULL) ? -(long long)(z >> 1) - 1 : (long long)(z >> 1);
}

// Device scratch of one codebook build (sizes for an alphabet of D symbols).
struct HuffScratch {
    unsigned long long *keys;     // [D]
    unsigned long long *keys2;    // [D]
    unsigned long long *sorted;   // [D]
    unsigned int *rank;           // [D]
    unsigned int *parent;         // [2D]
    unsigned int *anc;            // [2*2D] ping-pong
    unsigned int *dep;            // [2*2D] ping-pong
    unsigned long long *leafw;    // [D]   (used when the alphabet is too large for shared memory)
    unsigned long long *intw;     // [D]
    unsigned int *nsym;           // [1]
    unsigned long long *first;    // [64]
    unsigned int *count;          // [64]
    unsigned int *start;          // [64]
    uint8_t *len;                 // [D]
    unsigned long long *code;     // [D]
    uint16_t *sorted_sym;         // [D]
    uint32_t *lut1;               // [1 << kLutBits] first-level decoder table of every 13-bit prefix
    uint32_t *lut_sub;            // [kSubCap] second-level entries of longer codewords
    unsigned int *nsub;           // [1] second-level entries in use
    unsigned long long *lim;      // [64] left-justified upper limit of the codes of each length
    unsigned int *status;         // -> Scalars::status
    unsigned int *s_lo, *s_hi;    // -> Scalars
};
// The header fields that locate a container's sections, parsed on the device
// (a decompression that does not read the header back to the host).
struct DevHdr {
    unsigned long long off_len, off_chunk, off_bits;   // byte offsets of the sections
    unsigned long long nwords, total_bits, n_esc;
    unsigned int s_lo, s_hi, esc_w, pad;
};

size_t huff_scratch_bytes(unsigned int D);
void huff_scratch_carve(void *base, unsigned int D, Scalars *sc, HuffScratch *hs);

// Codebook from a histogram hist[D] (two-queue lengths, canonical codes).
cudaError_t launch_codebook(const unsigned long long *hist, unsigned int D, const HuffScratch &hs,
                            cudaStream_t s);
// Canonical tables + LUT from the code lengths lenb[0 .. s_hi - s_lo] of the
// symbols s_lo..s_hi (device bytes; every other symbol absent), decoder side.
cudaError_t launch_decode_tables(const uint8_t *lenb, unsigned int s_lo, unsigned int s_hi, unsigned int D,
                                 const HuffScratch &hs, cudaStream_t s);
// the same with the length table located through a device-parsed header
cudaError_t launch_decode_tables_dev(const uint8_t *base, const DevHdr *dh, unsigned int D, const HuffScratch &hs,
                                     cudaStream_t s);

// Encoder.  Layout of the destination: chunk table at chunk_out, bitstream at
// words (both device pointers, possibly inside a container whose offsets are
// only known on the device: then pass the base and the Scalars-derived
// offsets through ContainerLayout).
struct EncodeArgs {
    const uint16_t *sym;
    unsigned long long N;
    unsigned int D, K;
    const uint8_t *len;
    const unsigned long long *code;
    const long long *esc;             // null: plain symbols; else symbol 0 is the quantizer's
                                      // escape and esc[i] its code k (payload after the codeword,
                                      // in sc->esc_w bits)
    unsigned long long *chunk_bits;   // ws [nch+1] totals then offsets
    unsigned long long *bsum;         // ws [kEncBlocks] per-block sums, then offsets
    Scalars *sc;
    // destination
    uint8_t *container;               // if non-null: chunk table and bits go into the container
    int L;                            // levels (container layout)
    unsigned long long ncoord;        // node coordinates the container carries (0: none)
    unsigned long long capacity;      // bytes available at container / words
    unsigned long long *chunk_out;    // (container == null) chunk table destination
    uint32_t *words_out;              // (container == null) bitstream destination
    unsigned long long words_cap;
};
cudaError_t launch_encode(const EncodeArgs &a, cudaStream_t s);

struct HeaderArgs {
    int dtype, ndim, L, mode, tol_kind;
    unsigned long long dims[3];
    unsigned int D, K;
    double tol;
    unsigned long long N;
    const unsigned long long *hist;   // histogram: hist[0] = escapes recorded in the header
    const double *coords;             // node coordinates (device), ncoord values, or null
    unsigned long long ncoord;
};
cudaError_t launch_header(const HeaderArgs &h, const uint8_t *len, Scalars *sc, uint8_t *container,
                          cudaStream_t s);

// Batched forms for many fields at once (one block per field, the same
// device code as the single-field launches, so the same bytes).
struct CodebookJob {
    const unsigned long long *hist;
    unsigned int D;
    HuffScratch hs;
};
struct HeaderJob {
    HeaderArgs h;
    const uint8_t *len;
    Scalars *sc;
    uint8_t *out;
    unsigned long long *size_status;   // [2]: container bytes and device status (may be null)
};
// whether launch_codebook builds an alphabet of D symbols in one block
// (launch_codebook_batch takes only such alphabets)
bool codebook_fused(unsigned int D);
cudaError_t launch_codebook_batch(const CodebookJob *jobs, int n, cudaStream_t s);   // jobs: device [n]
cudaError_t launch_header_batch(const HeaderJob *jobs, int n, cudaStream_t s);       // jobs: device [n]

struct DecodeArgs {
    const uint32_t *words;
    unsigned long long nwords;
    const unsigned long long *chunk;  // chunk table (device)
    unsigned long long N, total_bits;
    unsigned int K;
    uint16_t *sym;
    long long *esc;                   // null: plain symbols; else receives k of every escape
    unsigned int esc_w;               // payload width of the escapes
    unsigned long long n_esc = 0;     // escapes in the stream (selects the escape stores)
    // non-null: words, nwords, chunk, total_bits and esc_w come from this
    // device-parsed header of the container at base (esc_w 0: no escapes)
    const uint8_t *base = nullptr;
    const DevHdr *dh = nullptr;
};
cudaError_t launch_decode(const DecodeArgs &a, const HuffScratch &hs, cudaStream_t s);
cudaError_t launch_histogram(const uint16_t *sym, unsigned long long N, unsigned D,
                             unsigned long long *hist, unsigned *status, cudaStream_t s);

// container offsets (same rule as the format definition)
__host__ __device__ inline unsigned long long a16(unsigned long long x) { return (x + 15) & ~15ULL; }

}  // namespace hpdr
