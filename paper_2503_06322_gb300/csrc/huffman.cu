// huffman.cu -- Huffman stage of Sec. IV-B (Alg. 2) for sm_103a: SortByKey of
// the frequencies, filter of zero frequencies, code lengths (tree_build),
// canonical codewords, encode + serialize, and the chunk-parallel decoder.
//
// Code lengths follow the two-queue Huffman rule (leaves sorted by
// (frequency, symbol); on equal weights a leaf is picked before a merged
// node).  It is computed here in rounds instead of one pick at a time: if w
// is the smallest weight left, every node created from now on weighs at least
// 2w, so all leaves and merged nodes of weight <= 2w are picked next, in
// merged order, before any new node; a round pairs an even number of them in
// parallel.  This yields exactly the picks of the sequential rule.
#include <cstdio>
#include "huffman.cuh"

namespace hpdr {
namespace {

constexpr int kRankBlocks = 152 * 2;
constexpr int kSmemKeys = 12288;     // keys one block stages in shared memory (96 KB)
constexpr int kSmemCodes = 16384;    // codewords staged by the encoder

__device__ __forceinline__ unsigned warp_sum(unsigned v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// keys of the present symbols, in increasing symbol order:
//   from a histogram: (frequency << 16) | s   (frequency > 0)
//   from lengths:     (length << 16) | s      (length > 0)
__global__ void __launch_bounds__(1024)
compact_kernel(const unsigned long long *hist, const uint8_t *len, unsigned D,
               unsigned long long *keys, unsigned *nsym, unsigned *s_lo, unsigned *s_hi)
{
    __shared__ unsigned wcnt[32], wpre[32];
    __shared__ unsigned base, lo, hi;
    const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) { base = 0; lo = 0xFFFFFFFFu; hi = 0; }
    __syncthreads();
    for (unsigned t0 = 0; t0 < D; t0 += 1024) {
        unsigned s = t0 + threadIdx.x;
        unsigned long long f = 0;
        if (s < D) f = hist ? hist[s] : (unsigned long long)len[s];
        bool p = f != 0;
        unsigned ball = __ballot_sync(0xffffffffu, p);
        if (lane == 0) wcnt[w] = __popc(ball);
        __syncthreads();
        if (w == 0) {
            unsigned v = wcnt[lane], x = v;
            for (int o = 1; o < 32; o <<= 1) {
                unsigned y = __shfl_up_sync(0xffffffffu, x, o);
                if ((int)lane >= o) x += y;
            }
            wpre[lane] = x - v;
        }
        __syncthreads();
        if (p) {
            keys[base + wpre[w] + __popc(ball & ((1u << lane) - 1))] = (f << 16) | s;
            atomicMin(&lo, s);
            atomicMax(&hi, s);
        }
        __syncthreads();
        if (threadIdx.x == 0) base += wpre[31] + wcnt[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *nsym = base;
        if (s_lo) { *s_lo = base ? lo : 0; *s_hi = base ? hi : 0; }
    }
}

// rank of every key among the n (unique) keys; scatter into sorted[] and/or rank[]
__global__ void __launch_bounds__(256)
rank_kernel(const unsigned long long *keys, const unsigned *nsym, unsigned long long *sorted,
            unsigned *rank_out)
{
    extern __shared__ unsigned long long sk[];
    const unsigned n = *nsym;
    const unsigned long long *K = keys;
    if (n <= (unsigned)kSmemKeys) {
        for (unsigned i = threadIdx.x; i < n; i += blockDim.x) sk[i] = keys[i];
        __syncthreads();
        K = sk;
    }
    const unsigned lane = threadIdx.x & 31;
    const unsigned wg = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const unsigned nw = gridDim.x * (blockDim.x >> 5);
    for (unsigned i = wg; i < n; i += nw) {
        const unsigned long long ki = K[i];
        unsigned c = 0;
        for (unsigned j = lane; j < n; j += 32) c += K[j] < ki ? 1u : 0u;
        c = warp_sum(c);
        if (lane == 0) {
            if (sorted) sorted[c] = ki;
            if (rank_out) rank_out[i] = c;
        }
    }
}

// all threads of a block take the same decision even if another block
// raises the status meanwhile
__device__ bool block_skip(const unsigned *status)
{
    __shared__ int flag;
    __syncthreads();
    if (threadIdx.x == 0) flag = *((volatile const unsigned *)status) != 0;
    __syncthreads();
    return flag != 0;
}

__device__ unsigned count_le(const unsigned long long *a, unsigned n, unsigned long long v)
{
    unsigned lo = 0, hi = n;
    while (lo < hi) { unsigned m = (lo + hi) >> 1; if (a[m] <= v) lo = m + 1; else hi = m; }
    return lo;
}
__device__ unsigned count_lt(const unsigned long long *a, unsigned n, unsigned long long v)
{
    unsigned lo = 0, hi = n;
    while (lo < hi) { unsigned m = (lo + hi) >> 1; if (a[m] < v) lo = m + 1; else hi = m; }
    return lo;
}

__device__ void length_tables(const HuffScratch &hs, unsigned *cnt)
{
    // first canonical code and start index of every length
    unsigned long long c = 0;
    int prev = -1;
    unsigned st = 0;
    bool ok = true;
    for (int L = 1; L <= kMaxCodeLen; L++) {
        hs.start[L] = st;
        hs.count[L] = cnt[L];
        if (cnt[L]) {
            if (prev >= 0) c <<= (L - prev);
            hs.first[L] = c;
            c += cnt[L];
            if (c > (1ULL << L)) ok = false;   // not a prefix code
            prev = L;
            st += cnt[L];
        } else {
            hs.first[L] = 0;
        }
    }
    hs.count[0] = 0;
    if (!ok) atomicExch(hs.status, (unsigned)DS_FORMAT);
    // left-justified limit of the codes of length <= L: (first_L + count_L) << (64 - L),
    // with first_L from the canonical recurrence for every L
    unsigned long long f = 0;
    bool started = false;
    for (int L = 1; L <= kMaxCodeLen; L++) {
        if (started) f <<= 1;
        if (cnt[L] && !started) { started = true; f = 0; }
        const unsigned long long nxt = f + cnt[L];
        hs.lim[L] = (nxt >= (1ULL << L)) ? ~0ULL : (nxt << (64 - L));
        f = nxt;
    }
    hs.lim[0] = 0;
}

// code lengths from the frequency-sorted leaves, one block
__global__ void __launch_bounds__(1024) merge_kernel(HuffScratch hs, unsigned D)
{
    extern __shared__ unsigned long long sm[];
    __shared__ unsigned ia, ib, nb, ka, kb, cnt[kMaxCodeLen + 2];
    __shared__ int done;
    const unsigned n = *hs.nsym;
    const unsigned tid = threadIdx.x;
    for (unsigned s = tid; s < D; s += blockDim.x) hs.len[s] = 0;
    for (unsigned L = tid; L < kMaxCodeLen + 2; L += blockDim.x) cnt[L] = 0;
    if (n == 0) return;
    if (n == 1) {
        __syncthreads();
        if (tid == 0) {
            unsigned s = (unsigned)(hs.sorted[0] & 0xFFFFu);
            hs.len[s] = 1;
            hs.keys2[0] = (1ULL << 16) | s;
            cnt[1] = 1;
            length_tables(hs, cnt);
        }
        return;
    }
    const bool insm = n <= (unsigned)kSmemKeys;
    unsigned long long *leafw = insm ? sm : hs.leafw;
    unsigned long long *intw = insm ? sm + n : hs.intw;
    for (unsigned i = tid; i < n; i += blockDim.x) {
        leafw[i] = hs.sorted[i] >> 16;
        intw[i] = 0;
    }
    if (tid == 0) { ia = ib = nb = 0; done = 0; }
    __syncthreads();
    const unsigned long long INF = ~0ULL;
    while (true) {
        if (tid == 0) {
            unsigned remA = n - ia, remB = nb - ib;
            if (remA + remB <= 1) {
                done = 1;
            } else {
                unsigned long long wa = remA ? leafw[ia] : INF, wb = remB ? intw[ib] : INF;
                unsigned long long wmin = wa < wb ? wa : wb;
                unsigned long long thr = wmin > (INF >> 1) ? INF : 2 * wmin;
                unsigned a = count_le(leafw + ia, remA, thr), b = count_le(intw + ib, remB, thr);
                if (a + b < 2) {
                    a = b = 0;
                    for (int t = 0; t < 2; t++) {
                        bool la = (a < remA) && (b >= remB || leafw[ia + a] <= intw[ib + b]);
                        if (la) a++; else b++;
                    }
                } else if ((a + b) & 1) {
                    if (a == 0) b--;
                    else if (b == 0) a--;
                    else if (intw[ib + b - 1] >= leafw[ia + a - 1]) b--;
                    else a--;
                }
                ka = a;
                kb = b;
            }
        }
        __syncthreads();
        if (done) break;
        const unsigned a = ka, b = kb;
        for (unsigned i = tid; i < a + b; i += blockDim.x) {
            unsigned long long w;
            unsigned q, node;
            if (i < a) {
                w = leafw[ia + i];
                q = i + count_lt(intw + ib, b, w);       // equal weights: the leaf first
                node = ia + i;
            } else {
                unsigned j = i - a;
                w = intw[ib + j];
                q = j + count_le(leafw + ia, a, w);
                node = n + ib + j;
            }
            unsigned t = nb + (q >> 1);
            atomicAdd(&intw[t], w);
            hs.parent[node] = n + t;
        }
        __syncthreads();
        if (tid == 0) { ia += a; ib += b; nb += (a + b) >> 1; }
        __syncthreads();
    }
    // depth of every node by pointer jumping (parents have larger indices)
    const unsigned total = 2 * n - 1, root = total - 1;
    unsigned *A0 = hs.anc, *A1 = hs.anc + total, *D0 = hs.dep, *D1 = hs.dep + total;
    for (unsigned i = tid; i < total; i += blockDim.x) {
        A0[i] = (i == root) ? root : hs.parent[i];
        D0[i] = (i == root) ? 0u : 1u;
    }
    __syncthreads();
    for (int step = 0; step < 7; step++) {
        for (unsigned i = tid; i < total; i += blockDim.x) {
            unsigned a = A0[i];
            D1[i] = D0[i] + D0[a];
            A1[i] = A0[a];
        }
        __syncthreads();
        unsigned *t = A0; A0 = A1; A1 = t;
        t = D0; D0 = D1; D1 = t;
    }
    for (unsigned i = tid; i < n; i += blockDim.x) {
        unsigned L = D0[i];
        if (A0[i] != root || L > (unsigned)kMaxCodeLen || L == 0) {
            atomicExch(hs.status, (unsigned)DS_LENGTH);
            L = kMaxCodeLen;
        }
        unsigned s = (unsigned)(hs.sorted[i] & 0xFFFFu);
        hs.len[s] = (uint8_t)L;
        hs.keys2[i] = ((unsigned long long)L << 16) | s;
        atomicAdd(&cnt[L], 1u);
    }
    __syncthreads();
    if (tid == 0) length_tables(hs, cnt);
}

// canonical codeword of every present symbol and the (length, symbol) order
__global__ void __launch_bounds__(256) assign_kernel(HuffScratch hs)
{
    const unsigned n = *hs.nsym;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        unsigned long long k = hs.keys2[i];
        unsigned s = (unsigned)(k & 0xFFFFu), L = (unsigned)(k >> 16);
        unsigned r = hs.rank[i];
        hs.code[s] = hs.first[L] + (r - hs.start[L]);
        hs.sorted_sym[r] = (uint16_t)s;
    }
}

// Decoder table entry of every 13-bit prefix t (P = kLutBits):
//   codeword of at most P bits:     symbol | L << 16                        (1 <= L <= P)
//   longer codewords, Lmax <= P + kSubMax, within the second-level budget:
//                                   kSubFlag | off | (Lmax - P) << 16; the next
//                                   Lmax - P bits r select lut_sub[off + r], an
//                                   entry symbol | L << 16 (0: no codeword)
//   other longer codewords:         kLongFlag | Lmin << 16 | (Lmax - Lmin) << 24
//                                   (canonical codes grow in length with their value)
//   no codeword (incomplete code):  0
constexpr uint32_t kLongFlag = 0x80000000u;
constexpr uint32_t kSubFlag = 0x20000000u;
// decoder copy of an entry of the escape symbol 0 whose codeword and payload
// (W bits) together fit 32 bits: L = codeword length + W
constexpr uint32_t kEscFolded = 0x40000000u;

// canonical length tables staged in shared memory
struct LenTabs {
    unsigned long long first[64], lim[64];
    unsigned start[64], count[64];
};

// length of the canonical codeword at the top of the left-aligned window,
// known to lie in [lo, hi]: the first length l in [lo, hi) whose limit lim[l]
// the window stays below, else hi (the limits do not decrease with l, so a
// binary search finds it)
__device__ __forceinline__ unsigned code_len_in(const LenTabs &t, unsigned long long win, unsigned lo, unsigned hi)
{
    while (lo < hi) {
        const unsigned m = (lo + hi) >> 1;
        if (win >= t.lim[m]) lo = m + 1; else hi = m;
    }
    return lo;
}

// symbol | L << 16 of the codeword of length L at the top of the window (0: none)
__device__ __forceinline__ uint32_t leaf_of(const LenTabs &t, const uint16_t *sorted_sym, unsigned n,
                                            unsigned long long win, unsigned L)
{
    const unsigned long long off = (win >> (64 - L)) - t.first[L];
    if (off >= t.count[L]) return 0u;
    const unsigned idx = t.start[L] + (unsigned)off;
    return idx < n ? ((uint32_t)sorted_sym[idx] | (L << 16)) : 0u;
}

// One block of 1024 threads, eight consecutive prefixes each.  The
// second-level tables are laid out in prefix order by a block scan of their
// sizes; prefixes past the budget keep long entries.  The sorted symbols are
// staged in shared memory when there are at most kLutSyms of them.
constexpr int kLutThreads = 1024;
constexpr unsigned kLutPer = (1u << kLutBits) / kLutThreads;
constexpr unsigned kLutSyms = 16384;
constexpr size_t kLutSmem = (4u << kLutBits) + 2 * kLutSyms;
__global__ void __launch_bounds__(kLutThreads, 1) lut_kernel(HuffScratch hs)
{
    __shared__ LenTabs T;
    __shared__ unsigned wsum[kLutThreads / 32];
    __shared__ unsigned total;
    extern __shared__ __align__(16) unsigned char lsm[];
    uint32_t *ent = reinterpret_cast<uint32_t *>(lsm);                         // [1 << kLutBits]
    uint16_t *ssym = reinterpret_cast<uint16_t *>(ent + (1u << kLutBits));      // [kLutSyms]
    const unsigned tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 64) {
        T.first[tid] = hs.first[tid];
        T.lim[tid] = hs.lim[tid];
        T.start[tid] = hs.start[tid];
        T.count[tid] = hs.count[tid];
    }
    const unsigned n = *hs.nsym;
    const uint16_t *sorted = n <= kLutSyms ? ssym : hs.sorted_sym;
    if (n <= kLutSyms)
        for (unsigned i = tid; i < n; i += kLutThreads) ssym[i] = hs.sorted_sym[i];
    __syncthreads();
    const bool ok = *hs.status == 0;
    unsigned maxL = 0;
    for (int l = kMaxCodeLen; l >= 1; l--) if (T.count[l]) { maxL = (unsigned)l; break; }
    const bool any = ok && maxL;
    const unsigned t0 = tid * kLutPer;
    constexpr unsigned long long kTail = (1ULL << (64 - kLutBits)) - 1;
    unsigned mine = 0;
    unsigned char sbs[kLutPer];
#pragma unroll
    for (unsigned j = 0; j < kLutPer; j++) {
        const unsigned t = t0 + j;
        uint32_t e = 0;
        sbs[j] = 0;
        if (any) {
            // the codeword whose left-justified range holds t's first bit string;
            // at most P bits long, it is a prefix of every extension of t
            const unsigned long long w0 = (unsigned long long)t << (64 - kLutBits);
            const unsigned lmin = code_len_in(T, w0, 1, maxL);
            if (lmin <= (unsigned)kLutBits) {
                e = leaf_of(T, sorted, n, w0, lmin);
            } else {
                const unsigned lmax = code_len_in(T, w0 | kTail, lmin, maxL);
                e = kLongFlag | (lmin << 16) | ((lmax - lmin) << 24);
                if (lmax <= (unsigned)(kLutBits + kSubMax)) {
                    sbs[j] = (unsigned char)(lmax - kLutBits);
                    mine += 1u << (lmax - kLutBits);
                }
            }
        }
        ent[t] = e;
    }
    // exclusive scan of the second-level sizes over the block
    unsigned incl = mine;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (unsigned)o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const unsigned v = wsum[lane];
        unsigned x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= (unsigned)o) x += y;
        }
        wsum[lane] = x - v;
        if (lane == 31) total = x < kSubCap ? x : kSubCap;
    }
    __syncthreads();
    unsigned off = wsum[warp] + incl - mine;
#pragma unroll
    for (unsigned j = 0; j < kLutPer; j++) {
        if (!sbs[j]) continue;
        const unsigned sz = 1u << sbs[j];
        if (off + sz <= kSubCap) ent[t0 + j] = kSubFlag | off | ((unsigned)sbs[j] << 16);
        off += sz;
    }
    __syncthreads();
    for (unsigned t = tid; t < (1u << kLutBits); t += kLutThreads) hs.lut1[t] = ent[t];
    // second-level entries: a warp per prefix, a lane per suffix
    for (unsigned t = warp; t < (1u << kLutBits); t += kLutThreads / 32) {
        const uint32_t e = ent[t];
        if ((e & (kLongFlag | kSubFlag)) != kSubFlag) continue;
        const unsigned sb = (e >> 16) & 0xFu, base = e & 0xFFFFu;
        const unsigned long long w0 = (unsigned long long)t << (64 - kLutBits);
        const unsigned lo = code_len_in(T, w0, 1, maxL);
        for (unsigned r = lane; r < (1u << sb); r += 32) {
            const unsigned long long w = w0 | ((unsigned long long)r << (64 - kLutBits - sb));
            hs.lut_sub[base + r] = leaf_of(T, sorted, n, w, code_len_in(T, w, lo, kLutBits + sb));
        }
    }
    if (tid == 0) *hs.nsub = any ? total : 0u;
}

// Canonical codewords (Sec. IV-B): the present symbols ordered by (length,
// symbol) get consecutive codewords within each length, so a symbol's rank is
// start[L] plus the number of smaller symbols of its length L, and its
// codeword first[L] plus that number.  The block (1024 threads) walks the
// alphabet in tiles of 1024 symbols: __match_any_sync groups a warp's lanes by
// length, wc[warp][L] holds per-warp counts that are then scanned over the
// warps of every length on top of the running totals of the earlier tiles.
constexpr int kWcStride = 65;     // 64 lengths, padded against bank conflicts
__device__ void canonical_assign(const uint8_t *lens, unsigned D, const unsigned *sstart,
                                 const unsigned long long *sfirst, unsigned *wc, unsigned *run,
                                 unsigned long long *code, uint16_t *sorted_sym)
{
    const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (unsigned i = threadIdx.x; i < 64; i += blockDim.x) run[i] = 0;
    for (unsigned t0 = 0; t0 < D; t0 += 1024) {
        for (unsigned i = threadIdx.x; i < 32 * kWcStride; i += blockDim.x) wc[i] = 0;
        __syncthreads();
        const unsigned s = t0 + threadIdx.x;
        const unsigned L = s < D ? lens[s] : 0u;
        const unsigned m = __match_any_sync(0xffffffffu, L);
        const unsigned below = __popc(m & ((1u << lane) - 1));
        if (below == 0) wc[w * kWcStride + L] = __popc(m);
        __syncthreads();
        for (unsigned Lq = w; Lq < 64; Lq += 32) {
            const unsigned x = wc[lane * kWcStride + Lq];
            unsigned y = x;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned z = __shfl_up_sync(0xffffffffu, y, o);
                if ((int)lane >= o) y += z;
            }
            const unsigned base = run[Lq];
            __syncwarp();
            wc[lane * kWcStride + Lq] = base + y - x;
            if (lane == 31) run[Lq] = base + y;
        }
        __syncthreads();
        if (L) {
            const unsigned k = wc[w * kWcStride + L] + below;
            if (code) code[s] = sfirst[L] + k;
            sorted_sym[sstart[L] + k] = (uint16_t)s;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// One-block codebook for alphabets of at most kFusedMaxD symbols, everything
// in shared memory: present symbols, their (frequency, symbol) order, the
// two-queue code lengths in rounds (as merge_kernel), depths by pointer
// jumping, canonical codewords.  Rounds that pick at most kWarpRound nodes,
// the common case once the smallest weights are merged, run on warp 0 alone
// without block barriers.
constexpr unsigned kFusedMaxD = 8192;
constexpr unsigned kWarpRound = 64;
constexpr size_t kCodebookSmem = 16ull * kFusedMaxD            // keys + sort buffer / internal weights
                                 + 2ull * 2 * kFusedMaxD         // parent / ancestor
                                 + 2ull * kFusedMaxD             // depth
                                 + kFusedMaxD                    // lengths by symbol
                                 + 4ull * 32 * kWcStride;        // per-warp length counts

// number of the first rem sorted values v(i) that are <= thr (v non-decreasing),
// by warp ballot over the first 32 and binary search beyond
template <typename F>
__device__ __forceinline__ unsigned warp_count_le(F v, unsigned rem, unsigned long long thr, unsigned lane)
{
    const bool p = lane < rem && v(lane) <= thr;
    const unsigned c = __popc(__ballot_sync(0xffffffffu, p));
    if (c < 32 || rem <= 32) return c;
    unsigned lo = 32, hi = rem;
    while (lo < hi) { const unsigned m = (lo + hi) >> 1; if (v(m) <= thr) lo = m + 1; else hi = m; }
    return lo;
}

// sorted ascending 8 keys in registers (odd-even transposition, 8 rounds)
__device__ __forceinline__ void sort8(unsigned long long (&k)[8])
{
#pragma unroll
    for (int r = 0; r < 8; r++) {
#pragma unroll
        for (int i = r & 1; i + 1 < 8; i += 2) {
            const unsigned long long a = k[i], b = k[i + 1];
            k[i] = a < b ? a : b;
            k[i + 1] = a < b ? b : a;
        }
    }
}

__device__ __forceinline__ void codebook_body(const unsigned long long *hist, unsigned D, const HuffScratch &hs)
{
    extern __shared__ __align__(16) unsigned char csm[];
    unsigned long long *key = reinterpret_cast<unsigned long long *>(csm);   // [kFusedMaxD]
    unsigned long long *aux = key + kFusedMaxD;                              // [kFusedMaxD]
    uint16_t *par = reinterpret_cast<uint16_t *>(aux + kFusedMaxD);          // [2 kFusedMaxD]
    uint16_t *dep = par + 2 * kFusedMaxD;                                    // [kFusedMaxD] as bytes x2
    uint8_t *lens = reinterpret_cast<uint8_t *>(dep + kFusedMaxD);           // [kFusedMaxD]
    unsigned *wc = reinterpret_cast<unsigned *>(lens + kFusedMaxD);          // [32 * kWcStride]
    uint8_t *depb = reinterpret_cast<uint8_t *>(dep);                        // [2 kFusedMaxD]
    __shared__ unsigned wcnt[32], wpre[32], cnt[64], run[64], sstart[64];
    __shared__ unsigned long long sfirst[64];
    __shared__ unsigned sh_n, sh_lo, sh_hi, s_ia, s_ib, s_nb, s_a, s_b;
    __shared__ int s_done;
    const unsigned tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned long long INF = ~0ULL;

    // 1. present symbols as keys (frequency << 16) | s, in symbol order
    if (tid == 0) { sh_n = 0; sh_lo = 0xFFFFFFFFu; sh_hi = 0; }
    for (unsigned i = tid; i < 64; i += blockDim.x) cnt[i] = 0;
    for (unsigned i = tid; i < D; i += blockDim.x) lens[i] = 0;
    __syncthreads();
    for (unsigned t0 = 0; t0 < D; t0 += 1024) {
        const unsigned s = t0 + tid;
        const unsigned long long f = s < D ? hist[s] : 0ULL;
        const bool p = f != 0;
        const unsigned ball = __ballot_sync(0xffffffffu, p);
        if (lane == 0) wcnt[w] = __popc(ball);
        __syncthreads();
        if (w == 0) {
            const unsigned v = wcnt[lane];
            unsigned x = v;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
                if ((int)lane >= o) x += y;
            }
            wpre[lane] = x - v;
        }
        __syncthreads();
        if (p) {
            key[sh_n + wpre[w] + __popc(ball & ((1u << lane) - 1))] = (f << 16) | s;
            atomicMin(&sh_lo, s);
            atomicMax(&sh_hi, s);
        }
        __syncthreads();
        if (tid == 0) sh_n += wpre[31] + wcnt[31];
        __syncthreads();
    }
    const unsigned n = sh_n;
    if (tid == 0) {
        *hs.nsym = n;
        *hs.s_lo = n ? sh_lo : 0;
        *hs.s_hi = n ? sh_hi : 0;
    }
    if (n == 0) {
        for (unsigned i = tid; i < D; i += blockDim.x) hs.len[i] = 0;
        return;
    }

    // 2. sort the keys (unique) ascending: runs of 8 in registers, then
    //    merge-path rounds in shared memory
    unsigned P = 8;
    while (P < n) P <<= 1;
    unsigned rounds = 0;
    for (unsigned r = 8; r < P; r <<= 1) rounds++;
    {
        unsigned long long *dst = (rounds & 1) ? aux : key;
        unsigned long long k8[8];
        const bool act = tid * 8 < P;
        if (act) {
#pragma unroll
            for (int i = 0; i < 8; i++) k8[i] = (tid * 8 + i < n) ? key[tid * 8 + i] : INF;
            sort8(k8);
        }
        __syncthreads();
        if (act) {
#pragma unroll
            for (int i = 0; i < 8; i++) dst[tid * 8 + i] = k8[i];
        }
        __syncthreads();
        unsigned long long *src = dst;
        for (unsigned R = 8; R < P; R <<= 1) {
            dst = (src == key) ? aux : key;
            if (act) {
                const unsigned o = tid * 8, pair = o / (2 * R), d = o % (2 * R);
                const unsigned long long *A = src + pair * 2 * R, *B = A + R;
                unsigned lo = d > R ? d - R : 0, hi = d < R ? d : R;
                while (lo < hi) {
                    const unsigned m = (lo + hi) >> 1;
                    if (A[m] <= B[d - m - 1]) lo = m + 1; else hi = m;
                }
                unsigned i = lo, j = d - lo;
#pragma unroll
                for (int e = 0; e < 8; e++) {
                    unsigned long long v;
                    if (j >= R || (i < R && A[i] <= B[j])) { v = A[i]; i++; } else { v = B[j]; j++; }
                    dst[o + e] = v;
                }
            }
            __syncthreads();
            src = dst;
        }
    }
    // key[0, n) sorted; aux becomes the internal node weights
    for (unsigned i = tid; i < n; i += blockDim.x) aux[i] = 0;
    unsigned long long *intw = aux;
    auto LW = [&](unsigned i) { return key[i] >> 16; };

    // 3. two-queue merging in rounds
    if (tid == 0) { s_ia = s_ib = s_nb = 0; s_done = 0; }
    __syncthreads();
    // s_done is read only between the barrier after warp 0 writes it and the
    // next round's barriers, so every warp leaves the loop at the same barrier
    while (n > 1) {
        if (w == 0) {
            unsigned ia = s_ia, ib = s_ib, nb = s_nb, a = 0, b = 0;
            int state = 0;
            while (true) {
                const unsigned remA = n - ia, remB = nb - ib;
                if (remA + remB <= 1) { state = 2; break; }
                const unsigned long long wa = remA ? LW(ia) : INF, wb = remB ? intw[ib] : INF;
                const unsigned long long wmin = wa < wb ? wa : wb;
                const unsigned long long thr = wmin > (INF >> 1) ? INF : 2 * wmin;
                a = warp_count_le([&](unsigned i) { return LW(ia + i); }, remA, thr, lane);
                b = warp_count_le([&](unsigned i) { return intw[ib + i]; }, remB, thr, lane);
                if (a + b < 2) {
                    a = b = 0;
                    for (int t = 0; t < 2; t++) {
                        const bool la = (a < remA) && (b >= remB || LW(ia + a) <= intw[ib + b]);
                        if (la) a++; else b++;
                    }
                } else if ((a + b) & 1) {
                    if (a == 0) b--;
                    else if (b == 0) a--;
                    else if (intw[ib + b - 1] >= LW(ia + a - 1)) b--;
                    else a--;
                }
                if (a + b > kWarpRound) { state = 1; break; }
                for (unsigned i = lane; i < a + b; i += 32) {
                    unsigned long long wt;
                    unsigned q, node;
                    if (i < a) {
                        wt = LW(ia + i);
                        unsigned lo = 0, hi = b;     // internal weights < wt come first
                        while (lo < hi) { const unsigned m = (lo + hi) >> 1; if (intw[ib + m] < wt) lo = m + 1; else hi = m; }
                        q = i + lo;
                        node = ia + i;
                    } else {
                        const unsigned j = i - a;
                        wt = intw[ib + j];
                        unsigned lo = 0, hi = a;     // leaves <= wt come first
                        while (lo < hi) { const unsigned m = (lo + hi) >> 1; if (LW(ia + m) <= wt) lo = m + 1; else hi = m; }
                        q = j + lo;
                        node = n + ib + j;
                    }
                    const unsigned t = nb + (q >> 1);
                    atomicAdd(&intw[t], wt);
                    par[node] = (uint16_t)(n + t);
                }
                __syncwarp();
                ia += a; ib += b; nb += (a + b) >> 1;
            }
            if (lane == 0) {
                s_ia = ia; s_ib = ib; s_nb = nb; s_a = a; s_b = b;
                s_done = state == 2;
            }
        }
        __syncthreads();
        if (s_done) break;
        {
            const unsigned ia = s_ia, ib = s_ib, nb = s_nb, a = s_a, b = s_b;
            for (unsigned i = tid; i < a + b; i += blockDim.x) {
                unsigned long long wt;
                unsigned q, node;
                if (i < a) {
                    wt = LW(ia + i);
                    q = i + count_lt(intw + ib, b, wt);
                    node = ia + i;
                } else {
                    const unsigned j = i - a;
                    wt = intw[ib + j];
                    unsigned lo = 0, hi = a;
                    while (lo < hi) { const unsigned m = (lo + hi) >> 1; if (LW(ia + m) <= wt) lo = m + 1; else hi = m; }
                    q = j + lo;
                    node = n + ib + j;
                }
                const unsigned t = nb + (q >> 1);
                atomicAdd(&intw[t], wt);
                par[node] = (uint16_t)(n + t);
            }
        }
        __syncthreads();
        if (tid == 0) { s_ia += s_a; s_ib += s_b; s_nb += (s_a + s_b) >> 1; }
        __syncthreads();
    }

    // 4. depth of every node by pointer jumping (parents have larger indices)
    const unsigned total = 2 * n - 1, root = total - 1;
    for (unsigned i = tid; i < total; i += blockDim.x) {
        if (i == root) par[i] = (uint16_t)root;
        depb[i] = i == root ? 0 : 1;
    }
    __syncthreads();
    for (int step = 0; step < 7; step++) {
        uint16_t na[16];
        uint8_t nd[16];
#pragma unroll
        for (int k = 0; k < 16; k++) {
            const unsigned i = tid + 1024u * k;
            if (i < total) {
                const unsigned a = par[i];
                const unsigned dd = (unsigned)depb[i] + depb[a];
                nd[k] = (uint8_t)(dd > 255 ? 255 : dd);
                na[k] = par[a];
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; k++) {
            const unsigned i = tid + 1024u * k;
            if (i < total) { par[i] = na[k]; depb[i] = nd[k]; }
        }
        __syncthreads();
    }

    // 5. code lengths, per-length counts, canonical tables and codewords
    for (unsigned i = tid; i < n; i += blockDim.x) {
        unsigned L = n == 1 ? 1u : depb[i];
        if (n > 1 && (par[i] != root || L > (unsigned)kMaxCodeLen || L == 0)) {
            atomicExch(hs.status, (unsigned)DS_LENGTH);
            L = kMaxCodeLen;
        }
        lens[(unsigned)(key[i] & 0xFFFFu)] = (uint8_t)L;
        atomicAdd(&cnt[L], 1u);
    }
    __syncthreads();
    for (unsigned i = tid; i < D; i += blockDim.x) hs.len[i] = lens[i];
    if (tid == 0) length_tables(hs, cnt);
    __syncthreads();
    if (tid < 64) { sstart[tid] = hs.start[tid]; sfirst[tid] = hs.first[tid]; }
    __syncthreads();
    canonical_assign(lens, D, sstart, sfirst, wc, run, hs.code, hs.sorted_sym);
}

__global__ void __launch_bounds__(1024, 1) codebook_kernel(const unsigned long long *hist, unsigned D, HuffScratch hs)
{
    codebook_body(hist, D, hs);
}

// one codebook per block: the codebooks of a batch of fields in one launch
__global__ void __launch_bounds__(1024, 1) codebook_batch_kernel(const CodebookJob *jobs)
{
    const CodebookJob j = jobs[blockIdx.x];
    codebook_body(j.hist, j.D, j.hs);
}

// Decoder tables from the code lengths of symbols s_lo..s_hi (every other
// symbol of the alphabet absent), one block of 1024 threads: counts,
// canonical tables, the (length, symbol) order of the symbols.
__global__ void __launch_bounds__(1024, 1) dec_tables_kernel(const uint8_t *lenb, unsigned s_lo, unsigned s_hi,
                                                             unsigned D, HuffScratch hs, const uint8_t *base,
                                                             const DevHdr *dh)
{
    if (dh) {
        // a header parsed on the device (and rejected there: nothing to build)
        if (block_skip(hs.status)) return;
        lenb = base + dh->off_len;
        s_lo = dh->s_lo;
        s_hi = dh->s_hi;
    }
    extern __shared__ __align__(16) unsigned char tsm[];
    unsigned *wc = reinterpret_cast<unsigned *>(tsm);                        // [32 * kWcStride]
    uint8_t *lens = tsm + 4 * 32 * kWcStride;                                // [D]
    __shared__ unsigned cnt[64], run[64], sstart[64], nsum;
    __shared__ unsigned long long sfirst[64];
    const unsigned tid = threadIdx.x;
    for (unsigned i = tid; i < 64; i += blockDim.x) cnt[i] = 0;
    if (tid == 0) nsum = 0;
    __syncthreads();
    unsigned mine = 0;
    for (unsigned s = tid; s < D; s += blockDim.x) {
        unsigned L = (s >= s_lo && s <= s_hi) ? lenb[s - s_lo] : 0u;
        if (L > (unsigned)kMaxCodeLen) { atomicExch(hs.status, (unsigned)DS_FORMAT); L = 0; }
        lens[s] = (uint8_t)L;
        if (L) { atomicAdd(&cnt[L], 1u); mine++; }
    }
    mine = warp_sum(mine);
    if ((tid & 31) == 0 && mine) atomicAdd(&nsum, mine);
    __syncthreads();
    if (tid == 0) {
        *hs.nsym = nsum;
        if (nsum == 0) atomicExch(hs.status, (unsigned)DS_FORMAT);
        length_tables(hs, cnt);
    }
    __syncthreads();
    if (tid < 64) { sstart[tid] = hs.start[tid]; sfirst[tid] = hs.first[tid]; }
    __syncthreads();
    canonical_assign(lens, D, sstart, sfirst, wc, run, nullptr, hs.sorted_sym);
}

// ---------------------------------------------------------------------------
// Encoder

struct Layout {
    unsigned long long off_len, off_chunk, off_bits, total;
};
__device__ __forceinline__ Layout container_layout(int L, unsigned long long ncoord, unsigned s_lo, unsigned s_hi,
                                                   unsigned long long nch, unsigned long long bits)
{
    Layout y;
    // the node coordinates (ncoord values, when the container carries them) follow q[L+1]
    y.off_len = a16(128 + 8ULL * (L + 1) + 8ULL * ncoord);
    y.off_chunk = a16(y.off_len + (s_hi - s_lo + 1));
    y.off_bits = a16(y.off_chunk + 8 * nch);
    y.total = y.off_bits + 4 * ((bits + 31) / 32);
    return y;
}

constexpr int kEncBlocks = 152 * 4;

// The encoder's unit of work: a warp takes r consecutive chunks (r K symbols,
// 32 per lane) when K < 1024 divides 1024, else one chunk.  The bitstream is
// continuous across chunks, so the grouping changes no output bit.
__host__ __device__ inline unsigned enc_group(unsigned K) { return (K < 1024 && 1024 % K == 0) ? 1024 / K : 1; }

// bits of every chunk (codewords + escape payloads); block b owns the
// contiguous chunk range [b*cpb, (b+1)*cpb) and leaves its sum in bsum
__global__ void __launch_bounds__(256) enc_count_kernel(EncodeArgs a)
{
    extern __shared__ uint8_t slen[];
    __shared__ unsigned long long wb[8];
    if (block_skip(&a.sc->status)) return;
    for (unsigned i = threadIdx.x; i < a.D; i += blockDim.x) slen[i] = a.len[i];
    __syncthreads();
    // an escape adds its payload width to its codeword
    if (a.esc && threadIdx.x == 0) slen[0] = (uint8_t)(slen[0] + a.sc->esc_w);
    __syncthreads();
    const unsigned long long nch = (a.N + a.K - 1) / a.K;
    const unsigned long long cpb = (nch + gridDim.x - 1) / gridDim.x;
    const unsigned long long c0 = blockIdx.x * cpb, c1 = c0 + cpb < nch ? c0 + cpb : nch;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long tb = 0;
    const unsigned r = enc_group(a.K);
    if (r > 1) {
        // r chunks per warp, 32 / r lanes per chunk, 32 symbols per lane
        const unsigned lpc = 32 / r;
        for (unsigned long long g = c0 + (unsigned long long)warp * r; g < c1; g += (blockDim.x >> 5) * r) {
            const unsigned long long c = g + lane / lpc;
            unsigned long long bits = 0;
            if (c < c1) {
                const unsigned long long beg = c * a.K + (unsigned long long)(lane % lpc) * 32;
                const unsigned long long cend = (c + 1) * a.K < a.N ? (c + 1) * a.K : a.N;
                if (beg + 32 <= cend) {
                    const uint4 *v = reinterpret_cast<const uint4 *>(a.sym + beg);
                    uint4 x[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) x[u] = v[u];
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const uint16_t *e = reinterpret_cast<const uint16_t *>(&x[u]);
#pragma unroll
                        for (int k = 0; k < 8; k++) bits += slen[e[k]];
                    }
                } else {
                    for (unsigned long long i = beg; i < cend; i++) bits += slen[a.sym[i]];
                }
            }
            // sum over the lpc lanes of each chunk
            for (unsigned o = 1; o < lpc; o <<= 1) bits += __shfl_xor_sync(0xffffffffu, bits, o);
            if (lane % lpc == 0 && c < c1) { a.chunk_bits[c] = bits; tb += bits; }
        }
        tb = warp_sum64(tb);
    } else
    for (unsigned long long c = c0 + warp; c < c1; c += blockDim.x >> 5) {
        const unsigned long long beg = c * a.K;
        const unsigned long long end = beg + a.K < a.N ? beg + a.K : a.N;
        unsigned long long bits = 0;
        if (end - beg == a.K) {
            // four 16-byte loads per lane in flight (K is a multiple of 128)
            const uint4 *v = reinterpret_cast<const uint4 *>(a.sym + beg);
            const unsigned nq = a.K / 8;
            for (unsigned i0 = lane; i0 < nq; i0 += 128) {
                uint4 x[4];
                bool ok[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    ok[u] = i0 + 32 * u < nq;
                    if (ok[u]) x[u] = v[i0 + 32 * u];
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    if (!ok[u]) continue;
                    const uint16_t *e = reinterpret_cast<const uint16_t *>(&x[u]);
#pragma unroll
                    for (int k = 0; k < 8; k++) bits += slen[e[k]];
                }
            }
        } else {
            for (unsigned long long i = beg + lane; i < end; i += 32) bits += slen[a.sym[i]];
        }
        bits = warp_sum64(bits);
        if (lane == 0) { a.chunk_bits[c] = bits; tb += bits; }
    }
    if (lane == 0) wb[warp] = tb;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long x = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) x += wb[w];
        a.bsum[blockIdx.x] = x;
    }
}

// exclusive scan of the block sums (one block), container layout and capacity
__global__ void __launch_bounds__(1024) enc_scan1_kernel(EncodeArgs a, int nb)
{
    __shared__ unsigned long long sb[1024];
    if (block_skip(&a.sc->status)) return;
    const int t = threadIdx.x;
    sb[t] = t < nb ? a.bsum[t] : 0;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        unsigned long long x = t >= o ? sb[t - o] : 0;
        __syncthreads();
        sb[t] += x;
        __syncthreads();
    }
    // inclusive -> exclusive
    if (t < nb) a.bsum[t] = t ? sb[t - 1] : 0;
    if (t == 0) {
        const unsigned long long nch = (a.N + a.K - 1) / a.K;
        const unsigned long long x = sb[1023];
        if (a.container) {
            Layout lay = container_layout(a.L, a.ncoord, a.sc->s_lo, a.sc->s_hi, nch, x);
            if (lay.total > a.capacity) atomicExch(&a.sc->status, (unsigned)DS_CAPACITY);
            a.sc->out_bytes = lay.total;
        } else {
            if ((x + 31) / 32 > a.words_cap) atomicExch(&a.sc->status, (unsigned)DS_CAPACITY);
        }
        a.sc->total_bits = x;
    }
}

__device__ __forceinline__ uint32_t *enc_words(const EncodeArgs &a, unsigned long long nch)
{
    if (!a.container) return a.words_out;
    Layout lay = container_layout(a.L, a.ncoord, a.sc->s_lo, a.sc->s_hi, nch, a.sc->total_bits);
    return reinterpret_cast<uint32_t *>(a.container + lay.off_bits);
}

// chunk offsets within each block's range (plus the block's offset), chunk
// table, and zeroed words where more than one writer will meet
__global__ void __launch_bounds__(256) enc_scan2_kernel(EncodeArgs a)
{
    __shared__ unsigned long long sb[256];
    if (block_skip(&a.sc->status)) return;
    const unsigned long long nch = (a.N + a.K - 1) / a.K;
    const unsigned long long cpb = (nch + gridDim.x - 1) / gridDim.x;
    const unsigned long long c0 = blockIdx.x * cpb, c1 = c0 + cpb < nch ? c0 + cpb : nch;
    uint32_t *words = enc_words(a, nch);
    unsigned long long *ctab = a.chunk_out;
    if (a.container) {
        Layout lay = container_layout(a.L, a.ncoord, a.sc->s_lo, a.sc->s_hi, nch, a.sc->total_bits);
        ctab = reinterpret_cast<unsigned long long *>(a.container + lay.off_chunk);
    }
    const unsigned long long total = a.sc->total_bits;
    unsigned long long carry = a.bsum[blockIdx.x];
    const int t = threadIdx.x;
    for (unsigned long long base = c0; base < c1; base += 256) {
        const unsigned long long c = base + t;
        unsigned long long v = c < c1 ? a.chunk_bits[c] : 0;
        sb[t] = v;
        __syncthreads();
        for (int o = 1; o < 256; o <<= 1) {
            unsigned long long x = t >= o ? sb[t - o] : 0;
            __syncthreads();
            sb[t] += x;
            __syncthreads();
        }
        if (c < c1) {
            const unsigned long long off = carry + sb[t] - v;
            a.chunk_bits[c] = off;
            ctab[c] = off;
            const unsigned long long cend = off + v;
            // a complete group of at least 1024 symbols (one warp, 32 or more per lane)
            // shares only its first word with the previous group and stores every
            // other word whole; other chunks are written word by word with atomics:
            // zero them
            const unsigned r = enc_group(a.K);
            const unsigned long long G = (unsigned long long)a.K * r;
            const bool full = (c / r + 1) * G <= a.N && G >= 1024;
            if (full) {
                if (c % r == 0) words[off >> 5] = 0u;
            } else {
                for (unsigned long long w = off >> 5; w <= ((cend ? cend - 1 : 0) >> 5); w++) words[w] = 0u;
            }
            if (c + 1 == nch && (total & 31)) words[total >> 5] = 0u;
        }
        __syncthreads();
        carry += sb[255];
        __syncthreads();
    }
    if (blockIdx.x == 0 && t == 0) a.chunk_bits[nch] = total;
}

// one warp per group of chunks (enc_group): every lane encodes 32 (K/32 when
// K >= 1024) consecutive symbols, assembling its bits in a 64-bit register and
// storing whole words; the partial words at lane boundaries are merged through
// shuffles (complete groups) or atomics (the last, partial group)
__global__ void __launch_bounds__(256) enc_write_kernel(EncodeArgs a)
{
    extern __shared__ uint32_t esm32[];
    if (block_skip(&a.sc->status)) return;
    // codeword table: code << 8 | length for codewords of at most 24 bits; a
    // length field of 0xFF sends the symbol to the global tables
    const bool code_sm = a.D <= (unsigned)kSmemCodes;
    uint32_t *spk = esm32;
    // per warp: the 32 symbols of every lane, 17 words per lane (conflict-free)
    uint32_t *sw = esm32 + (code_sm ? a.D : 0) + (threadIdx.x >> 5) * (32 * 17);
    const uint16_t *ss = reinterpret_cast<const uint16_t *>(sw + (threadIdx.x & 31) * 17);
    if (code_sm)
        for (unsigned i = threadIdx.x; i < a.D; i += blockDim.x) {
            const unsigned L = a.len[i];
            spk[i] = L <= 24 ? (uint32_t)((a.code[i] << 8) | L) : 0xFFu;
        }
    __syncthreads();
    // (codeword, length) of symbol s
    auto cw_of = [&](unsigned sv, unsigned long long &cw, int &L) {
        const uint32_t e = code_sm ? spk[sv] : 0xFFu;
        if ((e & 0xFFu) != 0xFFu) { cw = e >> 8; L = (int)(e & 0xFFu); }
        else { cw = a.code[sv]; L = a.len[sv]; }
    };
    const unsigned long long nch = (a.N + a.K - 1) / a.K;
    uint32_t *__restrict__ words = enc_words(a, nch);
    const long long *__restrict__ esc = a.esc;
    const int ew = esc ? (int)a.sc->esc_w : 0;       // escape payload width
    const unsigned lane = threadIdx.x & 31;
    const unsigned r = enc_group(a.K);
    const unsigned long long G = (unsigned long long)a.K * r;   // symbols per warp group
    const unsigned long long ngr = (a.N + G - 1) / G;
    const unsigned spl = (unsigned)(G >> 5);
    const unsigned long long wg = blockIdx.x * (unsigned long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const unsigned long long nw = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    for (unsigned long long c = wg; c < ngr; c += nw) {
        const unsigned long long beg = c * G;
        const unsigned long long end = beg + G < a.N ? beg + G : a.N;
        unsigned long long m0 = beg + (unsigned long long)lane * spl, m1 = m0 + spl;
        if (m0 > end) m0 = end;
        if (m1 > end) m1 = end;
        unsigned long long mb = 0;
        // full lanes of 8, 16 or 32 symbols stage them in shared memory (16-byte loads)
        const bool regs = (m1 - m0 == spl) && (spl == 32 || spl == 16 || spl == 8);
        if (regs) {
            const uint4 *v = reinterpret_cast<const uint4 *>(a.sym + m0);
            const int nq = (int)spl / 8;
            uint4 x[4];
#pragma unroll
            for (int q = 0; q < 4; q++) if (q < nq) x[q] = v[q];
            uint32_t *dw = sw + lane * 17;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                if (q < nq) {
                    dw[4 * q] = x[q].x; dw[4 * q + 1] = x[q].y; dw[4 * q + 2] = x[q].z; dw[4 * q + 3] = x[q].w;
                }
            }
#pragma unroll 4
            for (int q = 0; q < (int)spl; q++) {
                const unsigned sv = ss[q];
                const uint32_t e = code_sm ? spk[sv] : 0xFFu;
                mb += ((e & 0xFFu) != 0xFFu ? (e & 0xFFu) : a.len[sv]) + (sv == 0 ? ew : 0);
            }
        } else {
            for (unsigned long long i = m0; i < m1; i++) {
                const uint16_t s = a.sym[i];
                mb += a.len[s] + (s == 0 ? ew : 0);
            }
        }
        unsigned long long xb = mb;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long yb = __shfl_up_sync(0xffffffffu, xb, o);
            if ((int)lane >= o) xb += yb;
        }
        const unsigned long long start = a.chunk_bits[c * r] + xb - mb;
        unsigned long long acc = 0;
        unsigned nacc = (unsigned)(start & 31);
        unsigned long long widx = start >> 5;
        const unsigned long long fidx = widx;
        uint32_t firstw = 0;
        bool have_first = false;
        // append the low L bits of cw (L <= 64), most significant first
        auto emit = [&](unsigned long long cw, int L) {
            if (L <= 32) {
                // nacc < 32 here, so the codeword fits the 64-bit accumulator whole
                acc |= cw << (64 - nacc - L);
                nacc += L;
                if (nacc >= 32) {
                    const uint32_t wv = (uint32_t)(acc >> 32);
                    if (!have_first) { firstw = wv; have_first = true; }
                    else words[widx] = wv;
                    widx++;
                    acc <<= 32;
                    nacc -= 32;
                }
                return;
            }
            while (L > 0) {
                const int take = L > 32 ? 32 : L;
                const unsigned long long part = (cw >> (L - take)) & ((1ULL << take) - 1);
                L -= take;
                acc |= part << (64 - nacc - take);
                nacc += take;
                if (nacc >= 32) {
                    const uint32_t wv = (uint32_t)(acc >> 32);
                    if (!have_first) { firstw = wv; have_first = true; }
                    else words[widx] = wv;
                    widx++;
                    acc <<= 32;
                    nacc -= 32;
                }
            }
        };
        // codeword (cw, L) of symbol s at stream index i, with its escape payload
        auto put_cw = [&](unsigned long long cw, int L, uint16_t s, unsigned long long i) {
            if (ew && s == 0) {
                // codeword and zigzag(k) in ew bits, in one emission when they fit 64 bits
                const unsigned long long z = zigzag(esc[i]);
                if (L + ew <= 64) {
                    cw = (cw << ew) | z;
                    L += ew;
                } else {
                    emit(cw, L);
                    cw = z;
                    L = ew;
                }
            }
            emit(cw, L);
        };
        if (regs) {
            for (int q = 0; q < (int)spl; q += 4) {
                // the loads of four symbols first, then their emissions
                uint16_t sv[4];
                unsigned long long cv[4];
                int lv[4];
#pragma unroll
                for (int u = 0; u < 4; u++) sv[u] = ss[q + u];
#pragma unroll
                for (int u = 0; u < 4; u++) cw_of(sv[u], cv[u], lv[u]);
#pragma unroll
                for (int u = 0; u < 4; u++) put_cw(cv[u], lv[u], sv[u], m0 + q + u);
            }
        } else {
            for (unsigned long long i = m0; i < m1; i++) {
                const uint16_t sv = a.sym[i];
                unsigned long long cw;
                int L;
                cw_of(sv, cw, L);
                put_cw(cw, L, sv, i);
            }
        }
        const uint32_t lastw = (uint32_t)(acc >> 32);
        const bool has_last = nacc > 0;
        // a full group whose every lane holds >= 32 bits (always true with 32
        // symbols per lane): lane i's last partial word is lane i+1's first word
        const bool full = __all_sync(0xffffffffu, (end - beg == G) && mb >= 32);
        if (full) {
            const uint32_t prev = __shfl_up_sync(0xffffffffu, lastw, 1);
            const bool sh = (start & 31) != 0;
            if (lane > 0 && sh) firstw |= prev;
            if (have_first) {
                if (lane == 0 && sh) atomicOr(&words[fidx], firstw);
                else words[fidx] = firstw;
            }
            if (lane == 31 && has_last) atomicOr(&words[widx], lastw);
        } else {
            if (have_first) {
                if (start & 31) atomicOr(&words[fidx], firstw);
                else words[fidx] = firstw;
            }
            if (has_last) atomicOr(&words[widx], lastw);
        }
    }
}


__device__ __forceinline__ void put32(uint8_t *p, uint32_t v) { for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i)); }
__device__ __forceinline__ void put64(uint8_t *p, unsigned long long v) { for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i)); }
__device__ __forceinline__ void putd(uint8_t *p, double v) { put64(p, (unsigned long long)__double_as_longlong(v)); }

__device__ __forceinline__ void header_body(const HeaderArgs &h, const uint8_t *len, Scalars *sc, uint8_t *out)
{
    __shared__ uint8_t hdr[128];
    __shared__ uint32_t crct[256];
    if (block_skip(&sc->status)) return;
    const unsigned long long nch = (h.N + h.K - 1) / h.K;
    Layout lay = container_layout(h.L, h.ncoord, sc->s_lo, sc->s_hi, nch, sc->total_bits);
    const unsigned long long n_esc = h.hist ? h.hist[0] : 0ULL;
    // CRC-32 (reflected, polynomial 0xEDB88320) by a byte table, one entry per thread
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        uint32_t c = (uint32_t)i;
        for (int b = 0; b < 8; b++) c = (c >> 1) ^ (0xEDB88320u & (0u - (c & 1u)));
        crct[i] = c;
    }
    for (int i = threadIdx.x; i < 128; i += blockDim.x) hdr[i] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        hdr[0] = 'H'; hdr[1] = 'P'; hdr[2] = 'D'; hdr[3] = 'R';
        put32(hdr + 4, 3);
        put32(hdr + 8, (uint32_t)h.dtype);
        put32(hdr + 12, (uint32_t)h.ndim);
        for (int k = 0; k < 3; k++) put64(hdr + 16 + 8 * k, h.dims[k]);
        put32(hdr + 40, (uint32_t)h.L);
        put32(hdr + 44, (uint32_t)h.mode);
        put32(hdr + 48, (uint32_t)h.tol_kind | (h.ncoord ? 0x100u : 0u));
        put32(hdr + 52, h.D);
        put32(hdr + 56, h.K);
        put32(hdr + 60, sc->s_lo);
        putd(hdr + 64, h.tol);
        putd(hdr + 72, sc->tau_abs);
        putd(hdr + 80, sc->maxabs);
        putd(hdr + 88, sqrt(sc->sumsq / (double)h.N));
        put64(hdr + 96, h.N);
        put64(hdr + 104, n_esc);
        sc->n_esc = n_esc;
        put64(hdr + 112, sc->total_bits);
        put32(hdr + 120, sc->s_hi | ((n_esc ? sc->esc_w : 0u) << 16));
        uint32_t c = 0xFFFFFFFFu;
        for (int i = 0; i < 124; i++) c = crct[(c ^ hdr[i]) & 0xFFu] ^ (c >> 8);
        put32(hdr + 124, c ^ 0xFFFFFFFFu);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 128; i += blockDim.x) out[i] = hdr[i];
    const unsigned long long qend = 128 + 8ULL * (h.L + 1);
    for (int l = threadIdx.x; l <= h.L; l += blockDim.x) putd(out + 128 + 8 * l, sc->q[l]);
    for (unsigned long long i = threadIdx.x; i < h.ncoord; i += blockDim.x) putd(out + qend + 8 * i, h.coords[i]);
    for (unsigned long long i = qend + 8 * h.ncoord + threadIdx.x; i < lay.off_len; i += blockDim.x) out[i] = 0;
    const unsigned nlen = sc->s_hi - sc->s_lo + 1;
    for (unsigned i = threadIdx.x; i < nlen; i += blockDim.x) out[lay.off_len + i] = len[sc->s_lo + i];
    for (unsigned long long i = lay.off_len + nlen + threadIdx.x; i < lay.off_chunk; i += blockDim.x) out[i] = 0;
    for (unsigned long long i = lay.off_chunk + 8 * nch + threadIdx.x; i < lay.off_bits; i += blockDim.x) out[i] = 0;
}

__global__ void __launch_bounds__(256)
header_kernel(HeaderArgs h, const uint8_t *len, Scalars *sc, uint8_t *out)
{
    header_body(h, len, sc, out);
}

// one container header per block, then the field's {bytes, status} pair
__global__ void __launch_bounds__(256) header_batch_kernel(const HeaderJob *jobs)
{
    const HeaderJob &j = jobs[blockIdx.x];
    header_body(j.h, j.len, j.sc, j.out);
    __syncthreads();
    if (threadIdx.x == 0 && j.size_status) {
        j.size_status[0] = j.sc->out_bytes;
        j.size_status[1] = j.sc->status;
    }
}

// ---------------------------------------------------------------------------
// Decoder: one thread per chunk, canonical decode with a two-level table and
// a per-length fallback for the longest codewords.
//
// A thread decodes its chunk of K symbols.  It keeps the next bits of the
// chunk MSB-aligned in two 32-bit registers hi:lo (nb valid bits, at least 32
// before every read) and refills them a word at a time from a queue of two
// prefetched 16-byte blocks.  A codeword of at most 13 bits is one load from
// the first-level table of every 13-bit prefix; one of up to 23 bits is a
// second load from the table its prefix names, indexed by the bits after the
// prefix; either gives symbol and length, with no search.  Every other case
// (longer codewords, prefixes past the second-level budget, escape payloads
// that do not fit the 32-bit window, invalid codes) leaves the loop for an
// out-of-line routine that reads its window from global memory, after which
// the queue restarts at the new position.
constexpr int kDecThreads = 1024;
// In a stream where escapes are dense, escaped codes are gathered per thread
// for eight symbols ([8][kDecThreads] slots) and written as whole 32-byte
// sectors: single 8-byte stores scattered over the escape array cost a
// read-modify-write of their sector in DRAM (rel 1e-4 on 513^3: 2.26 -> 1.20
// ms).  Sparse escapes are stored one by one (the gathering costs more than it
// saves below about one escape in sixteen symbols).
constexpr size_t kDecEscSmem = 8ull * 8 * kDecThreads;
constexpr size_t kDecSmem = (4u << kLutBits) + 4 * kSubCap + sizeof(LenTabs) + kDecEscSmem;

__device__ __forceinline__ uint32_t ldw(const uint32_t *w, unsigned long long i, unsigned long long n)
{
    return i < n ? __ldg(w + i) : 0u;
}

// four words from an aligned block index (words past n read as zero)
__device__ __forceinline__ uint4 ld4(const uint32_t *w, unsigned long long i, unsigned long long n)
{
    if (i + 4 <= n && ((reinterpret_cast<uintptr_t>(w) & 15) == 0))
        return __ldg(reinterpret_cast<const uint4 *>(w + i));
    uint4 v;
    v.x = ldw(w, i, n); v.y = ldw(w, i + 1, n); v.z = ldw(w, i + 2, n); v.w = ldw(w, i + 3, n);
    return v;
}

struct BitQueue {
    const uint32_t *w;
    unsigned long long n;     // words in the stream
    uint4 pa, pb;             // current and next aligned block
    unsigned k;               // next word of pa
    unsigned long long nxt;   // next block to fetch
    __device__ __forceinline__ uint32_t next()
    {
        const uint32_t v = k == 0 ? pa.x : k == 1 ? pa.y : k == 2 ? pa.z : pa.w;
        if (++k == 4) { k = 0; pa = pb; pb = ld4(w, nxt, n); nxt += 4; }
        return v;
    }
    // position the queue at bit pos and load the first 64 bits from there
    __device__ __forceinline__ void prime(unsigned long long pos, uint32_t &hi, uint32_t &lo, int &nb)
    {
        const unsigned long long wb0 = (pos >> 5) & ~3ULL;
        pa = ld4(w, wb0, n);
        pb = ld4(w, wb0 + 4, n);
        nxt = wb0 + 8;
        k = (unsigned)((pos >> 5) & 3);
        const uint32_t w0 = next(), w1 = next();
        const unsigned sh = (unsigned)(pos & 31);
        hi = __funnelshift_l(w1, w0, sh);
        lo = w1 << sh;
        nb = 64 - (int)sh;
    }
};

// 64 bits of the stream from bit pos (words past the end read as zero)
__device__ __forceinline__ unsigned long long window64(const uint32_t *w, unsigned long long n,
                                                       unsigned long long pos)
{
    const unsigned long long i = pos >> 5;
    const unsigned sh = (unsigned)(pos & 31);
    const unsigned long long hi = (((unsigned long long)ldw(w, i, n)) << 32) | ldw(w, i + 1, n);
    return sh ? (hi << sh) | (ldw(w, i + 2, n) >> (32 - sh)) : hi;
}

struct SlowOut {
    unsigned long long pos;
    uint32_t sv, bad;
};

// A step the table loop does not take: the entry e at pos is a long entry,
// invalid, or an escape whose payload does not fit the 32-bit window.
__device__ __noinline__ SlowOut decode_slow(uint32_t e, unsigned long long pos, const uint32_t *words,
                                            unsigned long long nwords, const LenTabs *T, const uint16_t *symtab,
                                            unsigned nsym, int ew, long long *esc_i)
{
    SlowOut o;
    o.bad = 0;
    const unsigned long long win = window64(words, nwords, pos);
    uint32_t sv = e & 0xFFFFu;
    unsigned L = (e >> 16) & 0x3Fu;
    if (e & kLongFlag) {
        const unsigned lmin = L, lmax = L + ((e >> 24) & 0x3Fu);
        L = code_len_in(*T, win, lmin, lmax);
        const unsigned long long off = (win >> (64 - L)) - T->first[L];
        if (off >= T->count[L]) o.bad = 1;
        const unsigned idx = T->start[L] + (unsigned)(off < T->count[L] ? off : 0);
        sv = symtab[idx < nsym ? idx : 0];
    } else if (e == 0) {
        o.bad = 1;               // no codeword starts here
        L = 1;
    }
    pos += L;
    if (ew && sv == 0) {
        // escape payload: zigzag(k) in ew bits
        const unsigned long long z = window64(words, nwords, pos) >> (64 - ew);
        pos += (unsigned)ew;
        *esc_i = unzigzag(z);
    }
    o.pos = pos;
    o.sv = sv;
    return o;
}

__global__ void __launch_bounds__(kDecThreads, 1) decode_kernel(DecodeArgs a_in, HuffScratch hs)
{
    DecodeArgs a = a_in;
    if (a.dh) {
        if (block_skip(hs.status)) return;
        const DevHdr h = *a.dh;
        a.words = reinterpret_cast<const uint32_t *>(a.base + h.off_bits);
        a.nwords = h.nwords;
        a.chunk = reinterpret_cast<const unsigned long long *>(a.base + h.off_chunk);
        a.total_bits = h.total_bits;
        a.esc_w = h.esc_w;
        a.n_esc = h.n_esc;
        if (h.esc_w == 0) a.esc = nullptr;
    }
    extern __shared__ __align__(16) unsigned char dsm[];
    uint32_t *lut = reinterpret_cast<uint32_t *>(dsm);                       // [1 << kLutBits]
    uint32_t *sub = lut + (1u << kLutBits);                                   // [kSubCap]
    LenTabs *T = reinterpret_cast<LenTabs *>(sub + kSubCap);
    long long *escbuf = reinterpret_cast<long long *>(T + 1);                  // [8][kDecThreads]
    if (block_skip(hs.status)) return;
    const unsigned nsym = *hs.nsym;
    const unsigned nsub = *hs.nsub < kSubCap ? *hs.nsub : kSubCap;
    {
        // escape entries take their payload width into their length when both fit 32 bits
        const unsigned ewc = a.esc ? a.esc_w : 0u;
        auto fold = [&](uint32_t e) -> uint32_t {
            if (ewc && e && !(e & (kLongFlag | kSubFlag)) && (e & 0xFFFFu) == 0) {
                const unsigned L = (e >> 16) & 0x3Fu;
                if (L + ewc <= 32) e = kEscFolded | ((L + ewc) << 16);
            }
            return e;
        };
        for (int i = threadIdx.x; i < (1 << kLutBits); i += blockDim.x) lut[i] = fold(hs.lut1[i]);
        for (unsigned i = threadIdx.x; i < nsub; i += blockDim.x) sub[i] = fold(hs.lut_sub[i]);
    }
    if (threadIdx.x < 64) {
        T->first[threadIdx.x] = hs.first[threadIdx.x];
        T->lim[threadIdx.x] = hs.lim[threadIdx.x];
        T->start[threadIdx.x] = hs.start[threadIdx.x];
        T->count[threadIdx.x] = hs.count[threadIdx.x];
    }
    __syncthreads();
    const uint16_t *symtab = hs.sorted_sym;
    long long *const esc = a.esc;
    const int ew = esc ? (int)a.esc_w : 0;     // escape payload width (1..63)
    const bool gather = ew && a.n_esc * 16 > a.N;
    const unsigned long long nch = (a.N + a.K - 1) / a.K;
    // chunks interleave over the blocks so that every SM gets a share
    for (unsigned long long c = blockIdx.x + (unsigned long long)gridDim.x * threadIdx.x; c < nch;
         c += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long pos0 = a.chunk[c];
        const unsigned long long expect = (c + 1 < nch) ? a.chunk[c + 1] : a.total_bits;
        if (pos0 > a.total_bits || expect > a.total_bits || pos0 > expect) {
            atomicExch(hs.status, (unsigned)DS_FORMAT);
            continue;
        }
        BitQueue q;
        q.w = a.words;
        q.n = a.nwords;
        uint32_t hi, lo;
        int nb;
        q.prime(pos0, hi, lo, nb);
        unsigned long long used = 0;
        bool bad = false;
        // this thread's escaped codes of the current group of eight symbols:
        // slot j of the group at escbuf[j * kDecThreads + tid], bit j of emask
        long long *const eslot = escbuf + threadIdx.x;
        unsigned emask = 0;
        auto step = [&](unsigned long long i) -> uint16_t {
            uint32_t e = lut[hi >> (32 - kLutBits)];
            // a codeword of up to 23 bits: its second-level entry, indexed by
            // the bits after the prefix (all within hi, nb >= 32)
            if ((e & (kLongFlag | kSubFlag)) == kSubFlag)
                e = sub[(e & 0xFFFFu) + ((hi << kLutBits) >> (32 - ((e >> 16) & 0xFu)))];
            const uint32_t sv = e & 0xFFFFu;
            const unsigned L = (e >> 16) & 0x3Fu;
            const bool at_esc = ew && sv == 0;
            if ((e & kLongFlag) || e == 0 || (at_esc && !(e & kEscFolded))) {
                const unsigned j = (unsigned)(i & 7);
                const SlowOut o = decode_slow(e, pos0 + used, a.words, a.nwords, T, symtab, nsym, ew,
                                              !esc ? nullptr : gather ? eslot + (size_t)j * kDecThreads : esc + i);
                if (gather && o.sv == 0) emask |= 1u << j;
                bad |= o.bad != 0;
                used = o.pos - pos0;
                q.prime(o.pos, hi, lo, nb);
                return (uint16_t)o.sv;
            }
            // folded escape: codeword of L - ew bits, then zigzag(k) in ew bits
            if (at_esc) {
                const long long kv = unzigzag((unsigned long long)((hi << (L - ew)) >> (32 - ew)));
                if (gather) {
                    const unsigned j = (unsigned)(i & 7);
                    eslot[(size_t)j * kDecThreads] = kv;
                    emask |= 1u << j;
                } else {
                    esc[i] = kv;
                }
            }
            // drop L <= 32 bits, then refill to at least 32 valid bits: the
            // word is selected and merged by predication; only the block
            // load (every fourth refill) branches
            hi = L < 32 ? __funnelshift_l(lo, hi, L) : lo;
            lo = L < 32 ? lo << L : 0u;
            nb -= (int)L;
            used += L;
            {
                const bool need = nb < 32;
                const uint32_t wv = q.k == 0 ? q.pa.x : q.k == 1 ? q.pa.y : q.k == 2 ? q.pa.z : q.pa.w;
                const unsigned sh = need ? (unsigned)nb : 0u;
                hi = need ? (hi | (wv >> sh)) : hi;
                lo = need ? __funnelshift_rc(0u, wv, sh) : lo;
                nb += need ? 32 : 0;
                q.k += need ? 1u : 0u;
                if (q.k == 4) { q.k = 0; q.pa = q.pb; q.pb = ld4(q.w, q.nxt, q.n); q.nxt += 4; }
            }
            return (uint16_t)sv;
        };
        // the escaped codes of the group at i0 (a multiple of 8): each half
        // with an escape as one 32-byte store (the other slots carry stale
        // values, and nothing reads the escape array where no escape is)
        auto flush8 = [&](unsigned long long i0) {
            for (int h = 0; h < 2; h++) {
                if (!((emask >> (4 * h)) & 0xFu)) continue;
                const long long *src = eslot + (size_t)(4 * h) * kDecThreads;
                longlong2 *dst = reinterpret_cast<longlong2 *>(esc + i0 + 4 * h);
                dst[0] = make_longlong2(src[0], src[kDecThreads]);
                dst[1] = make_longlong2(src[2 * kDecThreads], src[3 * kDecThreads]);
            }
            emask = 0;
        };
        const unsigned long long beg = c * a.K;
        const unsigned long long end = beg + a.K < a.N ? beg + a.K : a.N;
        unsigned long long i = beg;
        // eight symbols per 16-byte store (K is a multiple of 128)
        for (; i + 8 <= end; i += 8) {
            uint4 o;
            o.x = (uint32_t)step(i) | ((uint32_t)step(i + 1) << 16);
            o.y = (uint32_t)step(i + 2) | ((uint32_t)step(i + 3) << 16);
            o.z = (uint32_t)step(i + 4) | ((uint32_t)step(i + 5) << 16);
            o.w = (uint32_t)step(i + 6) | ((uint32_t)step(i + 7) << 16);
            // streaming store: the symbols are written once and read by the next
            // kernel, so they should not push the bitstream out of L2
            __stcs(reinterpret_cast<uint4 *>(a.sym + i), o);
            if (emask) flush8(i);
        }
        // a last group of fewer than eight: its escapes one by one
        const unsigned long long i0 = i;
        for (; i < end; i++) a.sym[i] = step(i);
        for (unsigned j = 0; emask; j++, emask >>= 1)
            if (emask & 1u) esc[i0 + j] = eslot[(size_t)j * kDecThreads];
        if (bad || pos0 + used != expect) atomicExch(hs.status, (unsigned)DS_FORMAT);
    }
}

__global__ void __launch_bounds__(256)
hist_kernel(const uint16_t *sym, unsigned long long N, unsigned D, unsigned long long *hist,
            unsigned *status)
{
    extern __shared__ unsigned hsm[];
    const bool sm = D <= 16384;
    if (sm) for (unsigned i = threadIdx.x; i < D; i += blockDim.x) hsm[i] = 0;
    __syncthreads();
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < N;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        unsigned s = sym[i];
        if (s >= D) { atomicExch(status, (unsigned)DS_ARG); continue; }
        if (sm) atomicAdd(&hsm[s], 1u); else atomicAdd(&hist[s], 1ULL);
    }
    __syncthreads();
    if (sm)
        for (unsigned i = threadIdx.x; i < D; i += blockDim.x)
            if (hsm[i]) atomicAdd(&hist[i], (unsigned long long)hsm[i]);
}

// Histogram of an alphabet above 16384 symbols (up to 65536): two 16-bit
// counters per 32-bit shared word, 128 KB.  A block counts at most 32768 keys
// per round, so no counter carries into its neighbour, then adds the nonzero
// counts to the global histogram and clears its words.
constexpr int kHistWideThreads = 1024;
constexpr unsigned kHistWideRound = 32u * kHistWideThreads;
__global__ void __launch_bounds__(kHistWideThreads, 1)
hist_wide_kernel(const uint16_t *sym, unsigned long long N, unsigned D, unsigned long long *hist, unsigned *status)
{
    extern __shared__ unsigned hw[];
    const unsigned nw = (D + 1) / 2;
    for (unsigned i = threadIdx.x; i < nw; i += blockDim.x) hw[i] = 0;
    __syncthreads();
    for (unsigned long long r0 = blockIdx.x * (unsigned long long)kHistWideRound; r0 < N;
         r0 += (unsigned long long)gridDim.x * kHistWideRound) {
        const unsigned long long r1 = r0 + kHistWideRound < N ? r0 + kHistWideRound : N;
        if (r1 - r0 == kHistWideRound && ((uintptr_t)(sym + r0) & 15) == 0) {
            // a full round: four 16-byte loads (32 keys) per thread
            const uint4 *v = reinterpret_cast<const uint4 *>(sym + r0);
            uint4 x[4];
#pragma unroll
            for (int u = 0; u < 4; u++) x[u] = v[threadIdx.x + u * kHistWideThreads];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const unsigned w4[4] = {x[u].x, x[u].y, x[u].z, x[u].w};
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const unsigned s = (w4[q >> 1] >> (16 * (q & 1))) & 0xFFFFu;
                    if (s >= D) { atomicExch(status, (unsigned)DS_ARG); continue; }
                    atomicAdd(&hw[s >> 1], (s & 1) ? 0x10000u : 1u);
                }
            }
        } else {
            for (unsigned long long i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
                const unsigned s = sym[i];
                if (s >= D) { atomicExch(status, (unsigned)DS_ARG); continue; }
                atomicAdd(&hw[s >> 1], (s & 1) ? 0x10000u : 1u);
            }
        }
        __syncthreads();
        for (unsigned i = threadIdx.x; i < nw; i += blockDim.x) {
            const unsigned w = hw[i];
            if (w) {
                if (w & 0xFFFFu) atomicAdd(&hist[2 * i], (unsigned long long)(w & 0xFFFFu));
                if (w >> 16) atomicAdd(&hist[2 * i + 1], (unsigned long long)(w >> 16));
                hw[i] = 0;
            }
        }
        __syncthreads();
    }
}

PerDeviceOnce g_attr_done;
cudaError_t set_attrs_now()
{
    cudaError_t e = cudaFuncSetAttribute(rank_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmemKeys * 8);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemKeys * 16);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(codebook_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCodebookSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(codebook_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kCodebookSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(dec_tables_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 4 * 32 * kWcStride + 65536);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(enc_write_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(enc_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDecSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(lut_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLutSmem);
    return e;
}
cudaError_t set_attrs() { return once_per_device(g_attr_done, set_attrs_now); }

}  // namespace

size_t huff_scratch_bytes(unsigned int D)
{
    size_t d = D;
    size_t b = 0;
    auto add = [&](size_t x) { b += (x + 255) & ~size_t(255); };
    add(8 * d); add(8 * d); add(8 * d); add(4 * d);    // keys, keys2, sorted, rank
    add(4 * 2 * d); add(4 * 4 * d); add(4 * 4 * d);    // parent, anc, dep
    add(8 * d); add(8 * d);                            // leafw, intw
    add(4); add(8 * 64); add(4 * 64); add(4 * 64);     // nsym, first, count, start
    add(d); add(8 * d); add(2 * d); add(4u << kLutBits);
    add(8 * 64);
    add(4 * kSubCap); add(4);
    return b;
}

void huff_scratch_carve(void *base, unsigned int D, Scalars *sc, HuffScratch *hs)
{
    char *p = (char *)base;
    size_t d = D;
    auto take = [&](size_t x) { char *r = p; p += (x + 255) & ~size_t(255); return (void *)r; };
    hs->keys = (unsigned long long *)take(8 * d);
    hs->keys2 = (unsigned long long *)take(8 * d);
    hs->sorted = (unsigned long long *)take(8 * d);
    hs->rank = (unsigned *)take(4 * d);
    hs->parent = (unsigned *)take(4 * 2 * d);
    hs->anc = (unsigned *)take(4 * 4 * d);
    hs->dep = (unsigned *)take(4 * 4 * d);
    hs->leafw = (unsigned long long *)take(8 * d);
    hs->intw = (unsigned long long *)take(8 * d);
    hs->nsym = (unsigned *)take(4);
    hs->first = (unsigned long long *)take(8 * 64);
    hs->count = (unsigned *)take(4 * 64);
    hs->start = (unsigned *)take(4 * 64);
    hs->len = (uint8_t *)take(d);
    hs->code = (unsigned long long *)take(8 * d);
    hs->sorted_sym = (uint16_t *)take(2 * d);
    hs->lut1 = (uint32_t *)take(4u << kLutBits);
    hs->lim = (unsigned long long *)take(8 * 64);
    hs->lut_sub = (uint32_t *)take(4 * kSubCap);
    hs->nsub = (unsigned *)take(4);
    hs->status = &sc->status;
    hs->s_lo = &sc->s_lo;
    hs->s_hi = &sc->s_hi;
}

cudaError_t launch_codebook(const unsigned long long *hist, unsigned int D, const HuffScratch &hs,
                            cudaStream_t s)
{
    cudaError_t e = set_attrs();
    if (e != cudaSuccess) return e;
    if (D <= kFusedMaxD) {
        codebook_kernel<<<1, 1024, kCodebookSmem, s>>>(hist, D, hs);
        count_launch();
        return cudaGetLastError();
    }
    compact_kernel<<<1, 1024, 0, s>>>(hist, nullptr, D, hs.keys, hs.nsym, hs.s_lo, hs.s_hi);
    rank_kernel<<<kRankBlocks, 256, kSmemKeys * 8, s>>>(hs.keys, hs.nsym, hs.sorted, nullptr);
    merge_kernel<<<1, 1024, kSmemKeys * 16, s>>>(hs, D);
    rank_kernel<<<kRankBlocks, 256, kSmemKeys * 8, s>>>(hs.keys2, hs.nsym, nullptr, hs.rank);
    assign_kernel<<<64, 256, 0, s>>>(hs);
    count_launch(5);
    return cudaGetLastError();
}

cudaError_t launch_decode_tables(const uint8_t *lenb, unsigned int s_lo, unsigned int s_hi, unsigned int D,
                                 const HuffScratch &hs, cudaStream_t s)
{
    cudaError_t e = set_attrs();
    if (e != cudaSuccess) return e;
    dec_tables_kernel<<<1, 1024, 4 * 32 * kWcStride + D, s>>>(lenb, s_lo, s_hi, D, hs, nullptr, nullptr);
    lut_kernel<<<1, kLutThreads, kLutSmem, s>>>(hs);
    count_launch(2);
    return cudaGetLastError();
}

cudaError_t launch_decode_tables_dev(const uint8_t *base, const DevHdr *dh, unsigned int D, const HuffScratch &hs,
                                     cudaStream_t s)
{
    cudaError_t e = set_attrs();
    if (e != cudaSuccess) return e;
    dec_tables_kernel<<<1, 1024, 4 * 32 * kWcStride + D, s>>>(nullptr, 0u, 0u, D, hs, base, dh);
    lut_kernel<<<1, kLutThreads, kLutSmem, s>>>(hs);
    count_launch(2);
    return cudaGetLastError();
}

cudaError_t launch_encode(const EncodeArgs &a, cudaStream_t s)
{
    cudaError_t e = set_attrs();
    if (e != cudaSuccess) return e;
    enc_count_kernel<<<kEncBlocks, 256, a.D, s>>>(a);
    enc_scan1_kernel<<<1, 1024, 0, s>>>(a, kEncBlocks);
    enc_scan2_kernel<<<kEncBlocks, 256, 0, s>>>(a);
    const bool code_sm = a.D <= (unsigned)kSmemCodes;
    const size_t sm = (code_sm ? 4 * (size_t)a.D : 0) + 8 * 32 * 17 * 4;
    int per_sm = 0, nsm = 0, dev = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, enc_write_kernel, 256, sm) != cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 3;
        nsm = 152;
    }
    enc_write_kernel<<<(unsigned)(nsm * std::max(1, per_sm)), 256, sm, s>>>(a);
    count_launch(4);
    return cudaGetLastError();
}

cudaError_t launch_header(const HeaderArgs &h, const uint8_t *len, Scalars *sc, uint8_t *container,
                          cudaStream_t s)
{
    header_kernel<<<1, 256, 0, s>>>(h, len, sc, container);
    count_launch();
    return cudaGetLastError();
}

bool codebook_fused(unsigned int D) { return D <= kFusedMaxD; }

cudaError_t launch_codebook_batch(const CodebookJob *jobs, int n, cudaStream_t s)
{
    cudaError_t e = set_attrs();
    if (e != cudaSuccess) return e;
    if (n < 1) return cudaSuccess;
    codebook_batch_kernel<<<n, 1024, kCodebookSmem, s>>>(jobs);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_header_batch(const HeaderJob *jobs, int n, cudaStream_t s)
{
    if (n < 1) return cudaSuccess;
    header_batch_kernel<<<n, 256, 0, s>>>(jobs);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_histogram(const uint16_t *sym, unsigned long long N, unsigned D,
                             unsigned long long *hist, unsigned *status, cudaStream_t s)
{
    static PerDeviceOnce attr;
    cudaError_t ea = once_per_device(attr, [] {
        cudaError_t e = cudaFuncSetAttribute(hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(hist_wide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536 * 2);
        return e;
    });
    if (ea != cudaSuccess) return ea;
    if (D <= 16384) {
        hist_kernel<<<152 * 4, 256, D * 4, s>>>(sym, N, D, hist, status);
    } else {
        int dev = 0, nsm = 152;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            nsm = 152;
        }
        const unsigned long long rounds = (N + kHistWideRound - 1) / kHistWideRound;
        const unsigned grid = (unsigned)(rounds < (unsigned long long)nsm ? rounds : (unsigned long long)nsm);
        hist_wide_kernel<<<grid, kHistWideThreads, ((D + 1) / 2) * 4, s>>>(sym, N, D, hist, status);
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_decode(const DecodeArgs &a, const HuffScratch &hs, cudaStream_t s)
{
    cudaError_t e = set_attrs();
    if (e != cudaSuccess) return e;
    decode_kernel<<<sm_count(), kDecThreads, kDecSmem, s>>>(a, hs);
    count_launch();
    return cudaGetLastError();
}

}  // namespace hpdr
