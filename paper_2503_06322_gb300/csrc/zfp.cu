// zfp.cu -- fixed-rate ZFP compression (Alg. 3, Sec. IV-C) on the GPU.
//
// The paper's outline: the field is cut into blocks of 4^d values, each
// block aligned to its largest exponent and made fixed point, decorrelated by
// a near-orthogonal transform, and its bit planes serialized most significant
// first and cut at a fixed number of bits.  Every block's output has the same
// size, so blocks need no coordination: one thread codes one block, with the
// block held in registers (all loops over the 4^d values unrolled) and its
// bits written straight to its own words.
//
// The details the paper leaves open are read as follows (the container, a
// 64-byte header and the block words, is documented with hpdr_zfp_compress
// in include/hpdr.h):
//   blocks      row-major over ceil(n_k / 4) blocks per dimension, values in
//               a block row-major (last index fastest); positions past the
//               array edge repeat the last in-range value of their dimension,
//               and are dropped on decoding.
//   exponent    emax = the binary exponent e of the block's largest magnitude
//               (x = f 2^e, 1/2 <= |f| < 1); a block of zeros codes a 0 flag.
//   fixed point q = trunc(x 2^(P - 5 - emax)), P = 32 (f32) or 64 (f64).
//   transform   along the last dimension, then the others in reverse order,
//               every line (a0..a3) becomes (S, D, d0, d1):
//                 s0 = floor((a0 + a1)/2), d0 = a0 - a1, s1 = floor((a2 + a3)/2),
//                 d1 = a2 - a3, S = floor((s0 + s1)/2), D = s0 - s1,
//               an exactly invertible integer S-transform (two Haar levels);
//               magnitudes stay below 2^(P-2) after three dimensions.
//   order       by the sum over dimensions of the class of the index within
//               the line (S 0, D 1, d0 and d1 2), ties in block order.
//   negabinary  u = (q + 0xAA..A) xor 0xAA..A in P-bit arithmetic.
//   coding      rate * 4^d bits per block (a multiple of 32): a flag bit,
//               EB = 9 (f32) or 12 (f64) exponent bits (emax + 2^(EB-1),
//               least significant first), then planes P-1..0: the bits of the
//               n coefficients already significant as they are, then group
//               tests (one bit: any of n.. set; after a 1 the coefficients'
//               bits from n up to and including the next 1); the block stops
//               where its budget ends, the rest of its bits zero.  Bits fill
//               32-bit words least significant first.
#include <cstdint>
#include <cstring>
#include <cmath>
#include "internal.cuh"

namespace hpdr {
namespace {

constexpr int kZfpThreads = 128;
constexpr int kZfpHdr = 64;

struct ZfpGeom {
    long long n[3];             // dims (row-major, last fastest), unused = 1
    long long nb[3];            // blocks per dim
    unsigned long long nblocks;
    uint32_t maxbits;           // bits per block
};

struct ZfpHdrBytes {
    uint8_t b[kZfpHdr];
};

// sequency order of a block of 4^D coefficients, built at compile time
template <int D>
struct SeqOrder {
    unsigned char p[64];
    constexpr SeqOrder() : p{}
    {
        int key[64] = {};
        const int cls[4] = {0, 1, 2, 2};
        const int B = 1 << (2 * D);
        for (int i = 0; i < B; i++) {
            int s = 0, r = i;
            for (int k = 0; k < D; k++) { s += cls[r % 4]; r /= 4; }
            key[i] = s;
        }
        int m = 0;
        for (int s = 0; s <= 2 * D; s++)
            for (int i = 0; i < B; i++)
                if (key[i] == s) p[m++] = (unsigned char)i;
    }
};

template <typename T> struct ZfpTypes;
template <> struct ZfpTypes<float> {
    typedef int32_t SI;
    typedef uint32_t UI;
    static constexpr int P = 32, EB = 9;
    static constexpr uint32_t M = 0xAAAAAAAAu;
};
template <> struct ZfpTypes<double> {
    typedef long long SI;
    typedef unsigned long long UI;
    static constexpr int P = 64, EB = 12;
    static constexpr unsigned long long M = 0xAAAAAAAAAAAAAAAAull;
};

// one line of the forward / inverse transform (arithmetic shifts = floor)
template <typename SI>
__device__ __forceinline__ void fwd_line(SI &a0, SI &a1, SI &a2, SI &a3)
{
    const SI s0 = (a0 + a1) >> 1, d0 = a0 - a1;
    const SI s1 = (a2 + a3) >> 1, d1 = a2 - a3;
    a0 = (s0 + s1) >> 1;
    a1 = s0 - s1;
    a2 = d0;
    a3 = d1;
}
// (s, d) -> (x, y): x + y = 2s + (d & 1), x - y = d; d + (d & 1) is even
template <typename SI>
__device__ __forceinline__ void inv_pair(SI s, SI d, SI &x, SI &y)
{
    x = s + ((d + (d & 1)) >> 1);
    y = x - d;
}
template <typename SI>
__device__ __forceinline__ void inv_line(SI &a0, SI &a1, SI &a2, SI &a3)
{
    SI s0, s1, x0, x1, x2, x3;
    inv_pair(a0, a1, s0, s1);
    inv_pair(s0, a2, x0, x1);
    inv_pair(s1, a3, x2, x3);
    a0 = x0; a1 = x1; a2 = x2; a3 = x3;
}

template <int D, typename SI>
__device__ __forceinline__ void fwd_block(SI *q)
{
    constexpr int B = 1 << (2 * D);
#pragma unroll
    for (int k = D - 1; k >= 0; k--) {
        const int st = 1 << (2 * (D - 1 - k));
#pragma unroll
        for (int i = 0; i < B; i++)
            if (((i / st) & 3) == 0) fwd_line(q[i], q[i + st], q[i + 2 * st], q[i + 3 * st]);
    }
}
template <int D, typename SI>
__device__ __forceinline__ void inv_block(SI *q)
{
    constexpr int B = 1 << (2 * D);
#pragma unroll
    for (int k = 0; k < D; k++) {
        const int st = 1 << (2 * (D - 1 - k));
#pragma unroll
        for (int i = 0; i < B; i++)
            if (((i / st) & 3) == 0) inv_line(q[i], q[i + st], q[i + 2 * st], q[i + 3 * st]);
    }
}

// element offsets of the block's 4 positions along every dimension (edge
// positions clamped), so that value i sits at the sum of its D offsets
template <int D>
__device__ __forceinline__ void block_offsets(const ZfpGeom &g, unsigned long long b, long long off[3][4],
                                              bool inside[3][4])
{
    long long bi[3] = {0, 0, 0};
    unsigned long long r = b;
#pragma unroll
    for (int k = D - 1; k >= 0; k--) {
        bi[k] = (long long)(r % (unsigned long long)g.nb[k]);
        r /= (unsigned long long)g.nb[k];
    }
    long long stride = 1;
#pragma unroll
    for (int k = D - 1; k >= 0; k--) {
#pragma unroll
        for (int j = 0; j < 4; j++) {
            long long p = 4 * bi[k] + j;
            inside[k][j] = p < g.n[k];
            if (p > g.n[k] - 1) p = g.n[k] - 1;
            off[k][j] = p * stride;
        }
        stride *= g.n[k];
    }
}

template <int D>
__device__ __forceinline__ long long value_offset(const long long off[3][4], int i)
{
    long long o = 0;
#pragma unroll
    for (int k = 0; k < D; k++) o += off[k][(i >> (2 * (D - 1 - k))) & 3];
    return o;
}
template <int D>
__device__ __forceinline__ bool value_inside(const bool in[3][4], int i)
{
    bool ok = true;
#pragma unroll
    for (int k = 0; k < D; k++) ok = ok && in[k][(i >> (2 * (D - 1 - k))) & 3];
    return ok;
}

// bits of one block, least significant first, clipped at the block's budget
struct BitWriter {
    uint32_t *w;
    unsigned idx = 0;                 // next word
    unsigned long long acc = 0;       // pending bits
    int nacc = 0;
    uint32_t left;                    // budget left
    __device__ BitWriter(uint32_t *words, uint32_t budget) : w(words), left(budget) {}
    // append the low `cnt` bits of v (cnt <= 32); false once the budget is spent
    __device__ __forceinline__ bool put(uint32_t v, int cnt)
    {
        if (cnt > (int)left) cnt = (int)left;
        if (cnt > 0) {
            const uint32_t m = cnt == 32 ? 0xFFFFFFFFu : ((1u << cnt) - 1u);
            acc |= (unsigned long long)(v & m) << nacc;
            nacc += cnt;
            left -= (uint32_t)cnt;
            if (nacc >= 32) {
                w[idx++] = (uint32_t)acc;
                acc >>= 32;
                nacc -= 32;
            }
        }
        return left > 0;
    }
    __device__ __forceinline__ bool put64(unsigned long long v, int cnt)
    {
        if (cnt > 32) {
            if (!put((uint32_t)v, 32)) return false;
            return put((uint32_t)(v >> 32), cnt - 32);
        }
        return put((uint32_t)v, cnt);
    }
    // zero runs of any length
    __device__ __forceinline__ bool zeros(int cnt)
    {
        while (cnt > 0) {
            const int c = cnt > 32 ? 32 : cnt;
            if (!put(0u, c)) return false;
            cnt -= c;
        }
        return left > 0;
    }
    // write the pending bits and zero the block's remaining words
    __device__ __forceinline__ void finish(unsigned nwords)
    {
        if (nacc > 0) { w[idx++] = (uint32_t)acc; acc = 0; nacc = 0; }
        while (idx < nwords) w[idx++] = 0u;
    }
};

struct BitReader {
    const uint32_t *w;
    unsigned idx = 0;
    unsigned long long buf = 0;
    int nbuf = 0;
    uint32_t left;
    __device__ BitReader(const uint32_t *words, uint32_t budget) : w(words), left(budget) {}
    // the next min(cnt, left) bits (cnt <= 32) into *v; returns how many were read
    __device__ __forceinline__ int get(int cnt, uint32_t *v)
    {
        if (cnt > (int)left) cnt = (int)left;
        if (cnt <= 0) { *v = 0; return 0; }
        if (nbuf < cnt) {
            buf |= (unsigned long long)w[idx++] << nbuf;
            nbuf += 32;
        }
        const uint32_t m = cnt == 32 ? 0xFFFFFFFFu : ((1u << cnt) - 1u);
        *v = (uint32_t)buf & m;
        buf >>= cnt;
        nbuf -= cnt;
        left -= (uint32_t)cnt;
        return cnt;
    }
    // the next cnt bits (cnt <= min(32, left)) without consuming them
    __device__ __forceinline__ uint32_t peek(int cnt)
    {
        if (nbuf < cnt) {
            buf |= (unsigned long long)w[idx++] << nbuf;
            nbuf += 32;
        }
        return (uint32_t)buf & (cnt == 32 ? 0xFFFFFFFFu : ((1u << cnt) - 1u));
    }
    __device__ __forceinline__ void skip(int cnt)
    {
        buf >>= cnt;
        nbuf -= cnt;
        left -= (uint32_t)cnt;
    }
};

template <typename T, int D>
__global__ void __launch_bounds__(kZfpThreads) zfp_encode_kernel(const T *__restrict__ u, uint32_t *__restrict__ out,
                                                                 ZfpGeom g)
{
    typedef ZfpTypes<T> Z;
    typedef typename Z::SI SI;
    typedef typename Z::UI UI;
    constexpr int B = 1 << (2 * D), P = Z::P, EB = Z::EB;
    constexpr SeqOrder<D> ord{};
    const unsigned long long b = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    if (b >= g.nblocks) return;
    long long off[3][4];
    bool inside[3][4];
    block_offsets<D>(g, b, off, inside);
    T v[B];
    T mx = (T)0;
#pragma unroll
    for (int i = 0; i < B; i++) {
        v[i] = u[value_offset<D>(off, i)];
        const T a = v[i] < (T)0 ? -v[i] : v[i];
        mx = a > mx ? a : mx;
    }
    const unsigned nwords = g.maxbits / 32;
    BitWriter bw(out + b * nwords, g.maxbits);
    if (!(mx > (T)0)) {
        bw.put(0u, 1);
        bw.finish(nwords);
        return;
    }
    int emax;
    frexp((double)mx, &emax);
    bw.put(1u, 1);
    bw.put((uint32_t)(emax + (1 << (EB - 1))), EB);
    SI q[B];
#pragma unroll
    for (int i = 0; i < B; i++) q[i] = (SI)__double2ll_rz(ldexp((double)v[i], P - 5 - emax));
    fwd_block<D>(q);
    UI w[B];
    UI any = 0;
#pragma unroll
    for (int r = 0; r < B; r++) {
        w[r] = ((UI)q[ord.p[r]] + (UI)Z::M) ^ (UI)Z::M;
        any |= w[r];
    }
    int n = 0;
    for (int k = P - 1; k >= 0; k--) {
        unsigned long long mask = 0;
        if ((any >> k) & 1) {
#pragma unroll
            for (int r = 0; r < B; r++) mask |= (unsigned long long)((w[r] >> k) & 1) << r;
        }
        // the coefficients already significant, as they are
        if (n > 0 && !bw.put64(n == 64 ? mask : (mask & ((1ull << n) - 1ull)), n)) break;
        bool more = true;
        while (n < B) {
            const unsigned long long rest = mask >> n;   // n < B <= 64
            if (!rest) { more = bw.put(0u, 1); break; }
            const int j = __ffsll((long long)rest) - 1;
            // test bit 1, then j zeros and the coefficient's 1
            if (!bw.put(1u, 1) || !bw.zeros(j) || !bw.put(1u, 1)) { more = false; break; }
            n += j + 1;
        }
        if (!more || bw.left == 0) break;
    }
    bw.finish(nwords);
}

template <typename T, int D>
__global__ void __launch_bounds__(kZfpThreads) zfp_decode_kernel(const uint32_t *__restrict__ in, T *__restrict__ u,
                                                                 ZfpGeom g)
{
    typedef ZfpTypes<T> Z;
    typedef typename Z::SI SI;
    typedef typename Z::UI UI;
    constexpr int B = 1 << (2 * D), P = Z::P, EB = Z::EB;
    constexpr SeqOrder<D> ord{};
    const unsigned long long b = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    if (b >= g.nblocks) return;
    long long off[3][4];
    bool inside[3][4];
    block_offsets<D>(g, b, off, inside);
    const unsigned nwords = g.maxbits / 32;
    BitReader br(in + b * nwords, g.maxbits);
    uint32_t flag = 0;
    br.get(1, &flag);
    T val[B];
    if (!flag) {
#pragma unroll
        for (int i = 0; i < B; i++) val[i] = (T)0;
    } else {
        uint32_t eb = 0;
        br.get(EB, &eb);
        const int emax = (int)eb - (1 << (EB - 1));
        UI w[B];
#pragma unroll
        for (int r = 0; r < B; r++) w[r] = 0;
        int n = 0;
        bool more = true;
        for (int k = P - 1; k >= 0 && more; k--) {
            unsigned long long mask = 0;
            // verbatim bits of coefficients 0..n-1
            int got = 0;
            while (got < n) {
                const int c = n - got > 32 ? 32 : n - got;
                uint32_t x;
                const int r = br.get(c, &x);
                mask |= (unsigned long long)x << got;
                got += r;
                if (r < c) { more = false; break; }
            }
            while (more && n < B) {
                uint32_t t;
                if (br.get(1, &t) == 0) { more = false; break; }
                if (!t) break;
                // scan to the next 1, up to 32 bits at a time (a malformed
                // stream may run out at B)
                while (n < B) {
                    int avail = B - n < 32 ? B - n : 32;
                    if (avail > (int)br.left) avail = (int)br.left;
                    if (avail == 0) { more = false; break; }
                    const uint32_t x = br.peek(avail);
                    if (!x) {
                        br.skip(avail);
                        n += avail;
                        continue;
                    }
                    const int j = __ffs((int)x) - 1;
                    br.skip(j + 1);
                    n += j + 1;
                    mask |= 1ull << (n - 1);
                    break;
                }
            }
            if (mask) {
#pragma unroll
                for (int r = 0; r < B; r++) w[r] |= (UI)((mask >> r) & 1ull) << k;
            }
        }
        SI q[B];
#pragma unroll
        for (int r = 0; r < B; r++) q[ord.p[r]] = (SI)((w[r] ^ (UI)Z::M) - (UI)Z::M);
        inv_block<D>(q);
#pragma unroll
        for (int i = 0; i < B; i++) val[i] = (T)ldexp((double)q[i], emax - (P - 5));
    }
#pragma unroll
    for (int i = 0; i < B; i++)
        if (value_inside<D>(inside, i)) u[value_offset<D>(off, i)] = val[i];
}

__global__ void zfp_header_kernel(uint8_t *out, ZfpHdrBytes h)
{
    for (int i = threadIdx.x; i < kZfpHdr; i += blockDim.x) out[i] = h.b[i];
}

uint32_t zfp_crc32(const uint8_t *p, int n)
{
    uint32_t c = 0xFFFFFFFFu;
    for (int i = 0; i < n; i++) {
        c ^= p[i];
        for (int k = 0; k < 8; k++) c = (c >> 1) ^ (0xEDB88320u & (0u - (c & 1u)));
    }
    return ~c;
}

void zput32(uint8_t *p, uint32_t v) { for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i)); }
void zput64(uint8_t *p, uint64_t v) { for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i)); }
uint32_t zget32(const uint8_t *p) { uint32_t v = 0; for (int i = 0; i < 4; i++) v |= (uint32_t)p[i] << (8 * i); return v; }
uint64_t zget64(const uint8_t *p) { uint64_t v = 0; for (int i = 0; i < 8; i++) v |= (uint64_t)p[i] << (8 * i); return v; }

// geometry of a field at a rate; false on bad arguments
bool zfp_geom(int ndim, const size_t *dims, int dtype, uint32_t rate, ZfpGeom *g)
{
    if (ndim < 1 || ndim > 3 || !dims || (dtype != 0 && dtype != 1) || rate < 1 || rate > 256) return false;
    const uint32_t maxbits = rate << (2 * ndim);
    const int EB = dtype == 0 ? 9 : 12;
    if (maxbits % 32 || maxbits < (uint32_t)(EB + 2)) return false;
    memset(g, 0, sizeof(*g));
    g->nblocks = 1;
    for (int k = 0; k < 3; k++) {
        g->n[k] = k < ndim ? (long long)dims[k] : 1;
        if (g->n[k] < 1 || g->n[k] > (1ll << 40)) return false;
        g->nb[k] = (g->n[k] + 3) / 4;
        if (k < ndim) g->nblocks *= (unsigned long long)g->nb[k];
    }
    g->maxbits = maxbits;
    return true;
}

template <typename T>
cudaError_t launch_zfp(bool enc, int ndim, const void *src, void *dst, const ZfpGeom &g, cudaStream_t s)
{
    const unsigned grid = (unsigned)((g.nblocks + kZfpThreads - 1) / kZfpThreads);
    if (enc) {
        if (ndim == 1) zfp_encode_kernel<T, 1><<<grid, kZfpThreads, 0, s>>>((const T *)src, (uint32_t *)dst, g);
        else if (ndim == 2) zfp_encode_kernel<T, 2><<<grid, kZfpThreads, 0, s>>>((const T *)src, (uint32_t *)dst, g);
        else zfp_encode_kernel<T, 3><<<grid, kZfpThreads, 0, s>>>((const T *)src, (uint32_t *)dst, g);
    } else {
        if (ndim == 1) zfp_decode_kernel<T, 1><<<grid, kZfpThreads, 0, s>>>((const uint32_t *)src, (T *)dst, g);
        else if (ndim == 2) zfp_decode_kernel<T, 2><<<grid, kZfpThreads, 0, s>>>((const uint32_t *)src, (T *)dst, g);
        else zfp_decode_kernel<T, 3><<<grid, kZfpThreads, 0, s>>>((const uint32_t *)src, (T *)dst, g);
    }
    count_launch();
    return cudaGetLastError();
}

struct ZDevGuard {
    int prev = -1;
    bool changed = false;
    explicit ZDevGuard(int d)
    {
        cudaGetDevice(&prev);
        if (prev != d) changed = cudaSetDevice(d) == cudaSuccess;
    }
    ~ZDevGuard() { if (changed) cudaSetDevice(prev); }
};

}  // namespace
}  // namespace hpdr

using namespace hpdr;

extern "C" {

size_t hpdr_zfp_bound(int ndim, const size_t *dims, hpdr_dtype dtype, uint32_t rate)
{
    ZfpGeom g;
    if (!zfp_geom(ndim, dims, (int)dtype, rate, &g)) return 0;
    return (size_t)(kZfpHdr + g.nblocks * (g.maxbits / 8));
}

hpdr_status hpdr_zfp_compress(hpdr_ctx *ctx, const void *d_in, hpdr_dtype dtype, int ndim, const size_t *dims,
                              uint32_t rate, void *d_out, size_t out_capacity, size_t *out_bytes, void *stream)
{
    ZfpGeom g;
    if (!ctx || !d_in || !d_out || !out_bytes || !zfp_geom(ndim, dims, (int)dtype, rate, &g)) return HPDR_ERR_ARG;
    if (((uintptr_t)d_out & 15) || ((uintptr_t)d_in & ((dtype == HPDR_F64) ? 7 : 3))) return HPDR_ERR_ARG;
    const size_t total = (size_t)(kZfpHdr + g.nblocks * (g.maxbits / 8));
    if (out_capacity < total) return HPDR_ERR_CAPACITY;
    ZDevGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    ZfpHdrBytes h;
    memset(&h, 0, sizeof(h));
    memcpy(h.b, "HPDZ", 4);
    zput32(h.b + 4, 1);
    zput32(h.b + 8, (uint32_t)dtype);
    zput32(h.b + 12, (uint32_t)ndim);
    for (int k = 0; k < 3; k++) zput64(h.b + 16 + 8 * k, k < ndim ? (uint64_t)dims[k] : 1);
    zput32(h.b + 40, rate);
    zput32(h.b + 44, g.maxbits);
    zput64(h.b + 48, g.nblocks);
    zput32(h.b + 60, zfp_crc32(h.b, 60));
    uint8_t *out = (uint8_t *)d_out;
    zfp_header_kernel<<<1, 64, 0, s>>>(out, h);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return HPDR_ERR_CUDA;
    cudaError_t e = dtype == HPDR_F32 ? launch_zfp<float>(true, ndim, d_in, out + kZfpHdr, g, s)
                                      : launch_zfp<double>(true, ndim, d_in, out + kZfpHdr, g, s);
    if (e != cudaSuccess) return HPDR_ERR_CUDA;
    *out_bytes = total;
    return HPDR_OK;
}

hpdr_status hpdr_zfp_inspect(const void *in, size_t in_bytes, hpdr_dtype *dtype, int *ndim, size_t *dims,
                             uint32_t *rate)
{
    if (!in || !dtype || !ndim || !dims || !rate) return HPDR_ERR_ARG;
    if (in_bytes < (size_t)kZfpHdr) return HPDR_ERR_FORMAT;
    uint8_t h[kZfpHdr];
    cudaPointerAttributes at;
    bool dev = cudaPointerGetAttributes(&at, in) == cudaSuccess &&
               (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (dev) {
        if (cudaMemcpy(h, in, kZfpHdr, cudaMemcpyDeviceToHost) != cudaSuccess) return HPDR_ERR_CUDA;
    } else {
        memcpy(h, in, kZfpHdr);
    }
    if (memcmp(h, "HPDZ", 4) || zget32(h + 4) != 1 || zfp_crc32(h, 60) != zget32(h + 60)) return HPDR_ERR_FORMAT;
    const int dt = (int)zget32(h + 8), nd = (int)zget32(h + 12);
    size_t d[3];
    for (int k = 0; k < 3; k++) d[k] = (size_t)zget64(h + 16 + 8 * k);
    const uint32_t r = zget32(h + 40);
    ZfpGeom g;
    if (!zfp_geom(nd, d, dt, r, &g) || g.maxbits != zget32(h + 44) || g.nblocks != zget64(h + 48))
        return HPDR_ERR_FORMAT;
    if (kZfpHdr + g.nblocks * (g.maxbits / 8) > in_bytes) return HPDR_ERR_FORMAT;
    *dtype = (hpdr_dtype)dt;
    *ndim = nd;
    for (int k = 0; k < 3; k++) dims[k] = k < nd ? d[k] : 1;
    *rate = r;
    return HPDR_OK;
}

hpdr_status hpdr_zfp_decompress(hpdr_ctx *ctx, const void *d_in, size_t in_bytes, void *d_out, size_t out_capacity,
                                void *stream)
{
    if (!ctx || !d_in || !d_out) return HPDR_ERR_ARG;
    if ((uintptr_t)d_in & 15) return HPDR_ERR_ARG;
    ZDevGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamSynchronize(s) != cudaSuccess) return HPDR_ERR_CUDA;
    hpdr_dtype dt;
    int nd;
    size_t dims[3];
    uint32_t rate;
    hpdr_status st = hpdr_zfp_inspect(d_in, in_bytes, &dt, &nd, dims, &rate);
    if (st != HPDR_OK) return st;
    ZfpGeom g;
    zfp_geom(nd, dims, (int)dt, rate, &g);
    size_t N = 1;
    for (int k = 0; k < nd; k++) N *= dims[k];
    const size_t esz = dt == HPDR_F64 ? 8 : 4;
    if (out_capacity < N * esz) return HPDR_ERR_CAPACITY;
    if ((uintptr_t)d_out & (esz - 1)) return HPDR_ERR_ARG;
    const uint8_t *in = (const uint8_t *)d_in + kZfpHdr;
    cudaError_t e = dt == HPDR_F32 ? launch_zfp<float>(false, nd, in, d_out, g, s)
                                   : launch_zfp<double>(false, nd, in, d_out, g, s);
    return e == cudaSuccess ? HPDR_OK : HPDR_ERR_CUDA;
}

}  // extern "C"
