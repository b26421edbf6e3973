// levels_dev.cuh -- device helpers shared by the level kernels (levels.cu,
// decomp.cu): the quantization decision, stream indices of the level-major
// coefficient order, escapes and dequantization.  Not part of the ABI.
#pragma once
#include "levels.cuh"

namespace hpdr {
namespace {

// The quantization decision (Sec. IV-A, Alg. 1: linear quantization of the
// coefficients with the level's bin q): k = sign(x) floor(|x| rho + 1/2),
// rho = 1/q rounded to binary64 and every operation rounded to binary64,
// whatever the data type, so that codes agree with a binary64 decision on
// the same coefficients everywhere but at half-bin ties.  Codes whose
// magnitude reaches 2^62 are clamped there (the escape store then flags them).
template <typename T>
__device__ __forceinline__ long long quant_code(T x, double rho)
{
    const double ax = x < (T)0 ? -(double)x : (double)x;
    const double t = __dadd_rn(__dmul_rn(ax, rho), 0.5);
    long long k;
    if (t < 1073741824.0) k = (long long)(int)floor(t);
    else if (t < 4611686018427387904.0) k = (long long)floor(t);
    else k = kEscMax;
    return x < (T)0 ? -k : k;
}

// The same decision for a binary32 coefficient, in binary32 arithmetic on a
// double-word product (binary64 throughput is low on this part).  With
// rho = rho_hi + rho_lo (rho_hi = fl32(rho), rho_lo = fl32(rho - rho_hi)):
//   p = fl32(ax rho_hi); e = ax rho_hi - p exactly (one FMA); e2 = fl32(e + ax rho_lo),
// so ax rho = p + e2 to within about 2^-47 ax rho.  With n = rint(p) and
// d = p - n (exact), floor(ax rho + 1/2) = n + [d + e2 >= 1/2] - [d + e2 < -1/2],
// and both comparisons are exact (1/2 - d and -1/2 - d are representable
// whenever the result can change).  Valid while p < kSmallQuant = 2^22 (then
// ulp(p) <= 1/4, |d + e2| < 3/4, and n is an exact integer); the result
// differs from the binary64 decision only when ax rho lies within about
// 2^-46 ax rho of a half-integer.
constexpr float kSmallQuant = 4194304.0f;
__device__ __forceinline__ int quant_small_f32(float ax, float rho_hi, float rho_lo)
{
    const float p = __fmul_rn(ax, rho_hi);
    const float e = __fmaf_rn(ax, rho_hi, -p);
    const float e2 = __fmaf_rn(ax, rho_lo, e);
    const float n = rintf(p);
    const float d = __fsub_rn(p, n);
    return __float2int_rn(n) + (e2 >= __fsub_rn(0.5f, d) ? 1 : 0) - (e2 < __fsub_rn(-0.5f, d) ? 1 : 0);
}

__device__ __forceinline__ double rho64_of(const Scalars *sc, int l) { return sc->rho_d[l]; }


template <typename T> __device__ __forceinline__ T q_of(const Scalars *sc, int l);
template <> __device__ __forceinline__ float q_of<float>(const Scalars *sc, int l) { return sc->q_f[l]; }
template <> __device__ __forceinline__ double q_of<double>(const Scalars *sc, int l) { return sc->q[l]; }

template <typename T>
__device__ __forceinline__ long long stream_rank(const LevelGeom<T> &g, int p0, int p1, int p2)
{
    const long long m1 = g.dim[1].m, m2 = g.dim[2].m;
    const long long mc1 = g.dim[1].mc, mc2 = g.dim[2].mc;
    long long flat = ((long long)p0 * m1 + p1) * m2 + p2;
    long long cr = (long long)kept_before(p0) * mc1 * mc2;
    if (kept_pos(g.dim[0].m, p0)) {
        cr += (long long)kept_before(p1) * mc2;
        if (kept_pos((int)m1, p1)) cr += kept_before(p2);
    }
    return g.Nprev + flat - cr;
}

// Stream index of the new nodes of row (p0, p1) of level l:
//   every node new (p0 or p1 new):        base + p2
//   p0 and p1 kept (only odd p2 new):     base + (p2 - 1) / 2
template <typename T>
__device__ __forceinline__ long long row_base(const LevelGeom<T> &g, long long plane_base, bool k0,
                                              int p1)
{
    const long long m2 = g.dim[2].m, mc2 = g.dim[2].mc;
    return plane_base + (long long)p1 * m2 - (k0 ? (long long)kept_before(p1) * mc2 : 0LL);
}
template <typename T>
__device__ __forceinline__ long long plane_base_of(const LevelGeom<T> &g, int p0)
{
    const long long m1 = g.dim[1].m, m2 = g.dim[2].m;
    const long long mc1 = g.dim[1].mc, mc2 = g.dim[2].mc;
    return g.Nprev + (long long)p0 * m1 * m2 - (long long)kept_before(p0) * mc1 * mc2;
}

// an escaped code (symbol 0) keeps its k at its stream position; the encoder
// writes it into the bitstream after the escape's codeword, as zigzag(k) in
// the container's payload width.  Returns the bit length of zigzag(k).
__device__ __forceinline__ unsigned escape_store(const QuantOut &qo, long long si, long long k)
{
    if (k >= kEscMax || k <= -kEscMax) atomicExch(&qo.sc->status, (unsigned int)DS_ARG);
    qo.esc[si] = k;
    const unsigned long long z = k >= 0 ? 2ULL * (unsigned long long)k : 2ULL * (unsigned long long)(-(k + 1)) + 1ULL;
    return 64u - (unsigned)__clzll((long long)z);
}

// An escape of a binary32 coefficient (|k| >= D/2): its exact code (the
// double-word decision below 2^22, binary64 above) stored at its stream
// position; returns the payload bit length.  Out of line: escapes are rare.
__device__ __noinline__ unsigned escape_f32(const QuantOut &qo, long long si, float w, float rho_f, float rho_lo,
                                            double rho)
{
    const float ax = fabsf(w);
    long long k;
    if (__fmul_rn(ax, rho_f) < kSmallQuant) {
        const int ki = quant_small_f32(ax, rho_f, rho_lo);
        k = w < 0.0f ? -(long long)ki : (long long)ki;
    } else {
        k = quant_code(w, rho);
    }
    return escape_store(qo, si, k);
}

// quantize one coefficient into the symbol stream (+ block histogram / escapes)
template <typename T>
__device__ __forceinline__ void quant_emit(const QuantOut &qo, unsigned int *hs, bool smem_hist,
                                           long long si, T w, double rho)
{
    long long k = quant_code(w, rho);
    long long s = k + (long long)(qo.D / 2);
    unsigned int sym;
    if (s >= 1 && s <= (long long)qo.D - 1) {
        sym = (unsigned int)s;
    } else {
        sym = 0;
        atomicMax(&qo.sc->esc_w, escape_store(qo, si, k));
    }
    qo.sym[si] = (uint16_t)sym;
    if (smem_hist) atomicAdd(&hs[sym], 1u);
    else atomicAdd(&qo.hist[sym], 1ULL);
}

template <typename T>
__device__ __forceinline__ T dequant_sym(const SymIn &si_, unsigned s, long long idx, T q)
{
    if (s != 0) return mul_rn((T)((int)s - (int)(si_.D / 2)), q);
    return mul_rn((T)si_.esc[idx], q);
}

template <typename T>
__device__ __forceinline__ T dequant(const SymIn &si_, long long idx, int level)
{
    return dequant_sym<T>(si_, si_.sym[idx], idx, q_of<T>(si_.sc, level));
}

template <typename T>
__device__ __forceinline__ int first_coarse_at_or_after(const DimTables<T> &d, int p)
{
    // smallest coarse j with cpos(j) >= p
    int j = p <= 0 ? 0 : (p + 1) >> 1;
    return j < d.mc ? j : d.mc - 1;
}


}  // namespace

// Coarse planes per CTA (segment) for a grid of `tiles` x segments CTAs.
int choose_segment(int mc0, long long tiles, int per_sm);

// Resident CTAs per SM of a kernel at a block size and dynamic shared memory.
template <typename K>
int resident_ctas(K kernel, int threads, size_t smem)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        n = 1;
    }
    return n > 1 ? n : 1;
}

}  // namespace hpdr
