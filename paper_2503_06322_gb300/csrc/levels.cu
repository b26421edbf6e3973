// levels.cu -- per-level kernels of the multilevel decomposition (Sec. IV-A,
// Alg. 1) and of its inverse, for sm_103a.
//
// restrict_kernel is the bandwidth-critical one.  One CTA owns an 8 x 32 tile
// of coarse nodes in dims (1, 2) and streams a segment of dim 0 plane by plane
// (2.5-D blocking).  For each fine plane it
//   A. stages the level-l values of the tile region (with a 2-node halo) in
//      shared memory, three planes deep;
//   B. forms w, the new-node coefficients mc_l = v - lerp(v) (Alg. 1 lerp),
//      and, on the nodes it owns, hands them to a sink: quantization with the
//      level's bin + block histogram + symbol store (compression, Alg. 1
//      MapAndProcess and Alg. 2 histogram), or a coefficient store;
//   C./D. applies the restriction P^T M_l (Alg. 1 mass_trans) along dim 2
//      and dim 1 in shared memory and accumulates the dim-0 taps in registers,
//      so that only the coarse result b (1/8 of the level) is written.
// The result does not depend on the tiling: every coarse value sums its taps
// in a fixed order.
#include <cfloat>
#include "levels.cuh"

namespace hpdr {
namespace {

constexpr int TT1 = 8, TT2 = 32;                  // coarse tile (dims 1, 2)
constexpr int RR1 = 2 * TT1 + 4, RR2 = 2 * TT2 + 4;  // largest fine region
constexpr int RTHREADS = 256;
constexpr int kHistSmemMax = 16384;
constexpr int kNormBlocks = 152 * 8;

template <typename T>
__device__ __forceinline__ long long quant_code(T x, T rho)
{
    T ax = x < (T)0 ? -x : x;
    T y = mul_rn(ax, rho);
    T t = add_rn(y, (T)0.5);
    long long k = (long long)floor(t);
    return x < (T)0 ? -k : k;
}

template <typename T> __device__ __forceinline__ T rho_of(const Scalars *sc, int l);
template <> __device__ __forceinline__ float rho_of<float>(const Scalars *sc, int l) { return sc->rho_f[l]; }
template <> __device__ __forceinline__ double rho_of<double>(const Scalars *sc, int l) { return sc->rho_d[l]; }
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

// quantize one coefficient into the symbol stream (+ block histogram / outliers)
template <typename T>
__device__ __forceinline__ void quant_emit(const QuantOut &qo, unsigned int *hs, bool smem_hist,
                                           long long si, T w, T rho)
{
    long long k = quant_code(w, rho);
    long long s = k + (long long)(qo.D / 2);
    unsigned int sym;
    if (s >= 1 && s <= (long long)qo.D - 1) {
        sym = (unsigned int)s;
    } else {
        sym = 0;
        unsigned long long pos = atomicAdd(&qo.sc->n_out, 1ULL);
        if (pos < qo.out_cap) {
            qo.out_idx[pos] = (unsigned long long)si;
            qo.out_k[pos] = k;
        } else {
            atomicExch(&qo.sc->status, (unsigned int)DS_CAPACITY);
        }
    }
    qo.sym[si] = (uint16_t)sym;
    if (smem_hist) atomicAdd(&hs[sym], 1u);
    else atomicAdd(&qo.hist[sym], 1ULL);
}

template <typename T>
__device__ __forceinline__ T dequant(const SymIn &si_, long long idx, int level)
{
    unsigned int s = si_.sym[idx];
    long long k;
    if (s != 0) {
        k = (long long)s - (long long)(si_.D / 2);
    } else {
        // outliers are sorted by stream index
        unsigned long long lo = 0, hi = si_.n_out;
        while (lo < hi) {
            unsigned long long mid = (lo + hi) >> 1;
            if (si_.out_idx[mid] < (unsigned long long)idx) lo = mid + 1; else hi = mid;
        }
        if (lo < si_.n_out && si_.out_idx[lo] == (unsigned long long)idx) {
            k = si_.out_k[lo];
        } else {
            atomicExch(si_.status, (unsigned int)DS_FORMAT);
            k = 0;
        }
    }
    return mul_rn((T)k, q_of<T>(si_.sc, level));
}

template <typename T>
__device__ __forceinline__ int first_coarse_at_or_after(const DimTables<T> &d, int p)
{
    // smallest coarse j with cpos(j) >= p
    int j = p <= 0 ? 0 : (p + 1) >> 1;
    return j < d.mc ? j : d.mc - 1;
}

template <typename T, int SRC, int SINK>
__global__ void __launch_bounds__(RTHREADS)
restrict_kernel(RestrictArgs<T> a, int seg_len)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m0 = a.g.dim[0].m, m1 = a.g.dim[1].m, m2 = a.g.dim[2].m;
    const int mc0 = a.g.dim[0].mc, mc1 = a.g.dim[1].mc, mc2 = a.g.dim[2].mc;
    const int J2 = blockIdx.x * TT2, J1 = blockIdx.y * TT1;
    const int J0a = blockIdx.z * seg_len;
    const int J0b = min(J0a + seg_len, mc0);
    if (J0a >= J0b) return;
    const int n2 = min(TT2, mc2 - J2), n1 = min(TT1, mc1 - J1);
    const int lo2 = max(0, cpos_of(m2, mc2, J2) - 2) & ~1;
    const int hi2 = min(m2 - 1, cpos_of(m2, mc2, J2 + n2 - 1) + 2);
    const int lo1 = max(0, cpos_of(m1, mc1, J1) - 2) & ~1;
    const int hi1 = min(m1 - 1, cpos_of(m1, mc1, J1 + n1 - 1) + 2);
    const int lo0 = max(0, cpos_of(m0, mc0, J0a) - 2) & ~1;
    const int hi0 = min(m0 - 1, cpos_of(m0, mc0, J0b - 1) + 2);
    const int r1n = hi1 - lo1 + 1, r2n = hi2 - lo2 + 1;
    const int o2a = cpos_of(m2, mc2, J2), o2b = (J2 + n2 < mc2) ? cpos_of(m2, mc2, J2 + n2) : m2;
    const int o1a = cpos_of(m1, mc1, J1), o1b = (J1 + n1 < mc1) ? cpos_of(m1, mc1, J1 + n1) : m1;
    const int o0a = cpos_of(m0, mc0, J0a), o0b = (J0b < mc0) ? cpos_of(m0, mc0, J0b) : m0;

    T *V = reinterpret_cast<T *>(smem_raw);                 // [3][RR1][RR2] (FIELD)
    T *W = V + (SRC == (int)WSrc::FIELD ? 3 * RR1 * RR2 : 0);  // [RR1][RR2]
    T *R2s = W + RR1 * RR2;                                // [RR1][TT2]
    T *tap2s = R2s + RR1 * TT2;                            // [TT2*5]
    T *tap1s = tap2s + TT2 * 5;                            // [TT1*5]
    T *wl2s = tap1s + TT1 * 5, *wr2s = wl2s + RR2;         // [RR2]
    T *wl1s = wr2s + RR2, *wr1s = wl1s + RR1;              // [RR1]
    unsigned int *hs = reinterpret_cast<unsigned int *>(wr1s + RR1);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool smem_hist = (SINK == (int)Sink::QUANT) && a.qo.D <= (unsigned)kHistSmemMax;
    const T *tap2src = a.use_ptap ? a.g.dim[2].ptap : a.g.dim[2].tap;
    const T *tap1src = a.use_ptap ? a.g.dim[1].ptap : a.g.dim[1].tap;
    const T *tap0src = a.use_ptap ? a.g.dim[0].ptap : a.g.dim[0].tap;
    for (int i = tid; i < n2 * 5; i += RTHREADS) tap2s[i] = tap2src[J2 * 5 + i];
    for (int i = tid; i < n1 * 5; i += RTHREADS) tap1s[i] = tap1src[J1 * 5 + i];
    for (int i = tid; i < r2n; i += RTHREADS) { wl2s[i] = a.g.dim[2].wl[lo2 + i]; wr2s[i] = a.g.dim[2].wr[lo2 + i]; }
    for (int i = tid; i < r1n; i += RTHREADS) { wl1s[i] = a.g.dim[1].wl[lo1 + i]; wr1s[i] = a.g.dim[1].wr[lo1 + i]; }
    if (smem_hist)
        for (int i = tid; i < (int)a.qo.D; i += RTHREADS) hs[i] = 0u;

    T rho = (T)0;
    if (SINK == (int)Sink::QUANT) rho = rho_of<T>(a.qo.sc, a.g.level);

    auto load_plane = [&](int p) {
        T *dst = V + (p % 3) * RR1 * RR2;
        const T *src = a.v + ((long long)p * m1 + lo1) * m2 + lo2;
        for (int i1 = warp; i1 < r1n; i1 += RTHREADS / 32) {
            const T *row = src + (long long)i1 * m2;
            for (int i2 = lane; i2 < r2n; i2 += 32) dst[i1 * RR2 + i2] = row[i2];
        }
    };
    if (SRC == (int)WSrc::FIELD) load_plane(lo0);

    // per-thread output (j1l, j2l) and its dim-0 accumulators
    const int j1l = tid >> 5, j2l = tid & 31;
    const bool outp = j1l < n1 && j2l < n2;
    const int c1r = outp ? cpos_of(m1, mc1, J1 + j1l) - lo1 : 0;
    const int c2r = outp ? cpos_of(m2, mc2, J2 + j2l) - lo2 : 0;
    T acc0 = 0, acc1 = 0, acc2 = 0;
    int jb = J0a;
    const long long out_col = (long long)(J1 + j1l) * mc2 + (J2 + j2l);

    for (int p0 = lo0; p0 <= hi0; p0++) {
        if (SRC == (int)WSrc::FIELD && p0 + 1 <= hi0) load_plane(p0 + 1);
        __syncthreads();
        // ---- B: w on the region --------------------------------------------
        const bool f0 = !kept_pos(m0, p0);
        const bool own0 = p0 >= o0a && p0 < o0b;
        const int s0 = p0 % 3, sm = (p0 + 2) % 3, sp = (p0 + 1) % 3;
        T wl0 = (T)0, wr0 = (T)0;
        if (SRC == (int)WSrc::FIELD && f0) { wl0 = a.g.dim[0].wl[p0]; wr0 = a.g.dim[0].wr[p0]; }
        for (int i1 = warp; i1 < r1n; i1 += RTHREADS / 32) {
            const int p1 = lo1 + i1;
            const bool f1 = !kept_pos(m1, p1);
            const bool own01 = own0 && p1 >= o1a && p1 < o1b;
            for (int i2 = lane; i2 < r2n; i2 += 32) {
                const int p2 = lo2 + i2;
                const bool f2 = !kept_pos(m2, p2);
                const bool isnew = f0 || f1 || f2;
                T w = (T)0;
                if (SRC == (int)WSrc::FIELD) {
                    const T *P0 = V + s0 * RR1 * RR2;
                    if (isnew) {
                        auto val = [&](int s, int r) -> T {
                            const T *row = V + (s * RR1 + r) * RR2;
                            if (f2) return fma_rn(wr2s[i2], row[i2 + 1], mul_rn(wl2s[i2], row[i2 - 1]));
                            return row[i2];
                        };
                        auto pl = [&](int s) -> T {
                            if (f1) return fma_rn(wr1s[i1], val(s, i1 + 1), mul_rn(wl1s[i1], val(s, i1 - 1)));
                            return val(s, i1);
                        };
                        T lerp = f0 ? fma_rn(wr0, pl(sp), mul_rn(wl0, pl(sm))) : pl(s0);
                        w = sub_rn(P0[i1 * RR2 + i2], lerp);
                        if (SINK != (int)Sink::NONE && own01 && p2 >= o2a && p2 < o2b) {
                            long long si = stream_rank(a.g, p0, p1, p2);
                            if (SINK == (int)Sink::STREAM) a.coef_out[si] = w;
                            else quant_emit(a.qo, hs, smem_hist, si, w, rho);
                        }
                    }
                } else if (SRC == (int)WSrc::STREAM) {
                    if (isnew) w = a.coef_in[stream_rank(a.g, p0, p1, p2)];
                } else if (SRC == (int)WSrc::SYMBOLS) {
                    if (isnew) w = dequant<T>(a.symin, stream_rank(a.g, p0, p1, p2), a.g.level);
                } else {  // DENSE
                    if (isnew || !a.dense_new_only) w = a.v[((long long)p0 * m1 + p1) * m2 + p2];
                }
                W[i1 * RR2 + i2] = w;
            }
        }
        __syncthreads();
        // ---- C: restriction along dim 2 ---------------------------------------
        for (int i1 = warp; i1 < r1n; i1 += RTHREADS / 32) {
            if (lane < n2) {
                const int c = cpos_of(m2, mc2, J2 + lane) - lo2;
                T s = (T)0;
#pragma unroll
                for (int o = -2; o <= 2; o++) {
                    const int idx = c + o;
                    if (idx >= 0 && idx < r2n) s = fma_rn(tap2s[lane * 5 + o + 2], W[i1 * RR2 + idx], s);
                }
                R2s[i1 * TT2 + lane] = s;
            }
        }
        __syncthreads();
        // ---- D: restriction along dim 1, dim-0 taps into registers ------------
        if (outp) {
            T r = (T)0;
#pragma unroll
            for (int o = -2; o <= 2; o++) {
                const int idx = c1r + o;
                if (idx >= 0 && idx < r1n) r = fma_rn(tap1s[j1l * 5 + o + 2], R2s[idx * TT2 + j2l], r);
            }
            int jlo = first_coarse_at_or_after(a.g.dim[0], p0 - 2);
            if (jlo < J0a) jlo = J0a;
            while (jb < jlo && jb < J0b) {
                a.b[(long long)jb * mc1 * mc2 + out_col] = acc0;
                acc0 = acc1; acc1 = acc2; acc2 = (T)0;
                jb++;
            }
            {
                int j = jb, o = p0 - cpos_of(m0, mc0, j);
                if (j < J0b && o >= -2 && o <= 2) acc0 = fma_rn(tap0src[j * 5 + o + 2], r, acc0);
                j = jb + 1;
                if (j < J0b) { o = p0 - cpos_of(m0, mc0, j); if (o >= -2 && o <= 2) acc1 = fma_rn(tap0src[j * 5 + o + 2], r, acc1); }
                j = jb + 2;
                if (j < J0b) { o = p0 - cpos_of(m0, mc0, j); if (o >= -2 && o <= 2) acc2 = fma_rn(tap0src[j * 5 + o + 2], r, acc2); }
            }
            if (SRC == (int)WSrc::FIELD && SINK != (int)Sink::NONE && a.vc && kept_pos(m0, p0)) {
                const int j0 = cidx_of(m0, mc0, p0);
                if (j0 >= J0a && j0 < J0b)
                    a.vc[(long long)j0 * mc1 * mc2 + out_col] = V[(s0 * RR1 + c1r) * RR2 + c2r];
            }
        }
    }
    if (outp) {
        while (jb < J0b) {
            a.b[(long long)jb * mc1 * mc2 + out_col] = acc0;
            acc0 = acc1; acc1 = acc2; acc2 = (T)0;
            jb++;
        }
    }
    if (smem_hist) {
        __syncthreads();
        for (int i = tid; i < (int)a.qo.D; i += RTHREADS)
            if (hs[i]) atomicAdd(&a.qo.hist[i], (unsigned long long)hs[i]);
    }
}

template <typename T>
size_t restrict_smem(WSrc src, Sink sink, unsigned int D)
{
    size_t n = (src == WSrc::FIELD ? 3 : 0) * RR1 * RR2 + RR1 * RR2 + RR1 * TT2 + (TT2 + TT1) * 5 +
               2 * (RR1 + RR2);
    size_t b = n * sizeof(T);
    if (sink == Sink::QUANT && D <= (unsigned)kHistSmemMax) b += (size_t)D * sizeof(unsigned int);
    return b;
}

// --------------------------------------------------------------------------
// Thomas solves of the coarse mass matrix along one dimension (Alg. 1
// tridiag; the paper's Iterative abstraction: one sequential sweep per line,
// many lines in parallel).

template <typename T>
__global__ void __launch_bounds__(256)
solve_strided_kernel(T *b, int n, long long stride, long long nlines, const T *__restrict__ sub,
                     const T *__restrict__ cp, const T *__restrict__ inv_den, T *vc, int sign)
{
    long long line = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (line >= nlines) return;
    long long o = line / stride, i = line - o * stride;
    T *p = b + o * (long long)n * stride + i;
    T y = (T)0;
#pragma unroll 4
    for (int t = 0; t < n; t++) {
        y = mul_rn(fma_rn(-sub[t], y, p[(long long)t * stride]), inv_den[t]);
        p[(long long)t * stride] = y;
    }
    T x = (T)0;
    T *q = vc ? vc + o * (long long)n * stride + i : nullptr;
#pragma unroll 4
    for (int t = n - 1; t >= 0; t--) {
        x = fma_rn(-cp[t], x, p[(long long)t * stride]);
        if (sign == 0) p[(long long)t * stride] = x;
        else if (sign > 0) q[(long long)t * stride] = add_rn(q[(long long)t * stride], x);
        else q[(long long)t * stride] = sub_rn(q[(long long)t * stride], x);
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
solve_contig_kernel(T *b, int n, long long nlines, int rows, int pitch, const T *__restrict__ sub,
                    const T *__restrict__ cp, const T *__restrict__ inv_den, T *vc, int sign)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *S = reinterpret_cast<T *>(smem_raw);
    long long row0 = blockIdx.x * (long long)rows;
    int nr = (int)min((long long)rows, nlines - row0);
    const T *src = b + row0 * n;
    for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) {
        int r = idx / n, t = idx - r * n;
        S[r * pitch + t] = src[idx];
    }
    __syncthreads();
    if ((int)threadIdx.x < nr) {
        T *p = S + threadIdx.x * pitch;
        T y = (T)0;
        for (int t = 0; t < n; t++) { y = mul_rn(fma_rn(-sub[t], y, p[t]), inv_den[t]); p[t] = y; }
        T x = (T)0;
        for (int t = n - 1; t >= 0; t--) { x = fma_rn(-cp[t], x, p[t]); p[t] = x; }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) {
        int r = idx / n, t = idx - r * n;
        T z = S[r * pitch + t];
        long long gi = row0 * n + idx;
        if (sign == 0) b[gi] = z;
        else if (sign > 0) vc[gi] = add_rn(vc[gi], z);
        else vc[gi] = sub_rn(vc[gi], z);
    }
}

// --------------------------------------------------------------------------
// Recomposition of one level: kept nodes from the corrected coarse grid, new
// nodes = coefficient + multilinear interpolant (inverse of Alg. 1 lerp).

template <typename T, int SRC>
__global__ void __launch_bounds__(128)
expand_kernel(LevelGeom<T> g, const T *__restrict__ vc, const T *coef_in, SymIn symin, T *out)
{
    const int m0 = g.dim[0].m, m1 = g.dim[1].m, m2 = g.dim[2].m;
    const int mc0 = g.dim[0].mc, mc1 = g.dim[1].mc, mc2 = g.dim[2].mc;
    const long long row = blockIdx.x;
    const int p0 = (int)(row / m1), p1 = (int)(row - (long long)p0 * m1);
    const bool f0 = !kept_pos(m0, p0), f1 = !kept_pos(m1, p1);
    int a0, b0, a1, b1;
    T wl0 = 0, wr0 = 0, wl1 = 0, wr1 = 0;
    if (f0) { a0 = cidx_of(m0, mc0, p0 - 1); b0 = cidx_of(m0, mc0, p0 + 1); wl0 = g.dim[0].wl[p0]; wr0 = g.dim[0].wr[p0]; }
    else { a0 = b0 = cidx_of(m0, mc0, p0); }
    if (f1) { a1 = cidx_of(m1, mc1, p1 - 1); b1 = cidx_of(m1, mc1, p1 + 1); wl1 = g.dim[1].wl[p1]; wr1 = g.dim[1].wr[p1]; }
    else { a1 = b1 = cidx_of(m1, mc1, p1); }
    const T *wl2 = g.dim[2].wl, *wr2 = g.dim[2].wr;
    T *orow = out + row * m2;
    for (int p2 = threadIdx.x; p2 < m2; p2 += blockDim.x) {
        const bool f2 = !kept_pos(m2, p2);
        if (!(f0 || f1 || f2)) {
            orow[p2] = vc[((long long)a0 * mc1 + a1) * mc2 + cidx_of(m2, mc2, p2)];
            continue;
        }
        const int a2 = f2 ? cidx_of(m2, mc2, p2 - 1) : cidx_of(m2, mc2, p2);
        const int b2 = f2 ? cidx_of(m2, mc2, p2 + 1) : a2;
        const T w2l = f2 ? wl2[p2] : (T)0, w2r = f2 ? wr2[p2] : (T)0;
        auto val = [&](int c0, int c1) -> T {
            const T *r = vc + ((long long)c0 * mc1 + c1) * mc2;
            if (f2) return fma_rn(w2r, r[b2], mul_rn(w2l, r[a2]));
            return r[a2];
        };
        auto pl = [&](int c0) -> T {
            if (f1) return fma_rn(wr1, val(c0, b1), mul_rn(wl1, val(c0, a1)));
            return val(c0, a1);
        };
        T lerp = f0 ? fma_rn(wr0, pl(b0), mul_rn(wl0, pl(a0))) : pl(a0);
        long long si = stream_rank(g, p0, p1, p2);
        T c = (SRC == (int)WSrc::STREAM) ? coef_in[si] : dequant<T>(symin, si, g.level);
        orow[p2] = add_rn(c, lerp);
    }
}

// --------------------------------------------------------------------------
template <typename T, int SINK>
__global__ void level0_kernel(const T *v0, long long N0, T *coef_out, QuantOut qo)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N0) return;
    T x = v0[i];
    if (SINK == (int)Sink::STREAM) { coef_out[i] = x; return; }
    quant_emit(qo, nullptr, false, i, x, rho_of<T>(qo.sc, 0));
}

template <typename T, int SRC>
__global__ void level0_in_kernel(const T *coef_in, SymIn symin, long long N0, T *v0)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N0) return;
    v0[i] = (SRC == (int)WSrc::STREAM) ? coef_in[i] : dequant<T>(symin, i, 0);
}

// --------------------------------------------------------------------------
// max|u| and sum u^2: fixed grid, fixed per-thread order -> deterministic.

template <typename T>
__device__ __forceinline__ void nan_max(T &m, T x)
{
    if (x > m || x != x) m = (m != m) ? m : x;
}

template <typename T>
__global__ void __launch_bounds__(256) norm_kernel(const T *__restrict__ u, long long N, double *partials)
{
    T mx = (T)0;
    double ss = 0.0;
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long nth = (long long)gridDim.x * blockDim.x;
    constexpr int V = 16 / sizeof(T);
    const bool vec = (((uintptr_t)u) & 15) == 0;
    long long nv = vec ? N / V : 0;
    if (vec) {
        typedef typename std::conditional<sizeof(T) == 4, float4, double2>::type VT;
        const VT *uv = reinterpret_cast<const VT *>(u);
        for (long long i = tid; i < nv; i += nth) {
            VT x = __ldcs(uv + i);
            const T *e = reinterpret_cast<const T *>(&x);
#pragma unroll
            for (int k = 0; k < V; k++) {
                T ax = e[k] < (T)0 ? -e[k] : e[k];
                nan_max(mx, ax);
                ss += (double)e[k] * (double)e[k];
            }
        }
    }
    for (long long i = nv * V + tid; i < N; i += nth) {
        T x = u[i];
        T ax = x < (T)0 ? -x : x;
        nan_max(mx, ax);
        ss += (double)x * (double)x;
    }
    for (int o = 16; o > 0; o >>= 1) {
        T om = __shfl_down_sync(0xffffffffu, mx, o);
        double os = __shfl_down_sync(0xffffffffu, ss, o);
        nan_max(mx, om);
        ss += os;
    }
    __shared__ T smx[8];
    __shared__ double sss[8];
    int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { smx[w] = mx; sss[w] = ss; }
    __syncthreads();
    if (threadIdx.x == 0) {
        T m = smx[0];
        double s = sss[0];
        for (int i = 1; i < (int)(blockDim.x >> 5); i++) { nan_max(m, smx[i]); s += sss[i]; }
        partials[2 * blockIdx.x] = (double)m;
        partials[2 * blockIdx.x + 1] = s;
    }
}

__global__ void bins_kernel(BinArgs ba, const double *partials, int nparts, Scalars *sc)
{
    __shared__ double smx[256], sss[256];
    double mx = 0.0, ss = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        double m = partials[2 * i];
        if (m > mx || m != m) mx = (mx != mx) ? mx : m;
        ss += partials[2 * i + 1];
    }
    smx[threadIdx.x] = mx;
    sss[threadIdx.x] = ss;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            double m = smx[threadIdx.x + s];
            if (m > smx[threadIdx.x] || m != m) smx[threadIdx.x] = (smx[threadIdx.x] != smx[threadIdx.x]) ? smx[threadIdx.x] : m;
            sss[threadIdx.x] += sss[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    mx = smx[0];
    ss = sss[0];
    sc->maxabs = mx;
    sc->sumsq = ss;
    const int L = ba.L;
    bool ok = mx <= DBL_MAX;
    double nrm = ba.mode == 0 ? mx : sqrt(__ddiv_rn(ss, (double)ba.N));
    double tau = ba.tol_kind == 1 ? __dmul_rn(ba.tol, nrm) : ba.tol;
    sc->tau_abs = tau;
    double tp = 0.0;
    if (ok && mx > 0.0) {
        tp = __dsub_rn(tau, __dmul_rn(__dmul_rn(__dmul_rn(32.0, (double)(L + 1)), ba.eps), mx));
        if (!(tp > 0.0)) ok = false;
    }
    for (int l = 0; l <= L; l++) {
        double q;
        if (!ok || mx == 0.0) q = 1.0;
        else if (l == 0) q = __ddiv_rn(__dmul_rn(2.0, tp), (double)(L + 1));
        else q = __ddiv_rn(__dmul_rn(2.0, tp), __dmul_rn((double)(L + 1), __dadd_rn(1.0, ba.c[l])));
        sc->q[l] = q;
        double r = __ddiv_rn(1.0, q);
        sc->rho_d[l] = r;
        sc->rho_f[l] = __double2float_rn(r);
        sc->q_f[l] = __double2float_rn(q);
    }
    if (!ok) atomicExch(&sc->status, (unsigned int)DS_ARG);
}

template <typename T, int SRC, int SINK>
cudaError_t launch_restrict_t(const RestrictArgs<T> &a, cudaStream_t s)
{
    const int mc0 = a.g.dim[0].mc, mc1 = a.g.dim[1].mc, mc2 = a.g.dim[2].mc;
    const int gx = (mc2 + TT2 - 1) / TT2, gy = (mc1 + TT1 - 1) / TT1;
    const long long target = 152LL * 9;
    long long tiles = (long long)gx * gy;
    int seg = (int)std::max<long long>(8, (mc0 * tiles + target - 1) / target);
    if (seg > mc0) seg = mc0;
    const int gz = (mc0 + seg - 1) / seg;
    size_t sm = restrict_smem<T>((WSrc)SRC, (Sink)SINK, SINK == (int)Sink::QUANT ? a.qo.D : 0);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(restrict_kernel<T, SRC, SINK>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    restrict_kernel<T, SRC, SINK><<<dim3(gx, gy, gz), RTHREADS, sm, s>>>(a, seg);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

int norm_parts() { return kNormBlocks; }

template <typename T>
cudaError_t launch_restrict(WSrc src, Sink sink, const RestrictArgs<T> &a, cudaStream_t s)
{
    if (src == WSrc::FIELD && sink == Sink::QUANT) return launch_restrict_t<T, 0, 2>(a, s);
    if (src == WSrc::FIELD && sink == Sink::STREAM) return launch_restrict_t<T, 0, 1>(a, s);
    if (src == WSrc::FIELD) return launch_restrict_t<T, 0, 0>(a, s);
    if (src == WSrc::STREAM) return launch_restrict_t<T, 1, 0>(a, s);
    if (src == WSrc::SYMBOLS) return launch_restrict_t<T, 2, 0>(a, s);
    return launch_restrict_t<T, 3, 0>(a, s);
}

template <typename T>
cudaError_t launch_solves(const LevelGeom<T> &g, T *b, T *vc, int sign, cudaStream_t s)
{
    const long long c0 = g.dim[0].mc, c1 = g.dim[1].mc, c2 = g.dim[2].mc;
    int last = -1;
    for (int k = 0; k < 3; k++) if (g.dim[k].mc > 1 && g.dim[k].m > 1) last = k;
    for (int k = 0; k < 3; k++) {
        const DimTables<T> &d = g.dim[k];
        if (!(d.m > 1)) continue;
        int sg = (k == last) ? sign : 0;
        if (k < 2) {
            long long stride = (k == 0) ? c1 * c2 : c2;
            long long nlines = (k == 0) ? c1 * c2 : c0 * c2;
            int n = d.mc;
            solve_strided_kernel<T><<<(unsigned)((nlines + 255) / 256), 256, 0, s>>>(
                b, n, stride, nlines, d.sub, d.cp, d.inv_den, vc, sg);
        } else {
            int n = d.mc;
            long long nlines = c0 * c1;
            int pitch = n | 1;
            size_t rowbytes = (size_t)pitch * sizeof(T);
            int rows = (int)std::min<size_t>(64, (96 * 1024) / rowbytes);
            if (rows < 1) {
                solve_strided_kernel<T><<<(unsigned)((nlines + 255) / 256), 256, 0, s>>>(
                    b, n, 1, nlines, d.sub, d.cp, d.inv_den, vc, sg);
            } else {
                static bool attr = false;
                if (!attr) {
                    cudaFuncSetAttribute(solve_contig_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
                    attr = true;
                }
                solve_contig_kernel<T><<<(unsigned)((nlines + rows - 1) / rows), 256, rows * rowbytes, s>>>(
                    b, n, nlines, rows, pitch, d.sub, d.cp, d.inv_den, vc, sg);
            }
        }
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_expand(WSrc src, const LevelGeom<T> &g, const T *vc, const T *coef_in,
                          const SymIn &symin, T *out, cudaStream_t s)
{
    long long rows = (long long)g.dim[0].m * g.dim[1].m;
    if (src == WSrc::STREAM) expand_kernel<T, 1><<<(unsigned)rows, 128, 0, s>>>(g, vc, coef_in, symin, out);
    else expand_kernel<T, 2><<<(unsigned)rows, 128, 0, s>>>(g, vc, coef_in, symin, out);
    count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_level0(Sink sink, const T *v0, long long N0, T *coef_out, const QuantOut &qo,
                          cudaStream_t s)
{
    unsigned blocks = (unsigned)((N0 + 255) / 256);
    if (sink == Sink::STREAM) level0_kernel<T, 1><<<blocks, 256, 0, s>>>(v0, N0, coef_out, qo);
    else level0_kernel<T, 2><<<blocks, 256, 0, s>>>(v0, N0, coef_out, qo);
    count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_level0_in(WSrc src, const T *coef_in, const SymIn &symin, long long N0, T *v0,
                             cudaStream_t s)
{
    unsigned blocks = (unsigned)((N0 + 255) / 256);
    if (src == WSrc::STREAM) level0_in_kernel<T, 1><<<blocks, 256, 0, s>>>(coef_in, symin, N0, v0);
    else level0_in_kernel<T, 2><<<blocks, 256, 0, s>>>(coef_in, symin, N0, v0);
    count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_norm(const T *u, long long N, double *partials, int nparts, cudaStream_t s)
{
    norm_kernel<T><<<nparts, 256, 0, s>>>(u, N, partials);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_bins(const BinArgs &ba, const double *partials, int nparts, Scalars *sc,
                        cudaStream_t s)
{
    bins_kernel<<<1, 256, 0, s>>>(ba, partials, nparts, sc);
    count_launch();
    return cudaGetLastError();
}

#define INST(T)                                                                                   \
    template cudaError_t launch_restrict<T>(WSrc, Sink, const RestrictArgs<T> &, cudaStream_t);  \
    template cudaError_t launch_solves<T>(const LevelGeom<T> &, T *, T *, int, cudaStream_t);    \
    template cudaError_t launch_expand<T>(WSrc, const LevelGeom<T> &, const T *, const T *,       \
                                          const SymIn &, T *, cudaStream_t);                     \
    template cudaError_t launch_level0<T>(Sink, const T *, long long, T *, const QuantOut &,      \
                                          cudaStream_t);                                         \
    template cudaError_t launch_level0_in<T>(WSrc, const T *, const SymIn &, long long, T *,      \
                                             cudaStream_t);                                      \
    template cudaError_t launch_norm<T>(const T *, long long, double *, int, cudaStream_t);
INST(float)
INST(double)

}  // namespace hpdr
