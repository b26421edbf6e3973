// adjoint.cu -- transposes of recomposition and decomposition (the maps are
// linear, so backward passes need no saved forward state).
//
// One level of recomposition is  v_l = P (v_{l-1} - S c_l) + E_new c_l  with
// S = (x)M_{l-1}^{-1} (x)P^T M_l E_new; its transpose, from the level-l
// gradient g_l, is
//     g_{l-1} = P^T g_l,      g_{c_l} = g_l|new - E_new^T ((x)M_l P) (x)M_{l-1}^{-1} P^T g_l.
// One level of decomposition is  c_l = (v - P v|kept)|new,
// v_{l-1} = v|kept + S c_l; its transpose, from g_{c_l} and g_{v_{l-1}}, is
//     h = g_{c_l} + E_new^T ((x)M_l P) (x)M_{l-1}^{-1} g_{v_{l-1}},
//     g_{v_l} = E_new h + E_kept (g_{v_{l-1}} - P^T E_new h).
// P^T is the restriction kernel with the interpolation taps, M_{l-1}^{-1} the
// Thomas solves, and (x)M_l P is applied one dimension at a time below.
#include <cstring>
#include "internal.cuh"
#include "levels.cuh"

namespace hpdr {
namespace {

enum { MP_PLAIN = 0, MP_RT_FINAL = 1, MP_DT_FINAL = 2 };

// out (dims s0 x s1 x s2) = (M_l P) along dim k of in (dim k of size mc_k).
// Final modes (k = 0, output on the level-l grid):
//   MP_RT_FINAL: stream[rank(p)] = gsrc[p] - value   at the new nodes
//   MP_DT_FINAL: out[p] = coef[rank(p)] + value       at the new nodes
// One warp per output row (i0, i1), lanes along i2: the row's dimension-0
// and dimension-1 indices, the taps of a dimension-0 or -1 pass and, in the
// final modes, whether the row holds only new nodes and where its new nodes
// start in the stream are computed once per row; every load and store is
// coalesced along i2 (the kept rows of a kept plane write every other stream
// slot: only odd i2 are new there).
constexpr int kMpWarps = 8;
template <typename T, int MODE>
__global__ void __launch_bounds__(32 * kMpWarps)
mass_prolong_kernel(const T *__restrict__ in, T *__restrict__ out, long long s0, long long s1, long long s2, int k,
                    int mck, const T *__restrict__ etap, const int *__restrict__ efirst, LevelGeom<T> g,
                    const T *__restrict__ gsrc, T *__restrict__ stream, const T *__restrict__ coef)
{
    const long long rows = s0 * s1;
    const long long in1 = (k == 1) ? mck : s1, in2 = (k == 2) ? mck : s2;
    const int lane = threadIdx.x & 31;
    for (long long row = blockIdx.x * (long long)kMpWarps + (threadIdx.x >> 5); row < rows;
         row += (long long)gridDim.x * kMpWarps) {
        const long long i0 = row / s1, i1 = row - i0 * s1;
        // dimension-0 or -1 pass: the row's taps
        int rj0 = 0;
        T rt[3] = {(T)0, (T)0, (T)0};
        if (k != 2) {
            const long long pr = (k == 0) ? i0 : i1;
            rj0 = efirst[pr];
#pragma unroll
            for (int i = 0; i < 3; i++) rt[i] = etap[pr * 3 + i];
        }
        bool rownew = true;
        long long sbase = 0;
        if (MODE != MP_PLAIN) {
            const int p0 = (int)i0, p1 = (int)i1;
            const bool k0 = kept_pos(g.dim[0].m, p0), k1 = kept_pos(g.dim[1].m, p1);
            rownew = !k0 || !k1;
            long long cr = (long long)kept_before(p0) * g.dim[1].mc * g.dim[2].mc;
            if (k0) cr += (long long)kept_before(p1) * g.dim[2].mc;
            sbase = g.Nprev + row * s2 - cr;
        }
        // four columns per lane in flight (the buffers do not alias)
#pragma unroll 4
        for (long long i2 = lane; i2 < s2; i2 += 32) {
            const long long idx = row * s2 + i2;
            int j0;
            T tp[3];
            if (k == 2) {
                j0 = efirst[i2];
#pragma unroll
                for (int i = 0; i < 3; i++) tp[i] = etap[i2 * 3 + i];
            } else {
                j0 = rj0;
#pragma unroll
                for (int i = 0; i < 3; i++) tp[i] = rt[i];
            }
            T v = (T)0;
#pragma unroll
            for (int i = 0; i < 3; i++) {
                const int j = j0 + i;
                if (j < mck) {
                    const long long a0 = (k == 0) ? j : i0, a1 = (k == 1) ? j : i1, a2 = (k == 2) ? j : i2;
                    v = fma_rn(tp[i], in[(a0 * in1 + a1) * in2 + a2], v);
                }
            }
            if (MODE == MP_PLAIN) {
                out[idx] = v;
            } else {
                const int p2 = (int)i2;
                if (!rownew && kept_pos(g.dim[2].m, p2)) continue;
                const long long si = sbase + i2 - (rownew ? 0 : kept_before(p2));
                if (MODE == MP_RT_FINAL) stream[si] = sub_rn(gsrc[idx], v);
                else out[idx] = add_rn(coef[si], v);
            }
        }
    }
}

// decompose transpose: G(kept node of coarse q) = gv[q] - R[q]
template <typename T>
__global__ void set_kept_kernel(T *G, const T *gv, const T *R, LevelGeom<T> g)
{
    const long long c1 = g.dim[1].mc, c2 = g.dim[2].mc;
    const long long n = (long long)g.dim[0].mc * c1 * c2;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        long long q0, q1, q2;
        if (n < (1LL << 31)) {   // 32-bit divisions
            const unsigned u = (unsigned)q, t = u / (unsigned)c2;
            q2 = u - t * (unsigned)c2;
            q0 = t / (unsigned)c1;
            q1 = t - (unsigned)q0 * (unsigned)c1;
        } else {
            const long long t = q / c2;
            q2 = q - t * c2;
            q1 = t % c1;
            q0 = t / c1;
        }
        const long long p0 = cpos_of(g.dim[0].m, g.dim[0].mc, (int)q0);
        const long long p1 = cpos_of(g.dim[1].m, g.dim[1].mc, (int)q1);
        const long long p2 = cpos_of(g.dim[2].m, g.dim[2].mc, (int)q2);
        G[(p0 * g.dim[1].m + p1) * g.dim[2].m + p2] = sub_rn(gv[q], R[q]);
    }
}

template <typename T>
__global__ void copy_kernel(T *dst, const T *src, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

unsigned grid_for(long long n) { return (unsigned)std::min<long long>((n + 255) / 256, 152LL * 16); }
// rows of kMpWarps warps per block, capped at 16 blocks per SM
unsigned grid_rows(long long rows) { return (unsigned)std::min<long long>((rows + kMpWarps - 1) / kMpWarps, 152LL * 16); }

// y_f = (x)_k M_l P_k y, the last dimension-0 pass in a final mode
template <typename T, int MODE>
cudaError_t mass_prolong_all(const LevelGeom<T> &g, const T *y, T *t1, T *t2, T *out, const T *gsrc,
                             T *stream, const T *coef, cudaStream_t s)
{
    const long long m0 = g.dim[0].m, m1 = g.dim[1].m, m2 = g.dim[2].m;
    const long long c0 = g.dim[0].mc, c1 = g.dim[1].mc;
    // dim 2: c0 x c1 x c2 -> c0 x c1 x m2
    constexpr int B = 32 * kMpWarps;
    mass_prolong_kernel<T, MP_PLAIN><<<grid_rows(c0 * c1), B, 0, s>>>(y, t1, c0, c1, m2, 2, g.dim[2].mc, g.dim[2].etap,
                                                                     g.dim[2].efirst, g, nullptr, nullptr, nullptr);
    // dim 1: -> c0 x m1 x m2
    mass_prolong_kernel<T, MP_PLAIN><<<grid_rows(c0 * m1), B, 0, s>>>(t1, t2, c0, m1, m2, 1, g.dim[1].mc, g.dim[1].etap,
                                                                     g.dim[1].efirst, g, nullptr, nullptr, nullptr);
    // dim 0: -> m0 x m1 x m2, final
    mass_prolong_kernel<T, MODE><<<grid_rows(m0 * m1), B, 0, s>>>(t2, out, m0, m1, m2, 0, g.dim[0].mc, g.dim[0].etap,
                                                                 g.dim[0].efirst, g, gsrc, stream, coef);
    count_launch(3);
    return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t recompose_adjoint_run(const Plan &P, const LevelGeom<T> *geo, const T *gu, T *gcoef, T *ga, T *gb,
                                  T *y, T *t1, T *t2, unsigned *status, cudaStream_t s)
{
    const int L = P.L;
    const T *gl = gu;
    for (int l = L; l >= 1; l--) {
        const LevelGeom<T> &g = geo[l];
        T *gc = ((L - l) % 2 == 0) ? ga : gb;   // g_{l-1} = P^T g_l
        RestrictArgs<T> a;
        memset(&a, 0, sizeof(a));
        a.g = g;
        a.v = gl;
        a.use_ptap = 1;
        a.dense_new_only = 0;
        a.b = gc;
        a.status = status;
        cudaError_t e = launch_restrict<T>(WSrc::DENSE, Sink::NONE, a, s);
        if (e != cudaSuccess) return e;
        const long long nc = P.N[l - 1];
        copy_kernel<T><<<grid_for(nc), 256, 0, s>>>(y, gc, nc);
        count_launch();
        e = launch_solves<T>(g, y, nullptr, 0, s);
        if (e != cudaSuccess) return e;
        e = mass_prolong_all<T, MP_RT_FINAL>(g, y, t1, t2, nullptr, gl, gcoef, nullptr, s);
        if (e != cudaSuccess) return e;
        gl = gc;
    }
    copy_kernel<T><<<grid_for(P.N[0]), 256, 0, s>>>(gcoef, gl, P.N[0]);
    count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t decompose_adjoint_run(const Plan &P, const LevelGeom<T> *geo, const T *gcoef, T *gu, T *ga, T *gb,
                                  T *y, T *t1, T *t2, T *R, unsigned *status, cudaStream_t s)
{
    const int L = P.L;
    T *gv = (L == 0) ? gu : ((L % 2 == 1) ? ga : gb);
    copy_kernel<T><<<grid_for(P.N[0]), 256, 0, s>>>(gv, gcoef, P.N[0]);
    count_launch();
    for (int l = 1; l <= L; l++) {
        const LevelGeom<T> &g = geo[l];
        T *G = (l == L) ? gu : (((L - l) % 2 == 1) ? ga : gb);
        const long long nc = P.N[l - 1];
        copy_kernel<T><<<grid_for(nc), 256, 0, s>>>(y, gv, nc);
        count_launch();
        cudaError_t e = launch_solves<T>(g, y, nullptr, 0, s);
        if (e != cudaSuccess) return e;
        // new nodes: G = h = g_c + ((x)M_l P) y
        e = mass_prolong_all<T, MP_DT_FINAL>(g, y, t1, t2, G, nullptr, nullptr, gcoef, s);
        if (e != cudaSuccess) return e;
        // kept nodes: G = gv - P^T E_new h
        RestrictArgs<T> a;
        memset(&a, 0, sizeof(a));
        a.g = g;
        a.v = G;
        a.use_ptap = 1;
        a.dense_new_only = 1;
        a.b = R;
        a.status = status;
        e = launch_restrict<T>(WSrc::DENSE, Sink::NONE, a, s);
        if (e != cudaSuccess) return e;
        set_kept_kernel<T><<<grid_for(nc), 256, 0, s>>>(G, gv, R, g);
        count_launch();
        gv = G;
    }
    return cudaGetLastError();
}

template cudaError_t recompose_adjoint_run<float>(const Plan &, const LevelGeom<float> *, const float *, float *,
                                                  float *, float *, float *, float *, float *, unsigned *,
                                                  cudaStream_t);
template cudaError_t recompose_adjoint_run<double>(const Plan &, const LevelGeom<double> *, const double *,
                                                   double *, double *, double *, double *, double *, double *,
                                                   unsigned *, cudaStream_t);
template cudaError_t decompose_adjoint_run<float>(const Plan &, const LevelGeom<float> *, const float *, float *,
                                                  float *, float *, float *, float *, float *, float *,
                                                  unsigned *, cudaStream_t);
template cudaError_t decompose_adjoint_run<double>(const Plan &, const LevelGeom<double> *, const double *,
                                                   double *, double *, double *, double *, double *, double *,
                                                   double *, unsigned *, cudaStream_t);

}  // namespace hpdr
