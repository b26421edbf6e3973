// levels.cu -- per-level pieces of the multilevel decomposition (Sec. IV-A,
// Alg. 1) and of its inverse that are not the plane-streaming level kernels
// (those are in decomp.cu), for sm_103a:
//   * the Thomas solves of the coarse mass matrix along each dimension;
//   * level 0 (quantized or stored as it is) and its inverse;
//   * the norms of the field and the level bins;
//   * coarse_kernel: every level whose arrays fit one CTA's shared memory,
//     and level 0, in a single launch;
//   * the dispatch of restriction requests to the plane pipelines.
#include <cfloat>
#include <type_traits>
#include "levels_dev.cuh"

namespace hpdr {
namespace {

constexpr int kNormBlocks = 152 * 8;

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

// One thread per line, 32 adjacent lines per warp (every step one coalesced
// row), the line swept in place in global memory: the loads of the next sixteen
// steps are in flight while the current sixteen are computed; the Thomas
// factors sit in shared memory.
constexpr int kSolvePre = 16;

template <typename T>
__global__ void __launch_bounds__(256)
solve_stream_kernel(T *b, int n, long long st, long long ostride, long long ninner, long long nlines,
                    const T *__restrict__ sub, const T *__restrict__ cp, const T *__restrict__ inv_den)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *csub = reinterpret_cast<T *>(smem_raw), *ccp = csub + n, *cinv = ccp + n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) { csub[t] = sub[t]; ccp[t] = cp[t]; cinv[t] = inv_den[t]; }
    __syncthreads();
    const long long line = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (line >= nlines) return;
    long long o, i;
    if (ninner == 1) { o = line; i = 0; }
    else if (nlines <= 0xFFFFFFFFll) { o = (unsigned)line / (unsigned)ninner; i = line - o * ninner; }
    else { o = line / ninner; i = line - o * ninner; }     // 64-bit division only for huge grids
    T *p = b + o * ostride + i;
    constexpr int P = kSolvePre;
    const int nfull = n / P;   // blocks of P steps
    // forward sweep: y_t = (d_t - sub_t y_{t-1}) / den_t
    T y = (T)0;
    T cur[P], nxt[P];
    if (nfull > 0) {
#pragma unroll
        for (int u = 0; u < P; u++) cur[u] = p[(long long)u * st];
    }
    for (int k = 0; k < nfull; k++) {
        const int t0 = k * P;
        if (k + 1 < nfull) {
#pragma unroll
            for (int u = 0; u < P; u++) nxt[u] = p[(long long)(t0 + P + u) * st];
        }
#pragma unroll
        for (int u = 0; u < P; u++) {
            y = mul_rn(fma_rn(-csub[t0 + u], y, cur[u]), cinv[t0 + u]);
            p[(long long)(t0 + u) * st] = y;
        }
#pragma unroll
        for (int u = 0; u < P; u++) cur[u] = nxt[u];
    }
    for (int t = nfull * P; t < n; t++) {
        y = mul_rn(fma_rn(-csub[t], y, p[(long long)t * st]), cinv[t]);
        p[(long long)t * st] = y;
    }
    // backward sweep: x_t = y_t - cp_t x_{t+1}, from the end
    T x = (T)0;
    const int ntail = n - nfull * P;
    for (int t = n - 1; t >= n - ntail; t--) {
        x = fma_rn(-ccp[t], x, p[(long long)t * st]);
        p[(long long)t * st] = x;
    }
    if (nfull > 0) {
#pragma unroll
        for (int u = 0; u < P; u++) cur[u] = p[(long long)((nfull - 1) * P + u) * st];
    }
    for (int k = nfull - 1; k >= 0; k--) {
        const int t0 = k * P;
        if (k > 0) {
#pragma unroll
            for (int u = 0; u < P; u++) nxt[u] = p[(long long)(t0 - P + u) * st];
        }
#pragma unroll
        for (int u = P - 1; u >= 0; u--) {
            x = fma_rn(-ccp[t0 + u], x, cur[u]);
            p[(long long)(t0 + u) * st] = x;
        }
#pragma unroll
        for (int u = 0; u < P; u++) cur[u] = nxt[u];
    }
}

template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst_smem, const T *src)
{
    if (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst_smem)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// 32 lines per CTA, staged in shared memory as [n][32]: line i's element t at
// base + t*st + i (the 32 lines are contiguous), so every load and store of a
// step t is one coalesced 128-byte row; one warp then runs the 32 sweeps.
template <typename T>
__global__ void __launch_bounds__(128)
solve_tile_kernel(T *b, int n, long long st, long long ostride, int ninner,
                  const T *__restrict__ sub, const T *__restrict__ cp, const T *__restrict__ inv_den)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *S = reinterpret_cast<T *>(smem_raw);
    T *csub = S + n * 32, *ccp = csub + n, *cinv = ccp + n;   // Thomas factors, staged
    for (int t = threadIdx.x; t < n; t += blockDim.x) { csub[t] = sub[t]; ccp[t] = cp[t]; cinv[t] = inv_den[t]; }
    const int nblk = (ninner + 31) >> 5;
    const long long o = blockIdx.x / nblk;
    const int jb = (int)(blockIdx.x - o * nblk);
    const int nl = min(32, ninner - jb * 32);
    T *base = b + o * ostride + (long long)jb * 32;
    for (int idx = threadIdx.x; idx < n * 32; idx += blockDim.x) {
        const int t = idx >> 5, i = idx & 31;
        if (i < nl) cp_async_elem(&S[idx], base + (long long)t * st + i);
    }
    cp_async_wait_all();
    __syncthreads();
    if ((int)threadIdx.x < nl) {
        T *p = S + threadIdx.x;
        T y = (T)0;
        for (int t = 0; t < n; t++) { y = mul_rn(fma_rn(-csub[t], y, p[t * 32]), cinv[t]); p[t * 32] = y; }
        T x = (T)0;
        for (int t = n - 1; t >= 0; t--) { x = fma_rn(-ccp[t], x, p[t * 32]); p[t * 32] = x; }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * 32; idx += blockDim.x) {
        const int t = idx >> 5, i = idx & 31;
        if (i < nl) base[(long long)t * st + i] = S[idx];
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
solve_contig_kernel(T *b, int n, long long nlines, int rows, int pitch, const T *__restrict__ sub,
                    const T *__restrict__ cp, const T *__restrict__ inv_den, T *vc, int sign)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *S = reinterpret_cast<T *>(smem_raw);
    T *csub = S + (size_t)rows * pitch, *ccp = csub + n, *cinv = ccp + n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) { csub[t] = sub[t]; ccp[t] = cp[t]; cinv[t] = inv_den[t]; }
    const long long row0 = blockIdx.x * (long long)rows;
    const int nr = (int)min((long long)rows, nlines - row0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    // one warp per row: coalesced, no per-element division
    for (int r = warp; r < nr; r += nwarp) {
        const T *srow = b + (row0 + r) * n;
        T *drow = S + r * pitch;
        for (int t = lane; t < n; t += 32) cp_async_elem(&drow[t], srow + t);
    }
    cp_async_wait_all();
    __syncthreads();
    if ((int)threadIdx.x < nr) {
        T *p = S + threadIdx.x * pitch;
        T y = (T)0;
#pragma unroll 8
        for (int t = 0; t < n; t++) { y = mul_rn(fma_rn(-csub[t], y, p[t]), cinv[t]); p[t] = y; }
        T x = (T)0;
#pragma unroll 8
        for (int t = n - 1; t >= 0; t--) { x = fma_rn(-ccp[t], x, p[t]); p[t] = x; }
    }
    __syncthreads();
    if (sign == 0) {
        for (int r = warp; r < nr; r += nwarp) {
            const T *srow = S + r * pitch;
            const long long g0 = (row0 + r) * n;
            for (int t = lane; t < n; t += 32) b[g0 + t] = srow[t];
        }
        return;
    }
    // the read-modify-write of vc: a warp's elements j (row warp + nwarp (j / nk),
    // column lane + 32 (j mod nk)) in batches of U, every load of a batch
    // issued before its stores, so U loads per lane are in flight
    const int nk = (n + 31) / 32;
    const int rows_w = nr > warp ? (nr - warp + nwarp - 1) / nwarp : 0;
    const int nj = rows_w * nk;
    constexpr int U = sizeof(T) == 4 ? 12 : 8;
    for (int j0 = 0; j0 < nj; j0 += U) {
        T old[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int j = j0 + u, q = j / nk, t = lane + 32 * (j - q * nk);
            old[u] = (j < nj && t < n) ? vc[(row0 + warp + (long long)q * nwarp) * n + t] : (T)0;
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int j = j0 + u, q = j / nk, t = lane + 32 * (j - q * nk);
            if (j < nj && t < n) {
                const int r = warp + q * nwarp;
                const T z = S[r * pitch + t];
                const long long g = (row0 + r) * n + t;
                vc[g] = sign > 0 ? add_rn(old[u], z) : sub_rn(old[u], z);
            }
        }
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
    quant_emit(qo, nullptr, false, i, x, rho64_of(qo.sc, 0));
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
    T ssT = (T)0;   // per-thread partial sum in T (binary64 arithmetic is slow on this part)
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
                ssT = fma_rn(e[k], e[k], ssT);
            }
        }
    }
    for (long long i = nv * V + tid; i < N; i += nth) {
        T x = u[i];
        T ax = x < (T)0 ? -x : x;
        nan_max(mx, ax);
        ssT = fma_rn(x, x, ssT);
    }
    ss = (double)ssT;
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
    mx = smx[0];
    ss = sss[0];
    if (threadIdx.x == 0) {
        sc->maxabs = mx;
        sc->sumsq = ss;
    }
    const int L = ba.L;
    bool ok = mx <= DBL_MAX;
    double nrm = ba.mode == 0 ? mx : sqrt(__ddiv_rn(ss, (double)ba.N));
    double tau = ba.tol_kind == 1 ? __dmul_rn(ba.tol, nrm) : ba.tol;
    if (threadIdx.x == 0) sc->tau_abs = tau;
    double tp = 0.0;
    if (ok && mx > 0.0) {
        tp = __dsub_rn(tau, __dmul_rn(__dmul_rn(__dmul_rn(32.0, (double)(L + 1)), ba.eps), mx));
        if (!(tp > 0.0)) ok = false;
    }
    // one level per thread (two FP64 divisions each)
    for (int l = threadIdx.x; l <= L; l += blockDim.x) {
        double q;
        if (!ok || mx == 0.0) q = 1.0;
        else if (l == 0) q = __ddiv_rn(__dmul_rn(2.0, tp), (double)(L + 1));
        else q = __ddiv_rn(__dmul_rn(2.0, tp), __dmul_rn((double)(L + 1), __dadd_rn(1.0, ba.c[l])));
        sc->q[l] = q;
        double r = __ddiv_rn(1.0, q);
        sc->rho_d[l] = r;
        sc->rho_f[l] = __double2float_rn(r);
        sc->rho_lo[l] = __double2float_rn(__dsub_rn(r, (double)sc->rho_f[l]));
        sc->q_f[l] = __double2float_rn(q);
    }
    if (!ok && threadIdx.x == 0) atomicExch(&sc->status, (unsigned int)DS_ARG);
}

// --------------------------------------------------------------------------
// The coarse levels in one CTA.  Every level l <= ls (the largest level whose
// working arrays fit in shared memory) and level 0 run in a single 1024-thread
// block out of shared memory, instead of four or five launches per level.  A
// level of compression (Alg. 1) here:
//   1. v_c = the kept nodes of v, compacted; w = v - P v_c on the new nodes
//      (0 on kept ones), quantized or written to the stream;
//   2. b = (x)_k P^T M_l w, dimension 2, then 1, then 0 (5 taps each);
//   3. z = (x)_k M_{l-1}^{-1} b, Thomas sweeps along dimension 0, 1, then 2;
//   4. v_{l-1} = v_c + z.
// Recomposition runs the levels upwards: w from the stream, b and z as above,
// v_c = v_{l-1} - z, then v = P v_c + w.  P v_c is the multilinear
// interpolant, taken along dimension 2, then 1, then 0.
constexpr int kCoarseThreads = 1024;


// element counts of the shared arrays for top level ls (host and device)
template <typename T>
__host__ __device__ inline void coarse_sizes(const LevelGeom<T> &g, long long &nl, long long &nc, long long &r2,
                                             long long &r1)
{
    const long long m0 = g.dim[0].m, m1 = g.dim[1].m, m2 = g.dim[2].m;
    const long long c0 = g.dim[0].mc, c1 = g.dim[1].mc, c2 = g.dim[2].mc;
    nl = m0 * m1 * m2;
    nc = c0 * c1 * c2;
    r2 = m0 * m1 * c2;
    r1 = m0 * c1 * c2;
}

// multilinear interpolant of the compact coarse array X at fine node (p0, p1, p2)
template <typename T>
__device__ __forceinline__ T coarse_interp(const LevelGeom<T> &g, const T *X, int p0, int p1, int p2)
{
    const int c1 = g.dim[1].mc, c2 = g.dim[2].mc;
    int a[3], b[3];
    bool nw[3];
    const int p[3] = {p0, p1, p2};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const int m = g.dim[k].m, mc = g.dim[k].mc;
        nw[k] = !kept_pos(m, p[k]);
        if (nw[k]) { a[k] = cidx_of(m, mc, p[k] - 1); b[k] = cidx_of(m, mc, p[k] + 1); }
        else { a[k] = b[k] = cidx_of(m, mc, p[k]); }
    }
    auto along2 = [&](int i0, int i1) -> T {
        const T *row = X + ((long long)i0 * c1 + i1) * c2;
        if (!nw[2]) return row[a[2]];
        return fma_rn(g.dim[2].wr[p2], row[b[2]], mul_rn(g.dim[2].wl[p2], row[a[2]]));
    };
    auto along1 = [&](int i0) -> T {
        if (!nw[1]) return along2(i0, a[1]);
        return fma_rn(g.dim[1].wr[p1], along2(i0, b[1]), mul_rn(g.dim[1].wl[p1], along2(i0, a[1])));
    };
    if (!nw[0]) return along1(a[0]);
    return fma_rn(g.dim[0].wr[p0], along1(b[0]), mul_rn(g.dim[0].wl[p0], along1(a[0])));
}

// out = in restricted along dimension k with the 5 taps of P^T M_l; in has
// extents n[3] (n[k] = m), out the same with n[k] = mc
template <typename T>
__device__ void coarse_restrict(const DimTables<T> &d, int k, const int n[3], const T *in, T *out)
{
    int o[3] = {n[0], n[1], n[2]};
    o[k] = d.mc;
    const long long tot = (long long)o[0] * o[1] * o[2];
    const long long is[3] = {(long long)n[1] * n[2], n[2], 1};
    for (long long idx = threadIdx.x; idx < tot; idx += blockDim.x) {
        const int j2 = (int)(idx % o[2]);
        const long long r = idx / o[2];
        const int j1 = (int)(r % o[1]), j0 = (int)(r / o[1]);
        const int jj[3] = {j0, j1, j2};
        if (d.m <= 1) { out[idx] = in[j0 * is[0] + j1 * is[1] + j2]; continue; }
        const int jk = jj[k];
        const int c = cpos_of(d.m, d.mc, jk);
        long long base = 0;
#pragma unroll
        for (int q = 0; q < 3; q++) if (q != k) base += jj[q] * is[q];
        T acc = (T)0;
#pragma unroll
        for (int t = 0; t < 5; t++) {
            const int pos = c - 2 + t;
            if (pos < 0 || pos >= d.m) continue;
            acc = fma_rn(d.tap[jk * 5 + t], in[base + pos * is[k]], acc);
        }
        out[idx] = acc;
    }
}

// Thomas sweeps of (x)_k M_{l-1} on the compact coarse array B (extents c[3]), in place
template <typename T>
__device__ void coarse_solves(const LevelGeom<T> &g, const int c[3], T *B)
{
    for (int k = 0; k < 3; k++) {
        const DimTables<T> &d = g.dim[k];
        if (!(d.m > 1)) continue;
        const long long st = k == 0 ? (long long)c[1] * c[2] : k == 1 ? c[2] : 1;
        const int oa = k == 0 ? c[1] : c[0], ob = k == 2 ? c[1] : c[2];
        for (int line = threadIdx.x; line < oa * ob; line += blockDim.x) {
            const int u = line / ob, v = line - u * ob;
            long long base;
            if (k == 0) base = (long long)u * c[2] + v;
            else if (k == 1) base = (long long)u * c[1] * c[2] + v;
            else base = ((long long)u * c[1] + v) * c[2];
            T *p = B + base;
            const int n = d.mc;
            T y = (T)0;
            for (int t = 0; t < n; t++) { y = mul_rn(fma_rn(-d.sub[t], y, p[t * st]), d.inv_den[t]); p[t * st] = y; }
            T x = (T)0;
            for (int t = n - 1; t >= 0; t--) { x = fma_rn(-d.cp[t], x, p[t * st]); p[t * st] = x; }
        }
        __syncthreads();
    }
}

// b = (x)_k P^T M_l W into B (R2, R1 scratch)
template <typename T>
__device__ void coarse_rhs(const LevelGeom<T> &g, const T *W, T *R2, T *R1, T *B)
{
    const int m[3] = {g.dim[0].m, g.dim[1].m, g.dim[2].m};
    const int n2[3] = {m[0], m[1], m[2]};
    coarse_restrict<T>(g.dim[2], 2, n2, W, R2);
    __syncthreads();
    const int n1[3] = {m[0], m[1], g.dim[2].mc};
    coarse_restrict<T>(g.dim[1], 1, n1, R2, R1);
    __syncthreads();
    const int n0[3] = {m[0], g.dim[1].mc, g.dim[2].mc};
    coarse_restrict<T>(g.dim[0], 0, n0, R1, B);
    __syncthreads();
}

// MODE 0: compression (quantize), 1: decomposition (coefficient stream),
// 2: decompression (symbols), 3: recomposition (coefficient stream)
template <typename T, int MODE>
__device__ __forceinline__ void coarse_body(const CoarseArgs<T> &a)
{
    extern __shared__ __align__(16) unsigned char coarse_smem[];
    long long nl, nc, r2, r1;
    coarse_sizes<T>(a.g[a.ls], nl, nc, r2, r1);
    T *VA = reinterpret_cast<T *>(coarse_smem);   // [nl]
    T *VB = VA + nl;                                // [nc]
    T *W = VB + nc;                                 // [nl]
    T *R2 = W + nl;                                 // [r2]
    T *R1 = R2 + r2;                                // [r1]
    T *B = R1 + r1;                                 // [nc]
    T *VK = B + nc;                                 // [nc]
    const int tid = threadIdx.x;
    if (MODE <= 1) {
        for (long long i = tid; i < nl; i += blockDim.x) VA[i] = a.v_in[i];
        __syncthreads();
        T *V = VA, *Vn = VB;
        for (int l = a.ls; l >= 1; l--) {
            const LevelGeom<T> &g = a.g[l];
            const int m1 = g.dim[1].m, m2 = g.dim[2].m;
            const int c[3] = {g.dim[0].mc, g.dim[1].mc, g.dim[2].mc};
            const long long n = (long long)g.dim[0].m * m1 * m2, ncl = (long long)c[0] * c[1] * c[2];
            // 1. kept nodes, compacted
            for (long long j = tid; j < ncl; j += blockDim.x) {
                const int j2 = (int)(j % c[2]);
                const long long r = j / c[2];
                const int j1 = (int)(r % c[1]), j0 = (int)(r / c[1]);
                const long long f = ((long long)cpos_of(g.dim[0].m, c[0], j0) * m1 + cpos_of(m1, c[1], j1)) * m2 +
                                    cpos_of(m2, c[2], j2);
                VK[j] = V[f];
            }
            __syncthreads();
            //    coefficients of the new nodes
            const double rho = MODE == 0 ? rho64_of(a.qo.sc, l) : 0.0;
            for (long long i = tid; i < n; i += blockDim.x) {
                const int p2 = (int)(i % m2);
                const long long r = i / m2;
                const int p1 = (int)(r % m1), p0 = (int)(r / m1);
                if (kept_pos(g.dim[0].m, p0) && kept_pos(m1, p1) && kept_pos(m2, p2)) { W[i] = (T)0; continue; }
                const T w = sub_rn(V[i], coarse_interp<T>(g, VK, p0, p1, p2));
                W[i] = w;
                const long long si = stream_rank(g, p0, p1, p2);
                if (MODE == 0) quant_emit(a.qo, nullptr, false, si, w, rho);
                else a.coef_out[si] = w;
            }
            __syncthreads();
            // 2.-3.
            coarse_rhs<T>(g, W, R2, R1, B);
            coarse_solves<T>(g, c, B);
            // 4.
            for (long long j = tid; j < ncl; j += blockDim.x) Vn[j] = add_rn(VK[j], B[j]);
            __syncthreads();
            T *t = V; V = Vn; Vn = t;
        }
        // level 0
        const double rho0 = MODE == 0 ? rho64_of(a.qo.sc, 0) : 0.0;
        for (long long i = tid; i < a.N0; i += blockDim.x) {
            if (MODE == 0) quant_emit(a.qo, nullptr, false, i, V[i], rho0);
            else a.coef_out[i] = V[i];
        }
    } else {
        T *V = VA, *Vn = VB;
        // the same ping-pong as compression, run backwards: level l's grid lands
        // where compression read it (the top level in VA)
        if ((a.ls & 1) == 1) { V = VB; Vn = VA; }
        const T q0 = MODE == 2 ? q_of<T>(a.symin.sc, 0) : (T)0;
        for (long long i = tid; i < a.N0; i += blockDim.x)
            V[i] = MODE == 2 ? dequant_sym<T>(a.symin, a.symin.sym[i], i, q0) : a.coef_in[i];
        __syncthreads();
        for (int l = 1; l <= a.ls; l++) {
            const LevelGeom<T> &g = a.g[l];
            const int m1 = g.dim[1].m, m2 = g.dim[2].m;
            const int c[3] = {g.dim[0].mc, g.dim[1].mc, g.dim[2].mc};
            const long long n = (long long)g.dim[0].m * m1 * m2, ncl = (long long)c[0] * c[1] * c[2];
            const T q = MODE == 2 ? q_of<T>(a.symin.sc, l) : (T)0;
            for (long long i = tid; i < n; i += blockDim.x) {
                const int p2 = (int)(i % m2);
                const long long r = i / m2;
                const int p1 = (int)(r % m1), p0 = (int)(r / m1);
                if (kept_pos(g.dim[0].m, p0) && kept_pos(m1, p1) && kept_pos(m2, p2)) { W[i] = (T)0; continue; }
                const long long si = stream_rank(g, p0, p1, p2);
                W[i] = MODE == 2 ? dequant_sym<T>(a.symin, a.symin.sym[si], si, q) : a.coef_in[si];
            }
            __syncthreads();
            coarse_rhs<T>(g, W, R2, R1, B);
            coarse_solves<T>(g, c, B);
            for (long long j = tid; j < ncl; j += blockDim.x) VK[j] = sub_rn(V[j], B[j]);
            __syncthreads();
            for (long long i = tid; i < n; i += blockDim.x) {
                const int p2 = (int)(i % m2);
                const long long r = i / m2;
                const int p1 = (int)(r % m1), p0 = (int)(r / m1);
                const bool kept = kept_pos(g.dim[0].m, p0) && kept_pos(m1, p1) && kept_pos(m2, p2);
                Vn[i] = kept ? VK[((long long)cidx_of(g.dim[0].m, c[0], p0) * c[1] + cidx_of(m1, c[1], p1)) * c[2] +
                                  cidx_of(m2, c[2], p2)]
                             : add_rn(W[i], coarse_interp<T>(g, VK, p0, p1, p2));
            }
            __syncthreads();
            T *t = V; V = Vn; Vn = t;
        }
        for (long long i = tid; i < nl; i += blockDim.x) a.v_out[i] = V[i];
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kCoarseThreads, 1) coarse_kernel(CoarseArgs<T> a)
{
    coarse_body<T, MODE>(a);
}

// one field per block
template <typename T, int MODE>
__global__ void __launch_bounds__(kCoarseThreads, 1) coarse_batch_kernel(const CoarseArgs<T> *jobs)
{
    coarse_body<T, MODE>(jobs[blockIdx.x]);
}

}  // namespace

int norm_parts() { return kNormBlocks; }

// Coarse planes per CTA (segment) for a grid of `tiles` x segments CTAs:
// fill whole waves of the resident CTAs (per_sm per SM) while keeping the
// dim-0 halo (two fine planes each side of a segment) small.
int choose_segment(int mc0, long long tiles, int per_sm)
{
    const int nsm = sm_count();
    const long long slots = (long long)nsm * std::max(1, per_sm);
    double best = -1.0;
    int best_seg = mc0;
    for (int gz = 1; gz <= mc0 && gz <= 512; gz++) {
        const int seg = (mc0 + gz - 1) / gz;
        const long long ctas = tiles * ((mc0 + seg - 1) / seg);
        const long long waves = (ctas + slots - 1) / slots;
        const double score = (double)ctas / (double)(waves * slots) * (2.0 * seg) / (2.0 * seg + 4.0);
        if (score > best + 1e-9) { best = score; best_seg = seg; }
    }
    return best_seg;
}


template <typename T>
cudaError_t launch_restrict(WSrc src, Sink sink, const RestrictArgs<T> &a, cudaStream_t s)
{
    // the field source (compression, decomposition) and the decompression-side
    // sources (symbols, a coefficient stream, a dense level grid) run in the
    // warp-specialised plane pipelines of decomp.cu
    if (src == WSrc::FIELD) return launch_decomp<T>(sink, a, s);
    return launch_restrict_planes<T>(src, a, s);
}

constexpr bool kSolveStream = true;   // strided dimensions: streaming sweeps

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
        // the streaming sweep keeps the three factor tables in shared memory
        // (at most the default 48 KB); longer lines take the strided kernel
        if (k < 2 && sg == 0 && kSolveStream && 3 * (size_t)d.mc * sizeof(T) <= 48 * 1024) {
            // dim 0: lines (j1, j2), step c1*c2; dim 1: lines (j0, j2), step c2
            const long long st = (k == 0) ? c1 * c2 : c2;
            const long long outer = (k == 0) ? c1 : c0;
            const long long ostride = (k == 0) ? c2 : c1 * c2;
            const long long nlines = outer * c2;
            solve_stream_kernel<T><<<(unsigned)((nlines + 255) / 256), 256, 3 * (size_t)d.mc * sizeof(T), s>>>(
                b, d.mc, st, ostride, c2, nlines, d.sub, d.cp, d.inv_den);
        } else if (k < 2 && sg == 0 && (size_t)d.mc * 35 * sizeof(T) <= 160 * 1024) {
            // dim 0: lines (j1, j2), step c1*c2; dim 1: lines (j0, j2), step c2
            const long long st = (k == 0) ? c1 * c2 : c2;
            const long long outer = (k == 0) ? c1 : c0;
            const long long ostride = (k == 0) ? c2 : c1 * c2;
            const int ninner = (int)c2;
            static PerDeviceOnce attr;
            cudaError_t ea = once_per_device(attr, [] {
                return cudaFuncSetAttribute(solve_tile_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            164 * 1024);
            });
            if (ea != cudaSuccess) return ea;
            const long long grid = outer * ((ninner + 31) / 32);
            solve_tile_kernel<T><<<(unsigned)grid, 128, (size_t)d.mc * 35 * sizeof(T), s>>>(
                b, d.mc, st, ostride, ninner, d.sub, d.cp, d.inv_den);
        } else if (k < 2) {
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
            // the row tile and the three factor tables share the 100 KB limit
            const size_t tab = 3 * (size_t)n * sizeof(T);
            const size_t budget = std::min<size_t>(90 * 1024, tab < 100 * 1024 ? 100 * 1024 - tab : 0);
            int rows = (int)std::min<size_t>(64, budget / rowbytes);
            if (rows < 1) {
                solve_strided_kernel<T><<<(unsigned)((nlines + 255) / 256), 256, 0, s>>>(
                    b, n, 1, nlines, d.sub, d.cp, d.inv_den, vc, sg);
            } else {
                static PerDeviceOnce attr;
                cudaError_t ea = once_per_device(attr, [] {
                    return cudaFuncSetAttribute(solve_contig_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                100 * 1024);
                });
                if (ea != cudaSuccess) return ea;
                solve_contig_kernel<T><<<(unsigned)((nlines + rows - 1) / rows), 256,
                                         rows * rowbytes + 3 * (size_t)n * sizeof(T), s>>>(
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
    return launch_expand_planes<T>(src, g, vc, coef_in, symin, out, s);
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


template <typename T>
size_t coarse_smem_bytes(const LevelGeom<T> &g)
{
    long long nl, nc, r2, r1;
    coarse_sizes<T>(g, nl, nc, r2, r1);
    return (size_t)(2 * nl + 3 * nc + r2 + r1) * sizeof(T);
}

template <typename T>
int coarse_top(const Plan *P, const LevelGeom<T> *geo)
{
    int ls = 0;
    for (int l = 1; l <= P->L && l <= kCoarseMaxLevels; l++)
        if (coarse_smem_bytes<T>(geo[l]) <= kCoarseSmem) ls = l;
        else break;
    return ls;
}

template <typename T>
CoarseArgs<T> coarse_args(const Plan *P, const LevelGeom<T> *geo, int ls, const T *v_in, T *v_out,
                          const QuantOut &qo, T *coef_out, const SymIn &symin, const T *coef_in, size_t *smem)
{
    CoarseArgs<T> a;
    memset(&a, 0, sizeof(a));
    for (int l = 1; l <= ls && l <= kCoarseMaxLevels; l++) a.g[l] = geo[l];
    a.ls = ls;
    a.N0 = P->N[0];
    a.v_in = v_in; a.v_out = v_out; a.qo = qo; a.coef_out = coef_out; a.symin = symin; a.coef_in = coef_in;
    if (smem) *smem = ls >= 1 && ls <= kCoarseMaxLevels ? coarse_smem_bytes<T>(geo[ls]) : 0;
    return a;
}

template <typename T>
cudaError_t launch_coarse_batch(int mode, const CoarseArgs<T> *jobs, int n, size_t smem, cudaStream_t s)
{
    if (n < 1) return cudaSuccess;
    static PerDeviceOnce attr[4];
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e = once_per_device(attr[mode & 3], [&] {
            return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCoarseSmem);
        });
        if (e != cudaSuccess) return e;
        kern<<<n, kCoarseThreads, smem, s>>>(jobs);
        count_launch();
        return cudaGetLastError();
    };
    switch (mode) {
    case 0: return go(coarse_batch_kernel<T, 0>);
    case 1: return go(coarse_batch_kernel<T, 1>);
    case 2: return go(coarse_batch_kernel<T, 2>);
    default: return go(coarse_batch_kernel<T, 3>);
    }
}

template <typename T>
cudaError_t launch_coarse(int mode, const Plan *P, const LevelGeom<T> *geo, int ls, const T *v_in, T *v_out,
                          const QuantOut &qo, T *coef_out, const SymIn &symin, const T *coef_in, cudaStream_t s)
{
    if (ls < 1 || ls > kCoarseMaxLevels) return cudaErrorInvalidValue;
    size_t sm = 0;
    const CoarseArgs<T> a = coarse_args<T>(P, geo, ls, v_in, v_out, qo, coef_out, symin, coef_in, &sm);
    static PerDeviceOnce attr[4];
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e = once_per_device(attr[mode], [&] {
            return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCoarseSmem);
        });
        if (e != cudaSuccess) return e;
        kern<<<1, kCoarseThreads, sm, s>>>(a);
        count_launch();
        return cudaGetLastError();
    };
    switch (mode) {
    case 0: return go(coarse_kernel<T, 0>);
    case 1: return go(coarse_kernel<T, 1>);
    case 2: return go(coarse_kernel<T, 2>);
    default: return go(coarse_kernel<T, 3>);
    }
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
    template cudaError_t launch_norm<T>(const T *, long long, double *, int, cudaStream_t);      \
    template int coarse_top<T>(const Plan *, const LevelGeom<T> *);                              \
    template cudaError_t launch_coarse<T>(int, const Plan *, const LevelGeom<T> *, int, const T *, T *, \
                                          const QuantOut &, T *, const SymIn &, const T *, cudaStream_t); \
    template CoarseArgs<T> coarse_args<T>(const Plan *, const LevelGeom<T> *, int, const T *, T *,         \
                                          const QuantOut &, T *, const SymIn &, const T *, size_t *);      \
    template cudaError_t launch_coarse_batch<T>(int, const CoarseArgs<T> *, int, size_t, cudaStream_t);
INST(float)
INST(double)

}  // namespace hpdr
