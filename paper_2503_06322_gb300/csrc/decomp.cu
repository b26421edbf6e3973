// decomp.cu -- the two level kernels that move most of the bytes, for sm_103a:
//
//   decomp_kernel  one level of the multilevel decomposition of a field
//                  (Sec. IV-A, Alg. 1): the new-node coefficients
//                  mc_l = v - lerp(v), handed to a sink (quantization with
//                  the level's bin, the block histogram of Alg. 2 and the
//                  symbol store; or a coefficient store), the coarse copy v_c
//                  and the coarse right-hand side of the correction
//                  (mass_trans);
//   rsym_kernel    the restriction of the inverse direction: the dequantized
//                  symbols of one level through the same mass_trans
//                  (decompression), a level of a coefficient stream
//                  (recomposition), or a dense level grid, all or only its
//                  new nodes, through P^T M_l or P^T (the adjoints).
//
// Both are warp-specialised plane pipelines.  A CTA owns a tile of 14 x 32
// coarse nodes in dims (1, 2) and a segment of coarse planes of dim 0.  One
// producer warp streams the fine planes of the tile's region (the owned
// nodes plus a two-node halo) into a ring of shared-memory stages, one bulk
// asynchronous copy per row, completed on a "full" mbarrier per stage; seven
// consumer warps compute and hand each stage back on an "empty" mbarrier.
// Two CTAs of eight warps per SM leave each SM sub-partition four warps, so
// a thread may hold 128 registers.
// Every wait is bounded; a wait that runs out sets DS_TIMEOUT, the consumers
// leave their plane loop and the producer waits (with a long bound of its
// own) for every copy still in flight before the CTA exits.
//
// Consumer warp c owns coarse rows j1a = J1 + 2c and j1b = j1a + 1, lane l
// coarse column j2 = J2 + l.  For every staged plane p the lane forms the
// dim-2 restriction of the seven fine rows its two outputs need, then the
// dim-1 restriction, and accumulates the dim-0 taps of p in registers, so
// only b (1/8 of the level) is written.  decomp_kernel uses the Galerkin
// identity P^T M_l P = M_{l-1} of nested P1 spaces,
//     b = P^T M_l (v - P v_c) = ((x)_k P^T M_l) v - ((x)_k M_{l-1}) v_c,
// so it restricts the staged values of v directly and no warp needs another
// warp's coefficients: the consumers run without block barriers.  The
// coefficients of the lane's own 2 x 2 nodes per owned row pair take the
// multilinear interpolant of the kept planes around them; the interpolant
// J = I_1 I_2 v of a kept plane is formed once, while that plane is staged,
// and kept in registers for the new plane after it.
//
// Nothing depends on the tiling: every output sums its taps in a fixed order
// fixed by its global index, so batched, streamed and plain calls agree bit
// for bit, and decomposition (coefficient sink) and compression (quantizing
// sink) compute the same coefficients.
#include <type_traits>
#include "levels_dev.cuh"

namespace hpdr {

int g_wait_limit = kWaitPolls;

namespace {

constexpr int DCW = 7;                     // consumer warps, two coarse rows each
constexpr int DT1 = 2 * DCW, DT2 = 32;     // coarse tile, dims 1 and 2
constexpr int DTHREADS = (DCW + 1) * 32;   // plus one producer warp
constexpr int DR1 = 2 * DT1 + 4;           // largest region: fine rows
constexpr int DR2 = 2 * DT2 + 4;           //                 fine columns
constexpr int kHistWin = 4096;             // shared histogram: D/2 +- kHistWin and the escape symbol
// zero rows before the first stage and after the last: the window rows of a
// warp at the edge of the grid may lie up to two rows outside the region
template <typename E> __host__ __device__ constexpr int stage_pitch();
template <typename E> __host__ __device__ constexpr int guard_bytes() { return 3 * stage_pitch<E>(); }

template <typename T> __host__ __device__ constexpr int decomp_stages() { return sizeof(T) == 4 ? 6 : 3; }
template <typename T> __host__ __device__ constexpr int rsym_stages() { return 6; }
// bytes per staged row: the region plus the 16-byte alignment of its copy
template <typename E> __host__ __device__ constexpr int stage_pitch() { return ((DR2 * (int)sizeof(E) + 32) + 15) & ~15; }

// floats (or doubles) per row of the dequantized tile of rsym_kernel
constexpr int kWPitch = DR2 + 8;

// the interpolant of a kept plane at a lane's owned nodes: four owned rows,
// columns Ca and Ca + 1
template <typename T>
struct Interp {
    T v[4][2];
};

// dim-0 data of one staged plane, written by the producer
template <typename T>
struct PlaneInfo {
    int jlo;     // first coarse plane whose five-tap window holds the plane
    int pad;
    T tr[3];     // restriction taps toward coarse planes jlo..jlo+2 (0 outside the segment)
    T tm[3];     // coarse mass-matrix taps (kept planes; 0 otherwise)
    T wl, wr;    // interpolation weights of a new plane
};

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// A bounded wait that the whole warp agrees on.  Each poll suspends the warp
// for up to kSleepNs (it resumes as soon as the phase completes), so waiting
// costs no issue slots; `limit` polls bound the wait (kWaitPolls polls of
// 2 us: about two seconds).
constexpr uint32_t kSleepNs = 2000;
__device__ __forceinline__ bool wait_sleep_bounded(unsigned long long *bar, uint32_t parity, int limit)
{
    for (int i = 0; i < limit; i++)
        if (mbar_try_wait_sleep(bar, parity, kSleepNs)) return true;
    return false;
}
__device__ __forceinline__ bool warp_wait(unsigned long long *bar, uint32_t parity, int limit)
{
    const bool ok = wait_sleep_bounded(bar, parity, limit);
    return __all_sync(0xffffffffu, ok);
}
__device__ __forceinline__ void named_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}


// Geometry of one CTA, common to both kernels.
struct TileGeom {
    int J2, J1, J0a, J0b, n2, n1;
    int lo0, hi0, lo1, hi1, lo2, hi2, r1n, r2n;
    int o0a, o0b;   // owned fine planes [o0a, o0b)
};

template <typename T>
__device__ __forceinline__ TileGeom tile_geom(const LevelGeom<T> &g, int seg_len)
{
    TileGeom t;
    const int m0 = g.dim[0].m, m1 = g.dim[1].m, m2 = g.dim[2].m;
    const int mc0 = g.dim[0].mc, mc1 = g.dim[1].mc, mc2 = g.dim[2].mc;
    t.J2 = blockIdx.x * DT2;
    t.J1 = blockIdx.y * DT1;
    t.J0a = blockIdx.z * seg_len;
    t.J0b = min(t.J0a + seg_len, mc0);
    t.n2 = min(DT2, mc2 - t.J2);
    t.n1 = min(DT1, mc1 - t.J1);
    t.lo2 = max(0, cpos_of(m2, mc2, t.J2) - 2) & ~1;
    t.hi2 = min(m2 - 1, cpos_of(m2, mc2, t.J2 + t.n2 - 1) + 2);
    t.lo1 = max(0, cpos_of(m1, mc1, t.J1) - 2) & ~1;
    t.hi1 = min(m1 - 1, cpos_of(m1, mc1, t.J1 + t.n1 - 1) + 2);
    t.lo0 = max(0, cpos_of(m0, mc0, t.J0a) - 2) & ~1;
    t.hi0 = t.J0a < t.J0b ? min(m0 - 1, cpos_of(m0, mc0, t.J0b - 1) + 2) : t.lo0 - 1;
    t.r1n = t.hi1 - t.lo1 + 1;
    t.r2n = t.hi2 - t.lo2 + 1;
    t.o0a = cpos_of(m0, mc0, t.J0a);
    t.o0b = (t.J0b < mc0) ? cpos_of(m0, mc0, t.J0b) : m0;
    return t;
}

template <typename T>
__device__ __forceinline__ PlaneInfo<T> plane_info(const LevelGeom<T> &g, const TileGeom &tg, int p, bool ptap = false)
{
    const T *tap0 = ptap ? g.dim[0].ptap : g.dim[0].tap;
    const int m0 = g.dim[0].m, mc0 = g.dim[0].mc;
    PlaneInfo<T> pi;
    int jlo = first_coarse_at_or_after(g.dim[0], p - 2);
    if (jlo < tg.J0a) jlo = tg.J0a;
    pi.jlo = jlo;
    pi.pad = 0;
    const bool k0 = kept_pos(m0, p);
    const int jc = k0 ? cidx_of(m0, mc0, p) : -10;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const int j = jlo + i;
        const int o = p - cpos_of(m0, mc0, j);
        const bool inj = j < tg.J0b;
        pi.tr[i] = (inj && o >= -2 && o <= 2) ? tap0[j * 5 + o + 2] : (T)0;
        const int d = jc - j;
        pi.tm[i] = (inj && d >= -1 && d <= 1) ? g.dim[0].mtap[j * 3 + d + 1] : (T)0;
    }
    pi.wl = k0 ? (T)0 : g.dim[0].wl[p];
    pi.wr = k0 ? (T)0 : g.dim[0].wr[p];
    return pi;
}

// Per-warp description of the seven fine rows Ra - 2 .. Ra + 4 that the
// warp's two coarse rows j1a, j1b read, and of the restriction and mass taps
// of those rows (zero for rows outside the grid).
template <typename T>
struct WarpRows {
    bool va, vb;        // j1a, j1b inside the grid
    int j1a, j1b;
    int Ra, Rb, offb;   // kept rows of j1a, j1b; offb = Rb - Ra (1 or 2) = local row of j1b's window start
    int rl0;            // stage row of local row 0 (absolute row Ra - 2; may lie outside the region,
                        // where every tap is zero and the guard rows are read)
    uint32_t rm0;       // (Ra - 2) x m2 (mod 2^32): element offset of local row 0 inside its plane
    T t1a[5], t1b[5];   // dim-1 restriction taps of j1a (local rows 0..4) and j1b (offb..offb+4)
    T ma[5], mb[5];     // dim-1 coarse mass taps over the same windows (0 where no coarse row)
};

template <typename T>
__device__ __forceinline__ void warp_rows(const LevelGeom<T> &g, const TileGeom &tg, int c, bool use_mass,
                                          WarpRows<T> &w, bool ptap = false)
{
    const int m1 = g.dim[1].m, mc1 = g.dim[1].mc, m2 = g.dim[2].m;
    w.j1a = tg.J1 + 2 * c;
    w.j1b = w.j1a + 1;
    w.va = 2 * c < tg.n1;
    w.vb = 2 * c + 1 < tg.n1;
    const int ja = w.va ? w.j1a : tg.J1;
    w.Ra = cpos_of(m1, mc1, ja);
    w.Rb = w.vb ? cpos_of(m1, mc1, w.j1b) : w.Ra + 2;
    w.offb = w.Rb - w.Ra;
    w.rl0 = w.Ra - 2 - tg.lo1;
    w.rm0 = (uint32_t)(w.Ra - 2) * (uint32_t)m2;
    const T *tap = ptap ? g.dim[1].ptap : g.dim[1].tap, *mtap = g.dim[1].mtap;
#pragma unroll
    for (int o = 0; o < 5; o++) {
        w.t1a[o] = w.va ? tap[ja * 5 + o] : (T)0;
        w.t1b[o] = w.vb ? tap[w.j1b * 5 + o] : (T)0;
        w.ma[o] = (T)0;
        w.mb[o] = (T)0;
    }
    if (use_mass) {
#pragma unroll
        for (int d = -1; d <= 1; d++) {
            const int j = ja + d;
            if (w.va && j >= 0 && j < mc1) {
                const int o = cpos_of(m1, mc1, j) - w.Ra + 2;
#pragma unroll
                for (int q = 0; q < 5; q++)
                    if (q == o) w.ma[q] = mtap[ja * 3 + d + 1];
            }
            const int jb = w.j1b + d;
            if (w.vb && jb >= 0 && jb < mc1) {
                const int o = cpos_of(m1, mc1, jb) - w.Rb + 2;
#pragma unroll
                for (int q = 0; q < 5; q++)
                    if (q == o) w.mb[q] = mtap[w.j1b * 3 + d + 1];
            }
        }
    }
}

// Per-lane description of the five fine columns Ca - 2 .. Ca + 2 around the
// lane's kept column Ca (positions outside the grid carry zero taps and read
// finite shared memory: the stages start zeroed behind a zero guard).
template <typename T>
struct LaneCols {
    bool colv;        // j2 inside the grid
    bool has_b;       // Ca + 1 is a new node (then Ca + 2 is kept)
    int j2, Ca;
    int ca;           // local column of Ca in the region
    T t2[5], m2t[5];  // dim-2 restriction taps; coarse mass taps over the window
    T wl2, wr2;       // interpolation weights of Ca + 1
};

template <typename T>
__device__ __forceinline__ void lane_cols(const LevelGeom<T> &g, const TileGeom &tg, int lane, bool use_mass,
                                          LaneCols<T> &l, bool ptap = false)
{
    const T *tap2 = ptap ? g.dim[2].ptap : g.dim[2].tap;
    const int m2 = g.dim[2].m, mc2 = g.dim[2].mc;
    l.j2 = tg.J2 + lane;
    l.colv = lane < tg.n2;
    const int j = l.colv ? l.j2 : tg.J2;
    l.Ca = cpos_of(m2, mc2, j);
    l.ca = l.Ca - tg.lo2;
    l.has_b = l.colv && l.Ca + 1 < m2 && !kept_pos(m2, l.Ca + 1);
    l.wl2 = l.has_b ? g.dim[2].wl[l.Ca + 1] : (T)0;
    l.wr2 = l.has_b ? g.dim[2].wr[l.Ca + 1] : (T)0;
#pragma unroll
    for (int o = 0; o < 5; o++) {
        l.t2[o] = l.colv ? tap2[j * 5 + o] : (T)0;
        l.m2t[o] = (T)0;
    }
    if (use_mass) {
#pragma unroll
        for (int d = -1; d <= 1; d++) {
            const int jj = j + d;
            if (l.colv && jj >= 0 && jj < mc2) {
                const int o = cpos_of(m2, mc2, jj) - l.Ca + 2;
#pragma unroll
                for (int q = 0; q < 5; q++)
                    if (q == o) l.m2t[q] = g.dim[2].mtap[j * 3 + d + 1];
            }
        }
    }
}

// dim-2 then dim-1 restriction of one staged plane for the warp's two
// outputs; row(i) points at local row i in shared memory, at the lane's
// window start (column Ca - 2)
template <typename T, typename RowAddr>
__device__ __forceinline__ void restrict_plane(const WarpRows<T> &w, const T t2[5], RowAddr row, T &ra, T &rb)
{
    T s[7];
#pragma unroll
    for (int i = 0; i < 7; i++) {
        const T *a = row(i);
        T acc = (T)0;
#pragma unroll
        for (int o = 0; o < 5; o++) acc = fma_rn(t2[o], a[o], acc);
        s[i] = acc;
    }
    T x = (T)0, y = (T)0;
    const bool two = w.offb == 2;
#pragma unroll
    for (int o = 0; o < 5; o++) {
        x = fma_rn(w.t1a[o], s[o], x);
        y = fma_rn(w.t1b[o], two ? s[o + 2] : s[o + 1], y);
    }
    ra = x;
    rb = y;
}

// ---------------------------------------------------------------------------
// decomp_kernel

template <typename T>
struct DecompSmem {
    static constexpr int NST = decomp_stages<T>();
    static constexpr int PB = stage_pitch<T>();
    static constexpr size_t stage_bytes = (size_t)DR1 * PB;
    static constexpr size_t off_stage = guard_bytes<T>();
    static constexpr size_t off_full = off_stage + NST * stage_bytes + guard_bytes<T>();
    static constexpr size_t off_empty = off_full + NST * 8;
    static constexpr size_t off_info = off_empty + NST * 8;
    static constexpr size_t off_hist = (off_info + NST * sizeof(PlaneInfo<T>) + 15) & ~size_t(15);
    static size_t bytes(int hn) { return off_hist + (size_t)(hn + 1) * 4; }
};

template <typename T, int SINK>
__global__ void __launch_bounds__(DTHREADS, sizeof(T) == 4 ? 2 : 1)
decomp_kernel(RestrictArgs<T> a, int seg_len)
{
    using S = DecompSmem<T>;
    constexpr int NST = S::NST, PB = S::PB;
    constexpr bool QUANT = SINK == (int)Sink::QUANT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const LevelGeom<T> &g = a.g;
    const TileGeom tg = tile_geom(g, seg_len);
    if (tg.J0a >= tg.J0b) return;
    const int m0 = g.dim[0].m, m1 = g.dim[1].m, m2 = g.dim[2].m;
    const int mc0 = g.dim[0].mc, mc1 = g.dim[1].mc, mc2 = g.dim[2].mc;
    unsigned long long *full = reinterpret_cast<unsigned long long *>(smem_raw + S::off_full);
    unsigned long long *empty = reinterpret_cast<unsigned long long *>(smem_raw + S::off_empty);
    PlaneInfo<T> *pinfo = reinterpret_cast<PlaneInfo<T> *>(smem_raw + S::off_info);
    unsigned int *hs = reinterpret_cast<unsigned int *>(smem_raw + S::off_hist);
    const unsigned char *stage_p = smem_raw + S::off_stage;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int hhalf = QUANT ? min((int)a.qo.D / 2, kHistWin) : 0;
    const int hlo = (int)(a.qo.D / 2) - hhalf, hn = 2 * hhalf;
    const int nact = (tg.n1 + 1) >> 1;   // consumer warps with at least one coarse row
    const int limit = a.wait_limit;

    // zero the stages (reads outside the grid meet zeros or earlier planes'
    // finite values, times zero taps) and the histogram; barriers
    {
        uint4 *z = reinterpret_cast<uint4 *>(smem_raw);
        const int n16 = (int)(S::off_full / 16);
        for (int i = tid; i < n16; i += DTHREADS) z[i] = make_uint4(0u, 0u, 0u, 0u);
        if (QUANT)
            for (int i = tid; i <= hn; i += DTHREADS) hs[i] = 0u;
        fence_proxy_async();
        if (tid == 0) {
            for (int i = 0; i < NST; i++) {
                mbar_init(&full[i], 1);
                mbar_init(&empty[i], (uint32_t)nact);
            }
            mbar_fence_init();
        }
    }
    __syncthreads();

    if (warp == DCW) {
        // ---------------- producer ----------------
        // the dim-0 taps of the next plane are loaded while this plane's
        // copies are issued, so their latency overlaps the ring's wait
        PlaneInfo<T> pnext;
        if (lane == 0) pnext = plane_info(g, tg, tg.lo0);
        int k = 0;
        for (int p = tg.lo0; p <= tg.hi0; p++, k++) {
            const int slot = k % NST;
            if (k >= NST && !warp_wait(&empty[slot], (uint32_t)(((k / NST) - 1) & 1), limit)) {
                if (lane == 0) atomicExch(a.status, (unsigned)DS_TIMEOUT);
                break;
            }
            unsigned char *dst0 = smem_raw + S::off_stage + slot * S::stage_bytes;
            const unsigned char *src[2] = {nullptr, nullptr};
            uint32_t nb[2] = {0u, 0u};
            uint32_t bytes = 0;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int r = lane + 32 * h;
                if (r < tg.r1n) {
                    const T *row = a.v + ((long long)p * m1 + tg.lo1 + r) * m2 + tg.lo2;
                    const uintptr_t g0 = reinterpret_cast<uintptr_t>(row);
                    const uintptr_t g1 = g0 + (uintptr_t)tg.r2n * sizeof(T);
                    const uintptr_t s0 = g0 & ~uintptr_t(15);
                    uintptr_t s1 = (g1 + 15) & ~uintptr_t(15);
                    const uintptr_t lim = reinterpret_cast<uintptr_t>(a.src_end) & ~uintptr_t(15);
                    bool tail = false;
                    if (s1 > lim) { tail = true; s1 = lim; }
                    nb[h] = s1 > s0 ? (uint32_t)(s1 - s0) : 0u;
                    src[h] = reinterpret_cast<const unsigned char *>(s0);
                    bytes += nb[h];
                    // the bytes past the buffer's last 16-byte boundary: plain loads
                    if (tail) {
                        const uintptr_t t0 = s1 > g0 ? s1 : g0;
                        for (uintptr_t b = t0; b < g1; b += sizeof(T))
                            *reinterpret_cast<T *>(dst0 + r * PB + (b - s0)) = *reinterpret_cast<const T *>(b);
                    }
                }
            }
            if (lane == 0) pinfo[slot] = pnext;
            for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
            __syncwarp();
            if (lane == 0) mbar_arrive_expect_tx(&full[slot], bytes);
            __syncwarp();
#pragma unroll
            for (int h = 0; h < 2; h++)
                if (nb[h]) bulk_g2s(dst0 + (lane + 32 * h) * PB, src[h], nb[h], &full[slot]);
            if (lane == 0 && p < tg.hi0) pnext = plane_info(g, tg, p + 1);
        }
        // every copy still in flight lands before the CTA may exit
        for (int kk = max(0, k - NST); kk < k; kk++)
            wait_sleep_bounded(&full[kk % NST], (uint32_t)((kk / NST) & 1), kWaitPolls);
        return;
    }

    // ---------------- consumers ----------------
    WarpRows<T> wr;
    warp_rows(g, tg, warp, true, wr);
    LaneCols<T> lc;
    lane_cols(g, tg, lane, true, lc);
    unsigned ew = 0;   // widest escape payload seen by this thread
    if (wr.va) {
        const double rho = QUANT ? rho64_of(a.qo.sc, g.level) : 0.0;
        const float rho_hi = QUANT ? a.qo.sc->rho_f[g.level] : 0.f;
        const int halfD = (int)(a.qo.D / 2);
        const float rho_lo = QUANT ? a.qo.sc->rho_lo[g.level] : 0.f;

        // owned rows: Ra (kept), Ra + 1 (new, if any), Rb (kept, if j1b), Rb + 1 (new, if any)
        const bool s1 = wr.Ra + 1 < m1 && !kept_pos(m1, wr.Ra + 1);
        const bool s3 = wr.vb && wr.Rb + 1 < m1 && !kept_pos(m1, wr.Rb + 1);
        const T w1l = s1 ? g.dim[1].wl[wr.Ra + 1] : (T)0, w1r = s1 ? g.dim[1].wr[wr.Ra + 1] : (T)0;
        const T w3l = s3 ? g.dim[1].wl[wr.Rb + 1] : (T)0, w3r = s3 ? g.dim[1].wr[wr.Rb + 1] : (T)0;
        // stream offsets of the owned rows (Ra, Ra + 1, Rb, Rb + 1) inside a
        // plane: new planes hold every node of a row, kept planes skip the
        // kept nodes of the rows before it
        auto nro = [&](int sl) { return (sl < 2 ? wr.Ra : wr.Rb) * m2 + (sl & 1) * m2; };
        auto kro = [&](int sl) {
            const int r = (sl < 2 ? wr.Ra : wr.Rb) + (sl & 1);
            return r * m2 - kept_before(r) * mc2;
        };
        const int Cb = lc.Ca + 1;
        const long long cstride = (long long)mc1 * mc2;
        const long long out_a = (long long)wr.j1a * mc2 + lc.j2, out_b = (long long)wr.j1b * mc2 + lc.j2;
        const uint32_t bel = (uint32_t)(reinterpret_cast<uintptr_t>(a.v) / sizeof(T)) + (uint32_t)tg.lo2;
        const uint32_t m1m2 = (uint32_t)m1 * (uint32_t)m2;
        constexpr uint32_t VM = 16 / sizeof(T) - 1;
        const int lanecol = lc.ca - 2;
        // local row i of stage `slot` (plane p), at column Ca - 2: the row's
        // data starts at its copy's alignment offset inside the staged row
        auto rowaddr = [&](int slot, int p, int i) -> const T * {
            const uint32_t off = (bel + (uint32_t)p * m1m2 + wr.rm0 + (uint32_t)(i * m2)) & VM;
            return reinterpret_cast<const T *>(stage_p + slot * (int)S::stage_bytes + (wr.rl0 + i) * PB) +
                   (int)off + lanecol;
        };
        Interp<T> Jp;   // interpolant of the last kept plane at the owned nodes
#pragma unroll
        for (int sl = 0; sl < 4; sl++) Jp.v[sl][0] = Jp.v[sl][1] = (T)0;
        int jv = -1;  // plane whose interpolant Jp holds
        // J = I_1 I_2 v of the kept plane staged in `slot` (plane p), at the owned nodes
        auto form_J = [&](int slot, int p) -> Interp<T> {
            Interp<T> J;
            const T *aA = rowaddr(slot, p, 2) + 2;
            const T *aB = rowaddr(slot, p, 2 + wr.offb) + 2;
            const T *aC = rowaddr(slot, p, 4 + wr.offb) + 2;
            const T A0 = aA[0], A2 = aA[2];
            const T B0 = aB[0], B2 = aB[2];
            const T C0 = aC[0], C2 = aC[2];
            const T IA = fma_rn(lc.wr2, A2, mul_rn(lc.wl2, A0));
            const T IB = fma_rn(lc.wr2, B2, mul_rn(lc.wl2, B0));
            const T IC = fma_rn(lc.wr2, C2, mul_rn(lc.wl2, C0));
            J.v[0][0] = A0;
            J.v[0][1] = IA;
            J.v[1][0] = fma_rn(w1r, B0, mul_rn(w1l, A0));
            J.v[1][1] = fma_rn(w1r, IB, mul_rn(w1l, IA));
            J.v[2][0] = B0;
            J.v[2][1] = IB;
            J.v[3][0] = fma_rn(w3r, C0, mul_rn(w3l, B0));
            J.v[3][1] = fma_rn(w3r, IC, mul_rn(w3l, IB));
            return J;
        };
        // the sink of one coefficient at stream index base + off
        auto emit = [&](long long base, int off, T w) {
            if constexpr (SINK == (int)Sink::STREAM) {
                a.coef_out[base + off] = w;
            } else if constexpr (QUANT) {
                // k = sign(w) floor(|w| rho + 1/2) with binary64 semantics
                // (quant_code); codes near the escape range decide in binary64
                // (binary32 coefficients: the double-word decision, valid for
                // every code below 2^22, in 32-bit integers; escapes widen)
                unsigned sym;
                if constexpr (sizeof(T) == 4) {
                    const float ax = fabsf(w);
                    int ki;
                    if (__fmul_rn(ax, rho_hi) < kSmallQuant) ki = quant_small_f32(ax, rho_hi, rho_lo);
                    else ki = halfD;   // a code of 2^22 or more: an escape, decided below
                    if (ki < halfD) {
                        sym = (unsigned)(halfD + (w < (T)0 ? -ki : ki));
                    } else {
                        sym = 0u;
                        ew = max(ew, escape_f32(a.qo, base + off, w, rho_hi, rho_lo, rho));
                    }
                } else {
                    const long long k = quant_code(w, rho);
                    if (k > -halfD && k < halfD) {
                        sym = (unsigned)(halfD + (int)k);
                    } else {
                        sym = 0u;
                        ew = max(ew, escape_store(a.qo, base + off, k));
                    }
                }
                a.qo.sym[base + off] = (uint16_t)sym;
                const unsigned rel = sym - (unsigned)hlo;
                if (rel < (unsigned)hn) atomicAdd(&hs[rel], 1u);
                else if (sym == 0u) atomicAdd(&hs[hn], 1u);
                else atomicAdd(&a.qo.hist[sym], 1ULL);
            }
        };

        // local rows whose coarse mass sums are needed (a coarse row under a nonzero tap)
        unsigned mrows = 0;
#pragma unroll
        for (int i = 0; i < 7; i++) {
            const T mbi = wr.offb == 2 ? (i >= 2 ? wr.mb[i >= 2 ? i - 2 : 0] : (T)0)
                                       : (i >= 1 && i <= 5 ? wr.mb[i >= 1 && i <= 5 ? i - 1 : 0] : (T)0);
            const T mai = i <= 4 ? wr.ma[i <= 4 ? i : 0] : (T)0;
            if (mai != (T)0 || mbi != (T)0) mrows |= 1u << i;
        }
        T acc[2][3];
#pragma unroll
        for (int u = 0; u < 2; u++) acc[u][0] = acc[u][1] = acc[u][2] = (T)0;
        int jb = tg.J0a;
        bool ok = true;
        int k = 0, slot = 0;
        for (int p0 = tg.lo0; p0 <= tg.hi0; p0++, k++, slot = (slot + 1 == NST) ? 0 : slot + 1) {
            if (!warp_wait(&full[slot], (uint32_t)((k / NST) & 1), limit)) { ok = false; break; }
            const PlaneInfo<T> pi = pinfo[slot];
            const bool k0 = kept_pos(m0, p0);
            // ---- restriction of v, and of v_c through the coarse mass matrix
            T ra, rb;
            restrict_plane<T>(wr, lc.t2, [&](int i) { return rowaddr(slot, p0, i); }, ra, rb);
            if (k0) {
                T sm[7];
#pragma unroll
                for (int i = 0; i < 7; i++) {
                    sm[i] = (T)0;
                    if ((mrows >> i) & 1u) {
                        const T *ad = rowaddr(slot, p0, i);
                        T m = (T)0;
#pragma unroll
                        for (int o = 0; o < 5; o++) m = fma_rn(lc.m2t[o], ad[o], m);
                        sm[i] = m;
                    }
                }
                T ca_ = (T)0, cb_ = (T)0;
                const bool two = wr.offb == 2;
#pragma unroll
                for (int o = 0; o < 5; o++) {
                    ca_ = fma_rn(wr.ma[o], sm[o], ca_);
                    cb_ = fma_rn(wr.mb[o], two ? sm[o + 2] : sm[o + 1], cb_);
                }
                while (jb < pi.jlo && jb < tg.J0b) {
                    if (lc.colv) {
                        a.b[(long long)jb * cstride + out_a] = acc[0][0];
                        if (wr.vb) a.b[(long long)jb * cstride + out_b] = acc[1][0];
                    }
#pragma unroll
                    for (int u = 0; u < 2; u++) { acc[u][0] = acc[u][1]; acc[u][1] = acc[u][2]; acc[u][2] = (T)0; }
                    jb++;
                }
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    acc[0][i] = fma_rn(-pi.tm[i], ca_, fma_rn(pi.tr[i], ra, acc[0][i]));
                    acc[1][i] = fma_rn(-pi.tm[i], cb_, fma_rn(pi.tr[i], rb, acc[1][i]));
                }
            } else {
                while (jb < pi.jlo && jb < tg.J0b) {
                    if (lc.colv) {
                        a.b[(long long)jb * cstride + out_a] = acc[0][0];
                        if (wr.vb) a.b[(long long)jb * cstride + out_b] = acc[1][0];
                    }
#pragma unroll
                    for (int u = 0; u < 2; u++) { acc[u][0] = acc[u][1]; acc[u][1] = acc[u][2]; acc[u][2] = (T)0; }
                    jb++;
                }
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    acc[0][i] = fma_rn(pi.tr[i], ra, acc[0][i]);
                    acc[1][i] = fma_rn(pi.tr[i], rb, acc[1][i]);
                }
            }
            // ---- coefficients of the owned nodes
            if (p0 >= tg.o0a && p0 < tg.o0b) {
                const long long pb = plane_base_of(g, p0);
                if (k0) {
                    if (jv != p0) { Jp = form_J(slot, p0); jv = p0; }
                    const T *a2 = rowaddr(slot, p0, 2) + 2;
                    const T *a3 = rowaddr(slot, p0, 3) + 2;
                    const T *a4 = rowaddr(slot, p0, 2 + wr.offb) + 2;
                    const T *a5 = rowaddr(slot, p0, 3 + wr.offb) + 2;
                    const int j0 = cidx_of(m0, mc0, p0);
                    const int cko = (Cb - 1) >> 1;   // kept rows: only odd columns are new
                    if (lc.colv) {
                        // kept row Ra: Ca is a coarse node, Ca + 1 a new one
                        if (a.vc) a.vc[(long long)j0 * cstride + out_a] = a2[0];
                        if (lc.has_b) emit(pb, kro(0) + cko, sub_rn(a2[1], Jp.v[0][1]));
                        if (s1) {
                            emit(pb, kro(1) + lc.Ca, sub_rn(a3[0], Jp.v[1][0]));
                            if (lc.has_b) emit(pb, kro(1) + Cb, sub_rn(a3[1], Jp.v[1][1]));
                        }
                        if (wr.vb) {
                            if (a.vc) a.vc[(long long)j0 * cstride + out_b] = a4[0];
                            if (lc.has_b) emit(pb, kro(2) + cko, sub_rn(a4[1], Jp.v[2][1]));
                        }
                        if (s3) {
                            emit(pb, kro(3) + lc.Ca, sub_rn(a5[0], Jp.v[3][0]));
                            if (lc.has_b) emit(pb, kro(3) + Cb, sub_rn(a5[1], Jp.v[3][1]));
                        }
                    }
                } else {
                    // a new plane: the kept plane after it is staged in the next slot
                    const int nslot = (slot + 1 == NST) ? 0 : slot + 1;
                    if (!warp_wait(&full[nslot], (uint32_t)(((k + 1) / NST) & 1), limit)) { ok = false; break; }
                    const Interp<T> Jn = form_J(nslot, p0 + 1);
                    const T *a2 = rowaddr(slot, p0, 2) + 2;
                    const T *a3 = rowaddr(slot, p0, 3) + 2;
                    const T *a4 = rowaddr(slot, p0, 2 + wr.offb) + 2;
                    const T *a5 = rowaddr(slot, p0, 3 + wr.offb) + 2;
                    auto lerp0 = [&](int sl, int c) { return fma_rn(pi.wr, Jn.v[sl][c], mul_rn(pi.wl, Jp.v[sl][c])); };
                    if (lc.colv) {
                        emit(pb, nro(0) + lc.Ca, sub_rn(a2[0], lerp0(0, 0)));
                        if (lc.has_b) emit(pb, nro(0) + Cb, sub_rn(a2[1], lerp0(0, 1)));
                        if (s1) {
                            emit(pb, nro(1) + lc.Ca, sub_rn(a3[0], lerp0(1, 0)));
                            if (lc.has_b) emit(pb, nro(1) + Cb, sub_rn(a3[1], lerp0(1, 1)));
                        }
                        if (wr.vb) {
                            emit(pb, nro(2) + lc.Ca, sub_rn(a4[0], lerp0(2, 0)));
                            if (lc.has_b) emit(pb, nro(2) + Cb, sub_rn(a4[1], lerp0(2, 1)));
                        }
                        if (s3) {
                            emit(pb, nro(3) + lc.Ca, sub_rn(a5[0], lerp0(3, 0)));
                            if (lc.has_b) emit(pb, nro(3) + Cb, sub_rn(a5[1], lerp0(3, 1)));
                        }
                    }
                    Jp = Jn;
                    jv = p0 + 1;
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[slot]);
        }
        if (ok && lc.colv) {
            while (jb < tg.J0b) {
                a.b[(long long)jb * cstride + out_a] = acc[0][0];
                if (wr.vb) a.b[(long long)jb * cstride + out_b] = acc[1][0];
#pragma unroll
                for (int u = 0; u < 2; u++) { acc[u][0] = acc[u][1]; acc[u][1] = acc[u][2]; acc[u][2] = (T)0; }
                jb++;
            }
        }
        if (!ok && lane == 0) atomicExch(a.status, (unsigned)DS_TIMEOUT);
    }
    if (QUANT) {
        ew = __reduce_max_sync(0xffffffffu, ew);
        if (lane == 0 && ew) atomicMax(&a.qo.sc->esc_w, ew);
        named_sync(1, DCW * 32);
        for (int i = tid; i < hn; i += DCW * 32)
            if (hs[i]) atomicAdd(&a.qo.hist[hlo + i], (unsigned long long)hs[i]);
        if (tid == 0 && hs[hn]) atomicAdd(&a.qo.hist[0], (unsigned long long)hs[hn]);
    }
}

// ---------------------------------------------------------------------------
// rsym_kernel: b = ((x)_k R) w with R = P^T M_l (or P^T: use_ptap), where w
// is, by source,
//   SYMBOLS  the dequantized symbols of level l on its new nodes, 0 on the
//            kept ones (the inverse of Alg. 1 applies the same mass_trans to
//            the decoded coefficients);
//   STREAM   level l of a coefficient stream, laid out like the symbols;
//   DENSE    a level-l grid, every node or (dense_new_only) its new nodes.
// The producer stages each plane's rows (a row of a stream's kept plane that
// is kept in dim 1 holds only its odd positions); the consumers expand the
// region together into one of the shared tiles W, meet at one named barrier
// per plane (which also carries their vote on a wait that ran out), hand the
// stage back, and restrict W as decomp_kernel restricts v.

template <typename T, int SRC>
struct RsymSmem {
    // staged element: symbols (SYMBOLS) or values (STREAM, DENSE)
    using E = typename std::conditional<SRC == (int)WSrc::SYMBOLS, uint16_t, T>::type;
    static constexpr bool ESC = SRC == (int)WSrc::SYMBOLS;
    static constexpr int NST = rsym_stages<T>();
    static constexpr int PB = stage_pitch<E>();
    static constexpr size_t stage_bytes = (size_t)DR1 * PB;
    static constexpr int WROWS = DR1 + 6;     // zero rows around the region: two before, up to four after
    static constexpr size_t wtile_bytes = (size_t)WROWS * kWPitch * sizeof(T);
    static constexpr size_t off_w = 0;
    static constexpr size_t off_stage = off_w + 3 * wtile_bytes;   // three dequantized tiles
    static constexpr size_t off_full = off_stage + NST * stage_bytes;
    static constexpr size_t off_empty = off_full + NST * 8;
    static constexpr size_t off_info = off_empty + NST * 8;
    static constexpr size_t off_rows = (off_info + NST * sizeof(PlaneInfo<T>) + 15) & ~size_t(15);
    static constexpr int EPITCH = DR2;           // escaped codes of a plane: [DR1][DR2] int64
    static constexpr size_t off_esc = off_rows + (size_t)NST * DR1 * 16;
    static constexpr size_t bytes = off_esc + (ESC ? 2 * (size_t)DR1 * EPITCH * 8 : 0);
};

// an asynchronous 8-byte global -> shared copy (its own completion group per thread)
__device__ __forceinline__ void cp_async8(void *dst_smem, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// where a staged row of a plane sits in its source, written by the producer
// beside the row: the stream index of its first node (for escapes), the
// offset of its first element inside the staged copy, whether the row holds
// every node (1: a new row of the stream, or any row of a dense grid) or only
// the new nodes of a kept row (0), and whether every node of the row is new
struct SymRow {
    long long rb;
    int off;
    short rownew, allnew;
};

__device__ __forceinline__ bool named_sync_or(int id, int nthreads, bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

template <typename T, int SRC>
__global__ void __launch_bounds__(DTHREADS, 2)
rsym_kernel(RestrictArgs<T> a, int seg_len)
{
    using S = RsymSmem<T, SRC>;
    using E = typename S::E;
    constexpr bool SYM = SRC == (int)WSrc::SYMBOLS, DENSE = SRC == (int)WSrc::DENSE;
    const bool ptap = a.use_ptap != 0;
    constexpr int NST = S::NST, PB = S::PB;
    constexpr int NQ = (DR2 + 3) / 4;   // quads of four nodes per region row
    constexpr int kDqItems = (DR1 * NQ + DCW * 32 - 1) / (DCW * 32);   // quads per thread and plane
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const LevelGeom<T> &g = a.g;
    const TileGeom tg = tile_geom(g, seg_len);
    if (tg.J0a >= tg.J0b) return;
    const int m0 = g.dim[0].m, m1 = g.dim[1].m, m2 = g.dim[2].m;
    const int mc1 = g.dim[1].mc, mc2 = g.dim[2].mc;
    unsigned long long *full = reinterpret_cast<unsigned long long *>(smem_raw + S::off_full);
    unsigned long long *empty = reinterpret_cast<unsigned long long *>(smem_raw + S::off_empty);
    PlaneInfo<T> *pinfo = reinterpret_cast<PlaneInfo<T> *>(smem_raw + S::off_info);
    T *W0 = reinterpret_cast<T *>(smem_raw + S::off_w);
    SymRow *rowinfo = reinterpret_cast<SymRow *>(smem_raw + S::off_rows);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int limit = a.wait_limit;
    const SymIn &si_ = a.symin;

    {
        uint4 *z = reinterpret_cast<uint4 *>(smem_raw);
        const int n16 = (int)(S::off_full / 16);
        for (int i = tid; i < n16; i += DTHREADS) z[i] = make_uint4(0u, 0u, 0u, 0u);
        fence_proxy_async();
        if (tid == 0) {
            for (int i = 0; i < NST; i++) {
                mbar_init(&full[i], 1);
                mbar_init(&empty[i], 1);
            }
            mbar_fence_init();
        }
    }
    __syncthreads();

    if (warp == DCW) {
        // ---------------- producer: symbol rows of each plane ----------------
        PlaneInfo<T> pnext;
        if (lane == 0) pnext = plane_info(g, tg, tg.lo0, ptap);
        int k = 0;
        for (int p = tg.lo0; p <= tg.hi0; p++, k++) {
            const int slot = k % NST;
            if (k >= NST && !warp_wait(&empty[slot], (uint32_t)(((k / NST) - 1) & 1), limit)) {
                if (lane == 0) atomicExch(a.status, (unsigned)DS_TIMEOUT);
                break;
            }
            unsigned char *dst0 = smem_raw + S::off_stage + slot * S::stage_bytes;
            const bool k0 = kept_pos(m0, p);
            const long long pb = DENSE ? 0 : plane_base_of(g, p);
            uint32_t nb = 0;
            const unsigned char *src = nullptr;
            if (lane < tg.r1n) {
                const int p1 = tg.lo1 + lane;
                const bool allnew = !k0 || !kept_pos(m1, p1);
                // stream sources hold the new nodes only; a dense grid holds every node
                const bool rownew = DENSE || allnew;
                const long long rb = DENSE ? ((long long)p * m1 + p1) * m2 : row_base(g, pb, k0, p1);
                const long long first = rownew ? rb + tg.lo2 : rb + (tg.lo2 >> 1);
                const int cnt = rownew ? tg.r2n : ((tg.hi2 - tg.lo2) >> 1);
                const E *base = SYM ? reinterpret_cast<const E *>(si_.sym)
                                    : reinterpret_cast<const E *>(DENSE ? a.v : a.coef_in);
                const uintptr_t g0 = reinterpret_cast<uintptr_t>(base + first);
                SymRow sr_;
                sr_.rb = rb;
                sr_.off = (int)((g0 & 15) / sizeof(E));
                sr_.rownew = rownew ? 1 : 0;
                sr_.allnew = allnew ? 1 : 0;
                rowinfo[slot * DR1 + lane] = sr_;
                const uintptr_t g1 = g0 + (uintptr_t)cnt * sizeof(E);
                const uintptr_t s0 = g0 & ~uintptr_t(15);
                uintptr_t s1 = (g1 + 15) & ~uintptr_t(15);
                const uintptr_t lim = reinterpret_cast<uintptr_t>(a.src_end) & ~uintptr_t(15);
                bool tail = false;
                if (s1 > lim) { tail = true; s1 = lim; }
                if (g1 <= g0) { s1 = s0; tail = false; }
                nb = s1 > s0 ? (uint32_t)(s1 - s0) : 0u;
                src = reinterpret_cast<const unsigned char *>(s0);
                if (tail) {
                    const uintptr_t t0 = s1 > g0 ? s1 : g0;
                    for (uintptr_t b = t0; b < g1; b += sizeof(E))
                        *reinterpret_cast<E *>(dst0 + lane * PB + (b - s0)) = *reinterpret_cast<const E *>(b);
                }
            }
            if (lane == 0) pinfo[slot] = pnext;
            uint32_t bytes = nb;
            for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
            __syncwarp();
            if (lane == 0) mbar_arrive_expect_tx(&full[slot], bytes);
            __syncwarp();
            if (nb) bulk_g2s(dst0 + lane * PB, src, nb, &full[slot]);
            if (lane == 0 && p < tg.hi0) pnext = plane_info(g, tg, p + 1, ptap);
        }
        for (int kk = max(0, k - NST); kk < k; kk++)
            wait_sleep_bounded(&full[kk % NST], (uint32_t)((kk / NST) & 1), kWaitPolls);
        return;
    }

    // ---------------- consumers ----------------
    WarpRows<T> wr;
    warp_rows(g, tg, warp, false, wr, ptap);
    LaneCols<T> lc;
    lane_cols(g, tg, lane, false, lc, ptap);
    const T q = SYM ? q_of<T>(si_.sc, g.level) : (T)0;
    const bool new_only = a.dense_new_only != 0;
    const int lanecol = lc.ca - 2;
    const long long cstride = (long long)mc1 * mc2;
    const long long out_a = (long long)wr.j1a * mc2 + lc.j2, out_b = (long long)wr.j1b * mc2 + lc.j2;
    T acc[2][3];
#pragma unroll
    for (int u = 0; u < 2; u++) acc[u][0] = acc[u][1] = acc[u][2] = (T)0;
    int jb = tg.J0a;
    bool failed = false;
    const int nplanes = tg.hi0 - tg.lo0 + 1;
    const int nq = (tg.r2n + 3) >> 2;
    auto tile = [&](int kk) -> T * { return W0 + (size_t)(kk % 3) * (S::wtile_bytes / sizeof(T)) + 2 * kWPitch + 4; };
    // The dequantized tile of plane kk is filled one iteration before its
    // restriction: the values of its symbols now; its escaped codes travel
    // from global memory into a shared escape tile by asynchronous copies and
    // enter the tile on the next iteration, so their latency hides behind a
    // plane of work (a register destination would serialize the warp on
    // every escape it meets).
    struct Taps {
        int jlo;
        T tr[3];
    };
    long long *esc_tile0 = reinterpret_cast<long long *>(smem_raw + S::off_esc);
    // returns the mask of this thread's escaped nodes (bit 4 it + e)
    auto fill = [&](int kk, T *Wt) -> unsigned {
        const int sl = kk % NST;
        const unsigned char *st = smem_raw + S::off_stage + sl * S::stage_bytes;
        const SymRow *ri = rowinfo + sl * DR1;
        long long *et = esc_tile0 + (size_t)(kk & 1) * DR1 * S::EPITCH;
        unsigned escm = 0;
#pragma unroll
        for (int it = 0; it < kDqItems; it++) {
            const int u = tid + it * DCW * 32;
            const int i1 = u / NQ, qd = u - i1 * NQ, i2b = qd * 4;
            if (!(u < tg.r1n * NQ && qd < nq)) continue;
            const SymRow r = ri[i1];
            const E *sr = reinterpret_cast<const E *>(st + i1 * PB) + r.off;
            T wv[4];
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int i2 = i2b + e, p2 = tg.lo2 + i2;
                wv[e] = (T)0;
                if constexpr (DENSE) {
                    // every node of a dense grid, or only its new nodes
                    if (i2 < tg.r2n && (!new_only || r.allnew || !kept_pos(m2, p2))) wv[e] = (T)sr[i2];
                } else if (i2 < tg.r2n && (r.rownew || !kept_pos(m2, p2))) {
                    const int sx = r.rownew ? i2 : (i2 - 1) >> 1;
                    if constexpr (SYM) {
                        const unsigned sv = sr[sx];
                        if (sv != 0u) {
                            wv[e] = mul_rn((T)((int)sv - (int)(si_.D / 2)), q);
                        } else {
                            cp_async8(et + i1 * S::EPITCH + i2, si_.esc + r.rb + (r.rownew ? p2 : (p2 - 1) >> 1));
                            escm |= 1u << (4 * it + e);
                        }
                    } else {
                        wv[e] = (T)sr[sx];
                    }
                }
            }
            T *wd = Wt + i1 * kWPitch + i2b;
            if constexpr (sizeof(T) == 4) {
                *reinterpret_cast<float4 *>(wd) = make_float4(wv[0], wv[1], wv[2], wv[3]);
            } else {
                reinterpret_cast<double2 *>(wd)[0] = make_double2(wv[0], wv[1]);
                reinterpret_cast<double2 *>(wd)[1] = make_double2(wv[2], wv[3]);
            }
        }
        cp_async_commit();
        return escm;
    };
    // the escaped codes of plane kk (this thread's, copied one iteration ago) into its tile
    auto patch = [&](int kk, T *Wt, unsigned escm) {
        if (!SYM || !escm) return;
        const long long *et = esc_tile0 + (size_t)(kk & 1) * DR1 * S::EPITCH;
#pragma unroll
        for (int it = 0; it < kDqItems; it++) {
            const int u = tid + it * DCW * 32;
            const int i1 = u / NQ, i2b = (u - i1 * NQ) * 4;
#pragma unroll
            for (int e = 0; e < 4; e++)
                if ((escm >> (4 * it + e)) & 1u)
                    Wt[i1 * kWPitch + i2b + e] = mul_rn((T)et[i1 * S::EPITCH + i2b + e], q);
        }
    };
    auto taps_of = [&](int kk) -> Taps {
        const PlaneInfo<T> &pi = pinfo[kk % NST];
        Taps t;
        t.jlo = pi.jlo;
        t.tr[0] = pi.tr[0]; t.tr[1] = pi.tr[1]; t.tr[2] = pi.tr[2];
        return t;
    };
    unsigned ec = 0;
    Taps tc;
    tc.jlo = 0; tc.tr[0] = tc.tr[1] = tc.tr[2] = (T)0;
    {
        const bool ok = warp_wait(&full[0], 0u, limit);
        if (ok) {
            tc = taps_of(0);
            ec = fill(0, tile(0));
            cp_async_wait0();
            patch(0, tile(0), ec);
        }
        if (named_sync_or(1, DCW * 32, !ok)) failed = true;
        else if (tid == 0) mbar_arrive(&empty[0]);
    }
    // Each iteration fills the next plane's tile, restricts this plane's
    // (complete since the last barrier), then completes the next tile with its
    // escaped codes and meets the other consumers once: a warp reaches the
    // barrier with both pieces of work done, so the waits absorb the spread of
    // their sum rather than of the fill alone.
    for (int k = 0; k < nplanes && !failed; k++) {
        T *W = tile(k);
        // the next plane: symbols into its tile, its escaped codes in flight
        unsigned en = 0;
        Taps tn = tc;
        bool ok = true;
        if (k + 1 < nplanes) {
            ok = warp_wait(&full[(k + 1) % NST], (uint32_t)(((k + 1) / NST) & 1), limit);
            if (ok) { tn = taps_of(k + 1); en = fill(k + 1, tile(k + 1)); }
        }
        if (wr.va) {
            T ra, rb;
            restrict_plane<T>(wr, lc.t2, [&](int i) -> const T * { return W + (wr.rl0 + i) * kWPitch + lanecol; },
                              ra, rb);
            while (jb < tc.jlo && jb < tg.J0b) {
                if (lc.colv) {
                    a.b[(long long)jb * cstride + out_a] = acc[0][0];
                    if (wr.vb) a.b[(long long)jb * cstride + out_b] = acc[1][0];
                }
#pragma unroll
                for (int u = 0; u < 2; u++) { acc[u][0] = acc[u][1]; acc[u][1] = acc[u][2]; acc[u][2] = (T)0; }
                jb++;
            }
#pragma unroll
            for (int i = 0; i < 3; i++) {
                acc[0][i] = fma_rn(tc.tr[i], ra, acc[0][i]);
                acc[1][i] = fma_rn(tc.tr[i], rb, acc[1][i]);
            }
        }
        if (k + 1 < nplanes) {
            // the next plane's escaped codes (copied during the restriction) into its tile
            cp_async_wait0();
            if (ok) patch(k + 1, tile(k + 1), en);
            // next tile complete, stage k + 1 read, and every consumer knows whether a wait ran out
            if (named_sync_or(1, DCW * 32, !ok)) { failed = true; break; }
            if (tid == 0) mbar_arrive(&empty[(k + 1) % NST]);
        }
        tc = tn;
    }
    if (failed) {
        if (tid == 0) atomicExch(a.status, (unsigned)DS_TIMEOUT);
        return;
    }
    if (wr.va && lc.colv) {
        while (jb < tg.J0b) {
            a.b[(long long)jb * cstride + out_a] = acc[0][0];
            if (wr.vb) a.b[(long long)jb * cstride + out_b] = acc[1][0];
#pragma unroll
            for (int u = 0; u < 2; u++) { acc[u][0] = acc[u][1]; acc[u][1] = acc[u][2]; acc[u][2] = (T)0; }
            jb++;
        }
    }
}

// ---------------------------------------------------------------------------
// expand_kernel: recomposition of one level (the inverse of Alg. 1's lerp):
// kept nodes take the corrected coarse grid v_c, new nodes the coefficient
// plus the multilinear interpolant of v_c.  Warp w of a CTA owns coarse row
// j1 = J1 + w, lane l coarse column j2 = J2 + l; the CTA marches along the
// coarse planes of its segment.  For every coarse plane j0 the lane forms the
// interpolant J = I_1 I_2 v_c at its 2 x 2 fine nodes (rows Ra, Ra + 1,
// columns Ca, Ca + 1) once, and writes the kept fine plane of j0 and the new
// fine plane between j0 - 1 and j0 (lerp of the two J's).  The neighbouring
// column's coarse value comes from the next lane.  Every load is coalesced;
// no shared memory, no barriers.

constexpr int XW = 8;                  // warps (coarse rows) per CTA
constexpr int XTHREADS = XW * 32;

template <typename T, int SRC>
__global__ void __launch_bounds__(XTHREADS)
expand_kernel(LevelGeom<T> g, const T *__restrict__ vc, const T *__restrict__ coef_in, SymIn symin,
              T *__restrict__ out, int seg_len)
{
    const int m0 = g.dim[0].m, m1 = g.dim[1].m, m2 = g.dim[2].m;
    const int mc0 = g.dim[0].mc, mc1 = g.dim[1].mc, mc2 = g.dim[2].mc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j2 = blockIdx.x * 32 + lane, j1 = blockIdx.y * XW + warp;
    const int J0a = blockIdx.z * seg_len, J0b = min(J0a + seg_len, mc0);
    if (J0a >= J0b || blockIdx.y * XW >= mc1) return;
    const bool rowv = j1 < mc1;                // warp-uniform
    const bool colv = rowv && j2 < mc2;
    const int jc2 = min(j2, mc2 - 1), jr1 = min(j1, mc1 - 1);
    const int Ca = cpos_of(m2, mc2, jc2), Ra = cpos_of(m1, mc1, jr1);
    const bool hb = colv && Ca + 1 < m2 && !kept_pos(m2, Ca + 1);     // new column after Ca
    const bool hr = rowv && Ra + 1 < m1 && !kept_pos(m1, Ra + 1);     // new row after Ra
    const T wl2 = hb ? g.dim[2].wl[Ca + 1] : (T)0, wr2 = hb ? g.dim[2].wr[Ca + 1] : (T)0;
    const T wl1 = hr ? g.dim[1].wl[Ra + 1] : (T)0, wr1 = hr ? g.dim[1].wr[Ra + 1] : (T)0;
    const T q = SRC == (int)WSrc::SYMBOLS ? q_of<T>(symin.sc, g.level) : (T)0;
    const int halfD = (int)(symin.D / 2);
    const long long cplane = (long long)mc1 * mc2;
    // coarse column offsets of this lane and of the next column (lane 31 loads its own)
    const int c0 = jc2, c1 = min(jc2 + 1, mc2 - 1);
    const int r0 = jr1, r1 = min(jr1 + 1, mc1 - 1);
    // stream offsets inside a fine plane of the rows Ra (kept) and Ra + 1
    const int nro0 = Ra * m2, nro1 = (Ra + 1) * m2;
    const int kro0 = Ra * m2 - kept_before(Ra) * mc2, kro1 = (Ra + 1) * m2 - kept_before(Ra + 1) * mc2;
    // the raw inputs of one coarse plane j0: its coarse values and the
    // coefficient words of the new fine plane before it (x) and of its kept
    // fine plane (k); loaded one plane ahead of their use
    using W = typename std::conditional<SRC == (int)WSrc::SYMBOLS, unsigned, T>::type;
    struct Raw {
        T a00, a10, a01, a11;
        W x00, x01, x10, x11, k01, k10, k11;
        long long pbx, pbk;
    };
    const int jend = min(J0b, mc0 - 1);     // the new plane after the segment's last kept plane needs J(J0b)
    auto word = [&](long long si) -> W {
        if constexpr (SRC == (int)WSrc::STREAM) return coef_in[si];
        else return symin.sym[si];
    };
    auto load = [&](int j0) -> Raw {
        Raw r;
        const T *pl = vc + (long long)j0 * cplane;
        r.a00 = pl[(long long)r0 * mc2 + c0];
        r.a10 = pl[(long long)r1 * mc2 + c0];
        r.a01 = r.a11 = (T)0;
        if (lane == 31) { r.a01 = pl[(long long)r0 * mc2 + c1]; r.a11 = pl[(long long)r1 * mc2 + c1]; }
        const W z = (W)0;
        r.x00 = r.x01 = r.x10 = r.x11 = r.k01 = r.k10 = r.k11 = z;
        r.pbx = 0;    // no new plane before j0 (a new plane never starts the stream)
        r.pbk = -1;   // no kept plane of j0 in this segment
        const int P0 = cpos_of(m0, mc0, j0);
        if (j0 > J0a && colv) {
            const int Pn = cpos_of(m0, mc0, j0 - 1) + 1;
            if (Pn < P0) {
                const long long pb = plane_base_of(g, Pn);
                r.pbx = pb;
                r.x00 = word(pb + nro0 + Ca);
                if (hb) r.x01 = word(pb + nro0 + Ca + 1);
                if (hr) {
                    r.x10 = word(pb + nro1 + Ca);
                    if (hb) r.x11 = word(pb + nro1 + Ca + 1);
                }
            }
        }
        if (j0 < J0b && colv) {
            const long long pb = plane_base_of(g, P0);
            r.pbk = pb;
            if (hb) r.k01 = word(pb + kro0 + (Ca >> 1));
            if (hr) {
                r.k10 = word(pb + kro1 + Ca);
                if (hb) r.k11 = word(pb + kro1 + Ca + 1);
            }
        }
        return r;
    };
    struct J4 { T v00, v01, v10, v11; };
    J4 Jp = {(T)0, (T)0, (T)0, (T)0};
    if (!rowv) return;
    // Escaped codes (symbol 0) travel into shared slots by asynchronous
    // copies, one plane ahead of their use; with a register destination a
    // warp would wait on every node at which any lane escapes.
    extern __shared__ __align__(16) unsigned char xsm[];
    long long *eslot = reinterpret_cast<long long *>(xsm) + threadIdx.x * 7;   // [2][XTHREADS][7]
    bool pend = false;   // escapes of the current plane in flight
    auto issue_esc = [&](const Raw &r, int b) -> bool {
        if constexpr (SRC == (int)WSrc::SYMBOLS) {
            const bool any = (r.x00 == 0u && colv && r.pbx) || (r.x01 == 0u && hb && r.pbx) ||
                             (r.x10 == 0u && hr && r.pbx) || (r.x11 == 0u && hr && hb && r.pbx) ||
                             (r.k01 == 0u && hb && r.pbk >= 0) || (r.k10 == 0u && hr && r.pbk >= 0) ||
                             (r.k11 == 0u && hr && hb && r.pbk >= 0);
            if (!__any_sync(0xffffffffu, any)) return false;
            long long *e = eslot + (size_t)b * XTHREADS * 7;
            if (r.x00 == 0u && colv && r.pbx) cp_async8(e + 0, symin.esc + r.pbx + nro0 + Ca);
            if (r.x01 == 0u && hb && r.pbx) cp_async8(e + 1, symin.esc + r.pbx + nro0 + Ca + 1);
            if (r.x10 == 0u && hr && r.pbx) cp_async8(e + 2, symin.esc + r.pbx + nro1 + Ca);
            if (r.x11 == 0u && hr && hb && r.pbx) cp_async8(e + 3, symin.esc + r.pbx + nro1 + Ca + 1);
            if (r.k01 == 0u && hb && r.pbk >= 0) cp_async8(e + 4, symin.esc + r.pbk + kro0 + (Ca >> 1));
            if (r.k10 == 0u && hr && r.pbk >= 0) cp_async8(e + 5, symin.esc + r.pbk + kro1 + Ca);
            if (r.k11 == 0u && hr && hb && r.pbk >= 0) cp_async8(e + 6, symin.esc + r.pbk + kro1 + Ca + 1);
            cp_async_commit();
            return true;
        }
        return false;
    };
    // value of coefficient word w (slot j of buffer b holds its code when w is an escape)
    auto val = [&](W wv, int b, int j) -> T {
        if constexpr (SRC == (int)WSrc::STREAM) {
            return wv;
        } else {
            return wv != 0u ? mul_rn((T)((int)wv - halfD), q) : mul_rn((T)eslot[(size_t)b * XTHREADS * 7 + j], q);
        }
    };
    auto step = [&](int j0, Raw &cur, const Raw &nxt, int b) {
        // this plane's escapes were issued a step ago; the next plane's words
        // arrived a step ago: its escapes go in flight
        const bool pn = j0 + 1 <= jend && issue_esc(nxt, b ^ 1);
        if (pend) {
            if (pn) asm volatile("cp.async.wait_group 1;" ::: "memory");
            else asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        pend = pn;
        const Raw &r = cur;
        // J = I_1 I_2 v_c at the lane's 2 x 2 fine nodes; the next column from the next lane
        T a01 = __shfl_down_sync(0xffffffffu, r.a00, 1);
        T a11 = __shfl_down_sync(0xffffffffu, r.a10, 1);
        if (lane == 31) { a01 = r.a01; a11 = r.a11; }
        J4 J;
        J.v00 = r.a00;
        J.v01 = fma_rn(wr2, a01, mul_rn(wl2, r.a00));
        J.v10 = fma_rn(wr1, r.a10, mul_rn(wl1, r.a00));
        J.v11 = fma_rn(wr1, fma_rn(wr2, a11, mul_rn(wl2, r.a10)), mul_rn(wl1, J.v01));
        const int P0 = cpos_of(m0, mc0, j0);
        if (j0 > J0a && colv) {
            // the new fine plane between coarse planes j0 - 1 and j0, if any
            const int Pn = cpos_of(m0, mc0, j0 - 1) + 1;
            if (Pn < P0) {
                const T wl0 = g.dim[0].wl[Pn], wr0 = g.dim[0].wr[Pn];
                T *orow = out + ((long long)Pn * m1 + Ra) * m2;
                orow[Ca] = add_rn(val(r.x00, b, 0), fma_rn(wr0, J.v00, mul_rn(wl0, Jp.v00)));
                if (hb) orow[Ca + 1] = add_rn(val(r.x01, b, 1), fma_rn(wr0, J.v01, mul_rn(wl0, Jp.v01)));
                if (hr) {
                    orow += m2;
                    orow[Ca] = add_rn(val(r.x10, b, 2), fma_rn(wr0, J.v10, mul_rn(wl0, Jp.v10)));
                    if (hb) orow[Ca + 1] = add_rn(val(r.x11, b, 3), fma_rn(wr0, J.v11, mul_rn(wl0, Jp.v11)));
                }
            }
        }
        if (j0 < J0b && colv) {
            // the kept fine plane of coarse plane j0
            T *orow = out + ((long long)P0 * m1 + Ra) * m2;
            orow[Ca] = J.v00;
            if (hb) orow[Ca + 1] = add_rn(val(r.k01, b, 4), J.v01);
            if (hr) {
                orow += m2;
                orow[Ca] = add_rn(val(r.k10, b, 5), J.v10);
                if (hb) orow[Ca + 1] = add_rn(val(r.k11, b, 6), J.v11);
            }
        }
        Jp = J;
        // this plane's registers take the plane after next
        if (j0 + 2 <= jend) cur = load(j0 + 2);
    };
    Raw A = load(J0a);
    Raw B;
    if (J0a + 1 <= jend) B = load(J0a + 1);
    pend = issue_esc(A, 0);
    for (int j0 = J0a; j0 <= jend; j0 += 2) {
        step(j0, A, B, 0);
        if (j0 + 1 > jend) break;
        step(j0 + 1, B, A, 1);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}


}  // namespace

template <typename T>
cudaError_t launch_decomp(Sink sink, const RestrictArgs<T> &a0, cudaStream_t s)
{
    if (sink != Sink::QUANT && sink != Sink::STREAM) return cudaErrorInvalidValue;
    RestrictArgs<T> a = a0;
    a.wait_limit = g_wait_limit;
    const int mc0 = a.g.dim[0].mc, mc1 = a.g.dim[1].mc, mc2 = a.g.dim[2].mc;
    const int gx = (mc2 + DT2 - 1) / DT2, gy = (mc1 + DT1 - 1) / DT1;
    const int hn = sink == Sink::QUANT ? 2 * (int)std::min<unsigned>(a.qo.D / 2, kHistWin) : 0;
    const size_t sm = DecompSmem<T>::bytes(hn);
    // one set-up flag per kernel (both instantiations share a function type)
    static PerDeviceOnce attr_quant, attr_stream;
    auto go = [&](auto kern, PerDeviceOnce &attr) -> cudaError_t {
        cudaError_t e = once_per_device(attr, [&] {
            return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        });
        if (e != cudaSuccess) return e;
        const int seg = choose_segment(mc0, (long long)gx * gy, resident_ctas(kern, DTHREADS, sm));
        const int gz = (mc0 + seg - 1) / seg;
        kern<<<dim3(gx, gy, gz), DTHREADS, sm, s>>>(a, seg);
        count_launch();
        return cudaGetLastError();
    };
    if (sink == Sink::QUANT) return go(decomp_kernel<T, (int)Sink::QUANT>, attr_quant);
    return go(decomp_kernel<T, (int)Sink::STREAM>, attr_stream);
}

template <typename T>
cudaError_t launch_restrict_symbols(const RestrictArgs<T> &a0, cudaStream_t s)
{
    return launch_restrict_planes<T>(WSrc::SYMBOLS, a0, s);
}

template <typename T>
cudaError_t launch_restrict_planes(WSrc src, const RestrictArgs<T> &a0, cudaStream_t s)
{
    RestrictArgs<T> a = a0;
    a.wait_limit = g_wait_limit;
    const int mc0 = a.g.dim[0].mc, mc1 = a.g.dim[1].mc, mc2 = a.g.dim[2].mc;
    const long long nl = (long long)a.g.dim[0].m * a.g.dim[1].m * a.g.dim[2].m;
    // the end of the staged source: the level's stream (new nodes) or its dense grid
    if (src == WSrc::STREAM) a.src_end = a.coef_in + a.g.Nprev + (nl - (long long)mc0 * mc1 * mc2);
    if (src == WSrc::DENSE) a.src_end = a.v + nl;
    const int gx = (mc2 + DT2 - 1) / DT2, gy = (mc1 + DT1 - 1) / DT1;
    auto go = [&](auto kern, size_t sm, PerDeviceOnce &attr) -> cudaError_t {
        cudaError_t e = once_per_device(attr, [&] {
            return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        });
        if (e != cudaSuccess) return e;
        const int seg = choose_segment(mc0, (long long)gx * gy, resident_ctas(kern, DTHREADS, sm));
        const int gz = (mc0 + seg - 1) / seg;
        kern<<<dim3(gx, gy, gz), DTHREADS, sm, s>>>(a, seg);
        count_launch();
        return cudaGetLastError();
    };
    static PerDeviceOnce attr_sym, attr_stream, attr_dense;
    if (src == WSrc::STREAM)
        return go(rsym_kernel<T, (int)WSrc::STREAM>, RsymSmem<T, (int)WSrc::STREAM>::bytes, attr_stream);
    if (src == WSrc::DENSE)
        return go(rsym_kernel<T, (int)WSrc::DENSE>, RsymSmem<T, (int)WSrc::DENSE>::bytes, attr_dense);
    return go(rsym_kernel<T, (int)WSrc::SYMBOLS>, RsymSmem<T, (int)WSrc::SYMBOLS>::bytes, attr_sym);
}

template <typename T>
cudaError_t launch_expand_planes(WSrc src, const LevelGeom<T> &g, const T *vc, const T *coef_in,
                                 const SymIn &symin, T *out, cudaStream_t s)
{
    const int mc0 = g.dim[0].mc, mc1 = g.dim[1].mc, mc2 = g.dim[2].mc;
    const int gx = (mc2 + 31) / 32, gy = (mc1 + XW - 1) / XW;
    const bool stream = src == WSrc::STREAM;
    const size_t sm = stream ? 0 : (size_t)2 * XTHREADS * 7 * sizeof(long long);   // escape slots
    const int per_sm = stream ? resident_ctas(expand_kernel<T, (int)WSrc::STREAM>, XTHREADS, 0)
                              : resident_ctas(expand_kernel<T, (int)WSrc::SYMBOLS>, XTHREADS, sm);
    const int seg = choose_segment(mc0, (long long)gx * gy, per_sm);
    const int gz = (mc0 + seg - 1) / seg;
    if (stream)
        expand_kernel<T, (int)WSrc::STREAM><<<dim3(gx, gy, gz), XTHREADS, 0, s>>>(g, vc, coef_in, symin, out, seg);
    else
        expand_kernel<T, (int)WSrc::SYMBOLS><<<dim3(gx, gy, gz), XTHREADS, sm, s>>>(g, vc, coef_in, symin, out, seg);
    count_launch();
    return cudaGetLastError();
}

template cudaError_t launch_decomp<float>(Sink, const RestrictArgs<float> &, cudaStream_t);
template cudaError_t launch_decomp<double>(Sink, const RestrictArgs<double> &, cudaStream_t);
template cudaError_t launch_restrict_symbols<float>(const RestrictArgs<float> &, cudaStream_t);
template cudaError_t launch_restrict_symbols<double>(const RestrictArgs<double> &, cudaStream_t);
template cudaError_t launch_restrict_planes<float>(WSrc, const RestrictArgs<float> &, cudaStream_t);
template cudaError_t launch_restrict_planes<double>(WSrc, const RestrictArgs<double> &, cudaStream_t);
template cudaError_t launch_expand_planes<float>(WSrc, const LevelGeom<float> &, const float *, const float *,
                                                 const SymIn &, float *, cudaStream_t);
template cudaError_t launch_expand_planes<double>(WSrc, const LevelGeom<double> &, const double *, const double *,
                                                  const SymIn &, double *, cudaStream_t);

}  // namespace hpdr
