// internal.cuh -- shared declarations of the sm_103a library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <atomic>
#include <vector>
#include <map>
#include <string>
#include "../../include/hpdr.h"

namespace hpdr {

constexpr int kMaxLevels = 40;

// ---------------------------------------------------------------------------
// Geometry of one level pair (l, l-1), padded to three dimensions.  Dim k of a
// field with fewer dimensions is inactive: one node, kept, identity taps.

template <typename T>
struct DimTables {
    int m;              // nodes on level l
    int mc;             // nodes on level l-1
    const T *wl;        // [m] interpolation weight of the left coarse neighbour (new nodes)
    const T *wr;        // [m] ... of the right coarse neighbour
    const T *tap;       // [mc*5] restriction P^T M_l, offsets -2..2 around the kept position
    const T *ptap;      // [mc*5] transpose of interpolation P^T, offsets -2..2
    const T *sub;       // [mc] Thomas factors of M_{l-1}: sub-diagonal
    const T *cp;        // [mc] modified super-diagonal c'
    const T *inv_den;   // [mc] 1 / pivot
    const T *etap;      // [m*3] (M_l P): fine node p <- coarse nodes jfirst(p)..+2
    const int *efirst;  // [m] first coarse index of etap's three taps
    const T *mtap;      // [mc*3] rows of M_{l-1}: (sub, diag, super) of coarse node j
};

template <typename T>
struct LevelGeom {
    DimTables<T> dim[3];
    int level;               // l
    long long Nprev;         // N_{l-1}: start of level l's section in the stream
};

__host__ __device__ inline int cpos_of(int m, int mc, int j) { return (j + 1 < mc) ? 2 * j : m - 1; }
__host__ __device__ inline bool kept_pos(int m, int p) { return ((p & 1) == 0) || (p == m - 1); }
// number of kept positions strictly before p
__host__ __device__ inline int kept_before(int p) { return (p + 1) >> 1; }
// coarse index of a kept position
__host__ __device__ inline int cidx_of(int m, int mc, int p) { return (p == m - 1) ? mc - 1 : (p >> 1); }

// ---------------------------------------------------------------------------
// Explicitly rounded arithmetic: the quantization decision and the
// coefficients must not depend on how the compiler contracts expressions.

__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// ---------------------------------------------------------------------------
// Device-side scalars of one compression (one per field).

struct Scalars {
    double maxabs;            // max |u|
    double sumsq;             // sum u^2
    double tau_abs;           // absolute bound
    double q[kMaxLevels + 1]; // bins (binary64)
    double rho_d[kMaxLevels + 1];  // 1/q rounded to binary64
    float rho_f[kMaxLevels + 1];   // rho_d rounded to binary32 (high word)
    float rho_lo[kMaxLevels + 1];  // rho_d - rho_f rounded to binary32 (low word)
    float q_f[kMaxLevels + 1];
    unsigned long long n_esc;     // escaped codes (occurrences of symbol 0)
    unsigned long long total_bits;
    unsigned long long out_bytes; // container size
    unsigned int status;          // 0 ok, else an hpdr_status magnitude
    unsigned int esc_w;           // escape payload width: largest bit length of zigzag(k)
    unsigned int s_lo, s_hi;
    unsigned int maxbits_f32;     // max|u| as float bits (atomicMax)
    unsigned long long maxbits_f64;
};

// escaped codes must satisfy |k| < 2^62 (payload of at most 63 bits)
constexpr long long kEscMax = 1LL << 62;

enum DeviceStatus : unsigned int {
    DS_OK = 0,
    DS_ARG = 1,          // bound below the precision floor, or a code beyond +-2^62
    DS_CAPACITY = 3,     // output too small
    DS_FORMAT = 4,       // invalid stream on decode
    DS_LENGTH = 5,       // a code length above 63
    DS_TIMEOUT = 6,      // a bounded device-side wait gave up
};

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (global -> shared) completed on an mbarrier.

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// As mbar_try_wait, but a thread whose phase is not complete is suspended in
// hardware until the phase completes or about `ns` nanoseconds pass, so a
// waiting warp issues no instructions.
__device__ __forceinline__ bool mbar_try_wait_sleep(unsigned long long *bar, uint32_t parity, uint32_t ns)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}
// Waits for the phase with the given parity; gives up after `limit` polls.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, uint32_t parity, int limit)
{
    for (int i = 0; i < limit; i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// 16-byte aligned source, destination and size.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
constexpr int kWaitPolls = 1 << 20;

// ---------------------------------------------------------------------------
// Plans: hierarchy + device tables for one (shape, dtype).

struct Plan {
    int ndim;
    long long n[3];          // padded shape (leading inactive dims = 1)
    int L;
    int m[3][kMaxLevels + 1];
    long long N[kMaxLevels + 1];   // node count per level
    std::vector<double> corr_norm; // c_l
    void *tables = nullptr;        // one device allocation
    LevelGeom<float> gf[kMaxLevels + 1];
    LevelGeom<double> gd[kMaxLevels + 1];
    bool is_f64;
    // node coordinates given by the caller (dims[0] + ... + dims[ndim-1]
    // values, dimension 0 first), empty for unit spacing; coords_dev is
    // their device copy inside the tables
    std::vector<double> coords;
    const double *coords_dev = nullptr;
    size_t coords_off = 0;
};

struct Workspace {
    void *base = nullptr;
    size_t bytes = 0;
};

}  // namespace hpdr

struct hpdr_prof_rec {
    int id;
    cudaEvent_t a, b;
};

struct hpdr_ctx {
    int device;
    std::map<std::string, hpdr::Plan *> plans;
    hpdr::Workspace ws;
    void *host_pinned = nullptr;   // small pinned buffer for scalars read back
    // diagnostics: CUDA-event time per kernel group (off by default)
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_pool;
    size_t prof_used = 0;
    std::vector<hpdr_prof_rec> prof_recs;
    std::vector<std::string> prof_names;
    std::vector<double> prof_ms;
    std::vector<long long> prof_cnt;
    void *stream_res = nullptr;    // streams, events and slab buffers of the host-streamed pipeline
    void *batch_res = nullptr;     // worker streams and captured graphs of batched compression
};

namespace hpdr {

// number of kernels launched by this library since it was loaded
extern unsigned long long g_launches;
inline void count_launch(int n = 1) { g_launches += (unsigned long long)n; }

// Decompression of a container whose header the caller holds in host memory:
// no header read-back and no wait; the device status is OR-ed into *err_acc
// (a device word).  status_of_device maps such a word to an hpdr_status.
hpdr_status decompress_in_flight(hpdr_ctx *ctx, const uint8_t *hdr_host, size_t hdr_bytes, const void *d_in,
                                 size_t in_bytes, void *d_out, size_t out_capacity, cudaStream_t s,
                                 unsigned *err_acc);
hpdr_status status_of_device(unsigned st);
// Compression that does not wait: {container size, device status} arrive in
// the pinned host pair h_size_status (through the device pair d_pair) when
// the stream reaches the end of the call.
hpdr_status compress_in_flight(hpdr_ctx *ctx, const void *d_in, hpdr_dtype dtype, int ndim, const size_t *dims,
                               double tol, hpdr_tol_kind tol_kind, hpdr_mode mode, const hpdr_config *cfg,
                               void *d_out, size_t out_capacity, unsigned long long *h_size_status,
                               unsigned long long *d_pair, cudaStream_t s);

// diagnostics scope: records CUDA events around a group of launches
struct ProfScope {
    hpdr_ctx *ctx;
    int slot = -1;
    cudaStream_t s;
    ProfScope(hpdr_ctx *c, const char *name, cudaStream_t st);
    ~ProfScope();
};

// plan.cu
struct TableOff {
    size_t wl = 0, wr = 0, tap = 0, ptap = 0, sub = 0, cp = 0, inv_den = 0, etap = 0, efirst = 0, mtap = 0;
};
struct PlanImage {
    std::vector<unsigned char> bytes;   // host image of the device tables
    std::vector<TableOff> offF, offD;   // offsets of every (level, dim) table, binary32 / binary64
};
// hierarchy and host image of the tables of one (shape, type)
// coords: null (node i at coordinate i) or the node coordinates of every
// dimension, strictly increasing and finite, dimension 0 first
hpdr_status plan_image(int ndim, const size_t *dims, bool f64, Plan *P, PlanImage *img,
                       const double *coords = nullptr);
// point the plan's tables at a device copy of img.bytes
void bind_plan(Plan *P, const PlanImage &img, void *tables);
hpdr_status get_plan(hpdr_ctx *ctx, int ndim, const size_t *dims, bool f64, Plan **out,
                     const double *coords = nullptr);
hpdr_status ensure_workspace(hpdr_ctx *ctx, size_t bytes);
int levels_of(int ndim, const size_t *dims);

// streamed.cu
void destroy_stream_res(hpdr_ctx *ctx);

inline hpdr_status cuda_status(cudaError_t e) { return e == cudaSuccess ? HPDR_OK : HPDR_ERR_CUDA; }

inline int current_device()
{
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) { cudaGetLastError(); d = 0; }
    return d;
}

// A set-up step that must run once on every device the process uses (a
// kernel attribute such as its dynamic shared-memory limit belongs to one
// device's context).  Devices 0..63 keep a bit each; higher ordinals run the
// step on every call.  Thread-safe: a step may run twice when two threads race
// on its first call, which is harmless for idempotent steps.
struct PerDeviceOnce {
    std::atomic<unsigned long long> done{0};
};
template <typename F>
cudaError_t once_per_device(PerDeviceOnce &o, F step)
{
    const int dev = current_device();
    const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
    if (bit && (o.done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    const cudaError_t e = step();
    if (e == cudaSuccess && bit) o.done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}
// Number of SMs of the current device (cached per device).
int sm_count();

}  // namespace hpdr

#define HPDR_CUDA_TRY(expr)                                      \
    do {                                                         \
        cudaError_t _e = (expr);                                 \
        if (_e != cudaSuccess) return HPDR_ERR_CUDA;             \
    } while (0)
