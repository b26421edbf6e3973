// noalloc.cu -- multilevel decomposition without any device allocation.
//
// Some callers cannot allocate device memory on their call path: services
// that hand all device memory to their own pool at start-up (a later
// cudaMalloc would fail, or is forbidden by the service's rules), and
// latency-critical loops that cannot afford cudaMalloc/cudaFree, which may
// synchronize the device and take unbounded time.  For them
// hpdr_decompose_noalloc runs the same kernels as hpdr_decompose, with the
// plan tables and the level buffers placed in one fixed file-scope device
// array instead of a context workspace.
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include "internal.cuh"
#include "levels.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;   // 16 MiB, held by every GPU that loads the library
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices];                   // device address of the array, per device
std::mutex g_scratch_mutex;

// In host code g_noalloc_scratch names a host-side stand-in, not device
// memory: its device address is looked up once per device, with that device
// current, and passed to the kernels.
hpdr_status scratch_address(int dev, void **out)
{
    if (dev < 0 || dev >= kMaxDevices) return hpdr_status(HPDR_ERR_ARG);
    std::lock_guard<std::mutex> lk(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) { cudaGetLastError(); return HPDR_ERR_CUDA; }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return HPDR_OK;
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// Host images of the plan tables, one per (dtype, shape), kept until the
// process exits.  The tables reach the device by an asynchronous copy from
// this image, so the image must outlive every copy queued from it; a copy
// from pageable memory may still read its source after the call returns.
struct CachedPlan {
    hpdr::Plan P;
    hpdr::PlanImage img;
};
std::map<std::string, std::unique_ptr<CachedPlan>> g_plan_cache;
std::mutex g_plan_mutex;

hpdr_status cached_plan(int ndim, const size_t *dims, bool f64, const CachedPlan **out)
{
    std::string key = f64 ? "d" : "f";
    for (int k = 0; k < ndim && k < 3; k++) key += ":" + std::to_string(dims[k]);
    std::lock_guard<std::mutex> lk(g_plan_mutex);
    auto it = g_plan_cache.find(key);
    if (it == g_plan_cache.end()) {
        std::unique_ptr<CachedPlan> c(new CachedPlan());
        const hpdr_status st = hpdr::plan_image(ndim, dims, f64, &c->P, &c->img);
        if (st != HPDR_OK) return st;
        it = g_plan_cache.emplace(key, std::move(c)).first;
    }
    *out = it->second.get();
    return HPDR_OK;
}

template <typename T> const hpdr::LevelGeom<T> &geom_of(const hpdr::Plan &P, int l);
template <> const hpdr::LevelGeom<float> &geom_of<float>(const hpdr::Plan &P, int l) { return P.gf[l]; }
template <> const hpdr::LevelGeom<double> &geom_of<double>(const hpdr::Plan &P, int l) { return P.gd[l]; }

template <typename T>
hpdr_status decompose_into(const hpdr::Plan &P, const T *u, T *coef, char *scratch, size_t tables_bytes,
                           cudaStream_t s)
{
    using namespace hpdr;
    const int L = P.L;
    const size_t n1 = (size_t)(L >= 1 ? P.N[L - 1] : 1);
    char *p = scratch + up256(tables_bytes);
    Scalars *sc = reinterpret_cast<Scalars *>(p);
    p += up256(sizeof(Scalars));
    T *va = reinterpret_cast<T *>(p);
    p += up256(n1 * sizeof(T));
    T *vb = reinterpret_cast<T *>(p);
    p += up256(n1 * sizeof(T));
    T *b = reinterpret_cast<T *>(p);
    if (cudaMemsetAsync(sc, 0, sizeof(Scalars), s) != cudaSuccess) return HPDR_ERR_CUDA;
    QuantOut qo;
    memset(&qo, 0, sizeof(qo));
    const T *v = u;
    // the same split as hpdr_decompose: levels 1..ls and level 0 in one CTA
    const LevelGeom<T> *geo = &geom_of<T>(P, 0);
    const int ls = coarse_top<T>(&P, geo);
    for (int l = L; l > ls; l--) {
        T *vc = ((L - l) % 2 == 0) ? va : vb;
        RestrictArgs<T> a;
        memset(&a, 0, sizeof(a));
        a.g = geom_of<T>(P, l);
        a.v = v;
        a.src_end = v + P.N[l];
        a.status = &sc->status;
        a.coef_out = coef;
        a.b = b;
        a.vc = vc;
        if (launch_restrict<T>(WSrc::FIELD, Sink::STREAM, a, s) != cudaSuccess) return HPDR_ERR_CUDA;
        if (launch_solves<T>(a.g, b, vc, +1, s) != cudaSuccess) return HPDR_ERR_CUDA;
        v = vc;
    }
    if (ls >= 1) {
        SymIn none;
        memset(&none, 0, sizeof(none));
        if (launch_coarse<T>(1, &P, geo, ls, v, nullptr, qo, coef, none, nullptr, s) != cudaSuccess)
            return HPDR_ERR_CUDA;
    } else if (launch_level0<T>(Sink::STREAM, v, P.N[0], coef, qo, s) != cudaSuccess) {
        return HPDR_ERR_CUDA;
    }
    return HPDR_OK;
}

}  // namespace

extern "C" hpdr_status hpdr_decompose_noalloc(const void *d_u, void *d_coef, hpdr_dtype dtype, int ndim,
                                              const size_t *dims, void *stream)
{
    using namespace hpdr;
    if (!d_u || !d_coef || !dims || (dtype != HPDR_F32 && dtype != HPDR_F64)) return HPDR_ERR_ARG;
    if ((uintptr_t)d_u & 15) return HPDR_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return HPDR_ERR_CUDA; }
    void *scratch = nullptr;
    hpdr_status st = scratch_address(dev, &scratch);
    if (st != HPDR_OK) return st;
    const bool f64 = dtype == HPDR_F64;
    const CachedPlan *cp = nullptr;
    st = cached_plan(ndim, dims, f64, &cp);
    if (st != HPDR_OK) return st;
    const PlanImage &img = cp->img;
    Plan P = cp->P;
    const size_t esz = f64 ? 8 : 4;
    const size_t n1 = (size_t)(P.L >= 1 ? P.N[P.L - 1] : 1);
    const size_t need = up256(img.bytes.size()) + up256(sizeof(Scalars)) + 3 * up256(n1 * esz);
    if (need > kScratchBytes) return HPDR_ERR_CAPACITY;
    cudaStream_t s = (cudaStream_t)stream;
    // the source is the cached image, alive until exit
    if (cudaMemcpyAsync(scratch, img.bytes.data(), img.bytes.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return HPDR_ERR_CUDA;
    bind_plan(&P, img, scratch);
    if (f64)
        return decompose_into<double>(P, (const double *)d_u, (double *)d_coef, (char *)scratch,
                                      img.bytes.size(), s);
    return decompose_into<float>(P, (const float *)d_u, (float *)d_coef, (char *)scratch, img.bytes.size(), s);
}
