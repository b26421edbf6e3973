// streamed.cu -- compression of host-resident fields in slabs, with host-to-
// device copies, compression and device-to-host copies overlapped on three
// CUDA streams (the host-device pipeline of Sec. V, Fig. 7 and Alg. 4 with a
// fixed slab size).
//
// Slab i uses device buffers I[i%2] (input) and O[i%2] (output): two buffer
// pairs serve three stages because slab i+2 may only enter a buffer pair
// once slab i has left it (the extra dependency edges of Fig. 7).  The host
// enqueues the copy of slab i+1 before it compresses slab i, so the copy
// engine runs ahead of the compute engine, and the copy back of slab i runs
// while slab i+1 is compressed.
//
// Streamed container (little endian):
//   0 "HPDS"   4 u32 version (1)   8 u32 number of slabs   12 u32 dtype
//   16 u64 dims[3] (unused dims hold 1)   40 u32 ndim   44..63 zero
//   64 per slab: u64 first plane, u64 planes, u64 byte offset, u64 bytes
//   then the slab containers (format v1), each at a 16-byte boundary.
#include <cstring>
#include <vector>
#include "internal.cuh"

namespace {

constexpr uint64_t kStreamHdr = 64;

struct StreamRes {
    cudaStream_t s[3] = {nullptr, nullptr, nullptr};   // H2D, compute, D2H
    cudaEvent_t ev[8] = {};
    void *buf[4] = {nullptr, nullptr, nullptr, nullptr};
    size_t bytes[4] = {0, 0, 0, 0};
    unsigned *err = nullptr;        // device: statuses of in-flight decompressions, OR-ed
    unsigned long long *h_pairs = nullptr, *d_pairs = nullptr;   // per slab {size, status}
    size_t npairs = 0;
};

// slab split along dim 0: as few slabs as the byte budget allows, of equal
// size (differing by at most one plane), each of at least two planes
void split_slabs(size_t n0, size_t plane_bytes, size_t slab_bytes, std::vector<size_t> &first,
                 std::vector<size_t> &count)
{
    size_t p = plane_bytes ? slab_bytes / plane_bytes : n0;
    if (p < 2) p = 2;
    if (p > n0) p = n0;
    size_t ns = (n0 + p - 1) / p;
    while (ns > 1 && n0 / ns < 2) ns--;
    const size_t base = n0 / ns, extra = n0 % ns;
    size_t at = 0;
    for (size_t i = 0; i < ns; i++) {
        const size_t c = base + (i < extra ? 1 : 0);
        first.push_back(at);
        count.push_back(c);
        at += c;
    }
}

hpdr_status ensure_pairs(StreamRes *r, size_t n)
{
    if (r->npairs >= n) return HPDR_OK;
    if (r->h_pairs) { cudaDeviceSynchronize(); cudaFreeHost(r->h_pairs); r->h_pairs = nullptr; }
    if (r->d_pairs) { cudaFree(r->d_pairs); r->d_pairs = nullptr; }
    r->npairs = 0;
    if (cudaHostAlloc(&r->h_pairs, 2 * n * sizeof(unsigned long long), cudaHostAllocDefault) != cudaSuccess ||
        cudaMalloc(&r->d_pairs, 2 * n * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        return HPDR_ERR_NOMEM;
    }
    r->npairs = n;
    return HPDR_OK;
}

hpdr_status ensure_res(hpdr_ctx *ctx, StreamRes *&r, size_t in_bytes, size_t out_bytes)
{
    if (!ctx->stream_res) {
        r = new StreamRes();
        for (int i = 0; i < 3; i++)
            if (cudaStreamCreateWithFlags(&r->s[i], cudaStreamNonBlocking) != cudaSuccess) return HPDR_ERR_CUDA;
        for (int i = 0; i < 8; i++)
            if (cudaEventCreateWithFlags(&r->ev[i], cudaEventDisableTiming) != cudaSuccess) return HPDR_ERR_CUDA;
        if (cudaMalloc(&r->err, sizeof(unsigned)) != cudaSuccess) { cudaGetLastError(); return HPDR_ERR_NOMEM; }
        ctx->stream_res = r;
    }
    r = (StreamRes *)ctx->stream_res;
    const size_t want[4] = {in_bytes, in_bytes, out_bytes, out_bytes};
    for (int i = 0; i < 4; i++) {
        if (r->bytes[i] >= want[i]) continue;
        if (r->buf[i]) { cudaDeviceSynchronize(); cudaFree(r->buf[i]); r->buf[i] = nullptr; r->bytes[i] = 0; }
        if (cudaMalloc(&r->buf[i], want[i]) != cudaSuccess) { cudaGetLastError(); return HPDR_ERR_NOMEM; }
        r->bytes[i] = want[i];
    }
    return HPDR_OK;
}

void put32(uint8_t *p, uint32_t v) { memcpy(p, &v, 4); }
void put64(uint8_t *p, uint64_t v) { memcpy(p, &v, 8); }
uint32_t get32(const uint8_t *p) { uint32_t v; memcpy(&v, p, 4); return v; }
uint64_t get64(const uint8_t *p) { uint64_t v; memcpy(&v, p, 8); return v; }

}  // namespace

namespace hpdr {
void destroy_stream_res(hpdr_ctx *ctx)
{
    StreamRes *r = (StreamRes *)ctx->stream_res;
    if (!r) return;
    for (int i = 0; i < 4; i++) if (r->buf[i]) cudaFree(r->buf[i]);
    if (r->err) cudaFree(r->err);
    if (r->h_pairs) cudaFreeHost(r->h_pairs);
    if (r->d_pairs) cudaFree(r->d_pairs);
    for (int i = 0; i < 8; i++) if (r->ev[i]) cudaEventDestroy(r->ev[i]);
    for (int i = 0; i < 3; i++) if (r->s[i]) cudaStreamDestroy(r->s[i]);
    delete r;
    ctx->stream_res = nullptr;
}
}  // namespace hpdr

extern "C" hpdr_status hpdr_compress_host_streamed(hpdr_ctx *ctx, const void *h_in, hpdr_dtype dtype, int ndim,
                                                   const size_t *dims, double tol, hpdr_tol_kind tol_kind,
                                                   hpdr_mode mode, const hpdr_config *cfg, size_t slab_bytes,
                                                   void *h_out, size_t out_capacity, size_t *out_bytes)
{
    if (!ctx || !h_in || !h_out || !out_bytes || !dims || ndim < 1 || ndim > 3) return HPDR_ERR_ARG;
    if (dtype != HPDR_F32 && dtype != HPDR_F64) return HPDR_ERR_ARG;
    for (int k = 0; k < ndim; k++) if (dims[k] < 2) return HPDR_ERR_ARG;
    int dev_prev = -1;
    cudaGetDevice(&dev_prev);
    if (dev_prev != ctx->device) cudaSetDevice(ctx->device);
    struct Restore { int d, p; ~Restore() { if (d != p) cudaSetDevice(p); } } restore{ctx->device, dev_prev};
    const size_t esz = dtype == HPDR_F64 ? 8 : 4;
    size_t plane = esz;
    for (int k = 1; k < ndim; k++) plane *= dims[k];
    std::vector<size_t> first, count;
    if (ndim == 1) { first.push_back(0); count.push_back(dims[0]); }
    else split_slabs(dims[0], plane, slab_bytes ? slab_bytes : (size_t(256) << 20), first, count);
    const size_t ns = first.size();
    size_t maxp = 0;
    for (size_t c : count) maxp = std::max(maxp, c);
    size_t sd[3] = {maxp, ndim > 1 ? dims[1] : 1, ndim > 2 ? dims[2] : 1};
    if (ndim == 1) sd[0] = dims[0];
    const size_t bound = hpdr_compress_bound(ndim, sd, dtype, cfg);
    if (!bound) return HPDR_ERR_ARG;
    StreamRes *r = nullptr;
    hpdr_status st = ensure_res(ctx, r, maxp * plane, bound);
    if (st != HPDR_OK) return st;
    const uint64_t table = kStreamHdr + 32ull * ns;
    uint64_t at = (table + 15) & ~15ull;
    if (at > out_capacity) return HPDR_ERR_CAPACITY;
    uint8_t *out = (uint8_t *)h_out;
    std::vector<uint64_t> off(ns, 0), sz(ns, 0);
    cudaStream_t sH = r->s[0], sC = r->s[1], sD = r->s[2];
    cudaEvent_t *h2d_done = r->ev, *comp_done = r->ev + 2, *d2h_done = r->ev + 4;
    auto h2d = [&](size_t i) -> bool {
        const int j = (int)(i & 1);
        if (i >= 2 && cudaStreamWaitEvent(sH, comp_done[j], 0) != cudaSuccess) return false;
        const uint8_t *src = (const uint8_t *)h_in + first[i] * plane;
        {
            hpdr::ProfScope ps(ctx, "s_h2d", sH);
            if (cudaMemcpyAsync(r->buf[j], src, count[i] * plane, cudaMemcpyHostToDevice, sH) != cudaSuccess)
                return false;
        }
        return cudaEventRecord(h2d_done[j], sH) == cudaSuccess;
    };
    if (ensure_pairs(r, ns) != HPDR_OK) return HPDR_ERR_NOMEM;
    // The host enqueues the compression of slab i before it waits for slab
    // i - 1 (to learn its container size and copy it back), so the compute
    // stream always has the next slab queued.
    auto finish = [&](size_t k) -> hpdr_status {
        const int j = (int)(k & 1);
        if (cudaEventSynchronize(comp_done[j]) != cudaSuccess) return HPDR_ERR_CUDA;
        const unsigned long long nb = r->h_pairs[2 * k], stat = r->h_pairs[2 * k + 1];
        if (stat) return hpdr::status_of_device((unsigned)stat);
        if (at + nb > out_capacity) return HPDR_ERR_CAPACITY;
        off[k] = at;
        sz[k] = nb;
        if (cudaStreamWaitEvent(sD, comp_done[j], 0) != cudaSuccess) return HPDR_ERR_CUDA;
        {
            hpdr::ProfScope ps(ctx, "s_d2h", sD);
            if (cudaMemcpyAsync(out + at, r->buf[2 + j], nb, cudaMemcpyDeviceToHost, sD) != cudaSuccess)
                return HPDR_ERR_CUDA;
        }
        if (cudaEventRecord(d2h_done[j], sD) != cudaSuccess) return HPDR_ERR_CUDA;
        at = (at + nb + 15) & ~15ull;
        return HPDR_OK;
    };
    if (!h2d(0)) return HPDR_ERR_CUDA;
    for (size_t i = 0; i < ns; i++) {
        const int j = (int)(i & 1);
        if (i + 1 < ns && !h2d(i + 1)) return HPDR_ERR_CUDA;
        if (cudaStreamWaitEvent(sC, h2d_done[j], 0) != cudaSuccess) return HPDR_ERR_CUDA;
        if (i >= 2 && cudaStreamWaitEvent(sC, d2h_done[j], 0) != cudaSuccess) return HPDR_ERR_CUDA;
        size_t d[3] = {count[i], ndim > 1 ? dims[1] : 1, ndim > 2 ? dims[2] : 1};
        {
            hpdr::ProfScope ps(ctx, "s_compute", sC);
            st = hpdr::compress_in_flight(ctx, r->buf[j], dtype, ndim, d, tol, tol_kind, mode, cfg, r->buf[2 + j],
                                          r->bytes[2 + j], r->h_pairs + 2 * i, r->d_pairs + 2 * i, sC);
        }
        if (st != HPDR_OK) { cudaDeviceSynchronize(); return st; }
        if (cudaEventRecord(comp_done[j], sC) != cudaSuccess) return HPDR_ERR_CUDA;
        if (i >= 1) {
            st = finish(i - 1);
            if (st != HPDR_OK) { cudaDeviceSynchronize(); return st; }
        }
    }
    st = finish(ns - 1);
    if (st != HPDR_OK) { cudaDeviceSynchronize(); return st; }
    if (cudaStreamSynchronize(sD) != cudaSuccess || cudaStreamSynchronize(sH) != cudaSuccess) return HPDR_ERR_CUDA;
    memset(out, 0, table);
    memcpy(out, "HPDS", 4);
    put32(out + 4, 1);
    put32(out + 8, (uint32_t)ns);
    put32(out + 12, (uint32_t)dtype);
    for (int k = 0; k < 3; k++) put64(out + 16 + 8 * k, k < ndim ? dims[k] : 1);
    put32(out + 40, (uint32_t)ndim);
    for (size_t i = 0; i < ns; i++) {
        uint8_t *e = out + kStreamHdr + 32 * i;
        put64(e, first[i]);
        put64(e + 8, count[i]);
        put64(e + 16, off[i]);
        put64(e + 24, sz[i]);
    }
    // zero the padding between slab containers
    for (size_t i = 0; i < ns; i++) {
        const uint64_t end = off[i] + sz[i], nxt = (i + 1 < ns) ? off[i + 1] : ((end + 15) & ~15ull);
        if (nxt > end && nxt <= out_capacity) memset(out + end, 0, nxt - end);
    }
    if (ns) memset(out + table, 0, off[0] - table);
    *out_bytes = ns ? (size_t)(off[ns - 1] + sz[ns - 1]) : (size_t)at;
    return HPDR_OK;
}

extern "C" hpdr_status hpdr_decompress_host_streamed(hpdr_ctx *ctx, const void *h_in, size_t in_bytes, void *h_out,
                                                     size_t out_capacity)
{
    if (!ctx || !h_in || !h_out) return HPDR_ERR_ARG;
    const uint8_t *in = (const uint8_t *)h_in;
    if (in_bytes < kStreamHdr || memcmp(in, "HPDS", 4) != 0 || get32(in + 4) != 1) return HPDR_ERR_FORMAT;
    const size_t ns = get32(in + 8);
    const int dtype = (int)get32(in + 12), ndim = (int)get32(in + 40);
    if (dtype < 0 || dtype > 1 || ndim < 1 || ndim > 3 || ns == 0) return HPDR_ERR_FORMAT;
    if (kStreamHdr + 32ull * ns > in_bytes) return HPDR_ERR_FORMAT;
    size_t dims[3];
    for (int k = 0; k < 3; k++) dims[k] = (size_t)get64(in + 16 + 8 * k);
    const size_t esz = dtype == 1 ? 8 : 4;
    size_t plane = esz;
    for (int k = 1; k < ndim; k++) plane *= dims[k];
    if (dims[0] * plane > out_capacity) return HPDR_ERR_CAPACITY;
    std::vector<uint64_t> first(ns), count(ns), off(ns), sz(ns);
    size_t maxp = 0, maxc = 0, expect = 0;
    for (size_t i = 0; i < ns; i++) {
        const uint8_t *e = in + kStreamHdr + 32 * i;
        first[i] = get64(e); count[i] = get64(e + 8); off[i] = get64(e + 16); sz[i] = get64(e + 24);
        if (first[i] != expect || count[i] == 0 || off[i] + sz[i] > in_bytes || off[i] < kStreamHdr + 32ull * ns)
            return HPDR_ERR_FORMAT;
        expect += count[i];
        maxp = std::max<size_t>(maxp, count[i]);
        maxc = std::max<size_t>(maxc, sz[i]);
    }
    if (expect != dims[0]) return HPDR_ERR_FORMAT;
    int dev_prev = -1;
    cudaGetDevice(&dev_prev);
    if (dev_prev != ctx->device) cudaSetDevice(ctx->device);
    struct Restore { int d, p; ~Restore() { if (d != p) cudaSetDevice(p); } } restore{ctx->device, dev_prev};
    StreamRes *r = nullptr;
    // buffers 0,1 hold containers here and 2,3 the decompressed slabs
    hpdr_status st = ensure_res(ctx, r, std::max(maxc, maxp * plane), std::max(maxc, maxp * plane));
    if (st != HPDR_OK) return st;
    cudaStream_t sH = r->s[0], sC = r->s[1], sD = r->s[2];
    cudaEvent_t *h2d_done = r->ev, *comp_done = r->ev + 2, *d2h_done = r->ev + 4;
    auto h2d = [&](size_t i) -> bool {
        const int j = (int)(i & 1);
        if (i >= 2 && cudaStreamWaitEvent(sH, comp_done[j], 0) != cudaSuccess) return false;
        {
            hpdr::ProfScope ps(ctx, "s_h2d", sH);
            if (cudaMemcpyAsync(r->buf[j], in + off[i], sz[i], cudaMemcpyHostToDevice, sH) != cudaSuccess) return false;
        }
        return cudaEventRecord(h2d_done[j], sH) == cudaSuccess;
    };
    // the host never waits inside the loop: every slab's header is read from
    // the host copy of the container and the statuses are checked at the end
    if (cudaMemsetAsync(r->err, 0, sizeof(unsigned), sC) != cudaSuccess) return HPDR_ERR_CUDA;
    if (!h2d(0)) return HPDR_ERR_CUDA;
    for (size_t i = 0; i < ns; i++) {
        const int j = (int)(i & 1);
        if (i + 1 < ns && !h2d(i + 1)) return HPDR_ERR_CUDA;
        if (cudaStreamWaitEvent(sC, h2d_done[j], 0) != cudaSuccess) return HPDR_ERR_CUDA;
        if (i >= 2 && cudaStreamWaitEvent(sC, d2h_done[j], 0) != cudaSuccess) return HPDR_ERR_CUDA;
        {
            hpdr::ProfScope ps(ctx, "s_compute", sC);
            const size_t hb = std::min<size_t>((size_t)sz[i], 128 + 8 * (hpdr::kMaxLevels + 1));
            st = hpdr::decompress_in_flight(ctx, in + off[i], hb, r->buf[j], sz[i], r->buf[2 + j],
                                            r->bytes[2 + j], sC, r->err);
        }
        if (st != HPDR_OK) { cudaDeviceSynchronize(); return st; }
        if (cudaEventRecord(comp_done[j], sC) != cudaSuccess) return HPDR_ERR_CUDA;
        if (cudaStreamWaitEvent(sD, comp_done[j], 0) != cudaSuccess) return HPDR_ERR_CUDA;
        {
            hpdr::ProfScope ps(ctx, "s_d2h", sD);
            if (cudaMemcpyAsync((uint8_t *)h_out + first[i] * plane, r->buf[2 + j], count[i] * plane,
                                cudaMemcpyDeviceToHost, sD) != cudaSuccess)
                return HPDR_ERR_CUDA;
        }
        if (cudaEventRecord(d2h_done[j], sD) != cudaSuccess) return HPDR_ERR_CUDA;
    }
    if (cudaStreamSynchronize(sD) != cudaSuccess || cudaStreamSynchronize(sH) != cudaSuccess ||
        cudaStreamSynchronize(sC) != cudaSuccess)
        return HPDR_ERR_CUDA;
    unsigned err = 0;
    if (cudaMemcpy(&err, r->err, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return HPDR_ERR_CUDA;
    if (err) return hpdr::status_of_device(err);
    return HPDR_OK;
}
