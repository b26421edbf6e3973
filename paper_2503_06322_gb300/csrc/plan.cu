// plan.cu -- host side: hierarchy, per-level operator tables, correction norms,
// context and workspace management (the context-memory reuse of Sec. III-B).
//
// For every level pair (l, l-1) and dimension the plan holds, in binary32 and
// binary64 copies:
//   * interpolation weights of the new nodes (Alg. 1 lerp: piecewise-linear
//     in the node coordinates);
//   * the restriction P^T M_l as five taps around every kept position
//     (Alg. 1 mass_trans), and P^T alone for the transposed maps;
//   * Thomas factors of the coarse mass matrix M_{l-1} (Alg. 1 tridiag);
//   * the three taps of M_l P from coarse to fine nodes (transposes only).
#include <cmath>
#include <cstring>
#include <cstdio>
#include <string>
#include "internal.cuh"

namespace hpdr {

int sm_count()
{
    static std::atomic<int> cache[64];
    const int dev = current_device();
    if (dev >= 0 && dev < 64) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        n = 152;
    }
    if (dev >= 0 && dev < 64) cache[dev].store(n, std::memory_order_relaxed);
    return n;
}

static int coarsen(int m) { return (m % 2) ? (m + 1) / 2 : m / 2 + 1; }

int levels_of(int ndim, const size_t *dims)
{
    int L = 1 << 30;
    for (int k = 0; k < ndim; k++) {
        long long n = (long long)dims[k];
        int c = 0;
        while (n > 2) { n = coarsen((int)n); c++; }
        L = c < L ? c : L;
    }
    return L;
}

namespace {

struct Dim1 {
    // coordinates of every level, finest level L last
    std::vector<std::vector<double>> x;
};

// host tables of one (level, dim), binary64
struct HostTab {
    int m, mc;
    std::vector<double> wl, wr, tap, ptap, sub, cp, inv_den, etap, mtap;
    std::vector<int> efirst;
};

void mass_entries(const std::vector<double> &x, int p, double &diag, double &lo, double &hi)
{
    int m = (int)x.size();
    double hl = p > 0 ? x[p] - x[p - 1] : 0.0;
    double hr = p + 1 < m ? x[p + 1] - x[p] : 0.0;
    diag = (hl + hr) / 3.0;
    lo = hl / 6.0;
    hi = hr / 6.0;
}

HostTab build_tab(const std::vector<double> &xf, const std::vector<double> &xc, bool active)
{
    HostTab t;
    int m = (int)xf.size(), mc = (int)xc.size();
    t.m = m; t.mc = mc;
    t.wl.assign(m, 0.0); t.wr.assign(m, 0.0);
    t.tap.assign(mc * 5, 0.0); t.ptap.assign(mc * 5, 0.0);
    t.sub.assign(mc, 0.0); t.cp.assign(mc, 0.0); t.inv_den.assign(mc, 1.0);
    t.etap.assign(m * 3, 0.0); t.efirst.assign(m, 0);
    t.mtap.assign(mc * 3, 0.0);
    if (!active) {
        t.tap[2] = 1.0; t.ptap[2] = 1.0; t.etap[0] = 1.0; t.mtap[1] = 1.0;
        return t;
    }
    for (int p = 0; p < m; p++) {
        if (kept_pos(m, p)) continue;
        double a = xf[p - 1], b = xf[p + 1], c = xf[p];
        t.wl[p] = (b - c) / (b - a);
        t.wr[p] = (c - a) / (b - a);
    }
    // dense P (m x mc) entries as a function
    auto P = [&](int p, int j) -> double {
        if (p < 0 || p >= m) return 0.0;
        if (kept_pos(m, p)) return cidx_of(m, mc, p) == j ? 1.0 : 0.0;
        double v = 0.0;
        if (cidx_of(m, mc, p - 1) == j) v += t.wl[p];
        if (cidx_of(m, mc, p + 1) == j) v += t.wr[p];
        return v;
    };
    auto Mf = [&](int p, int q) -> double {
        if (p < 0 || p >= m || q < 0 || q >= m) return 0.0;
        double d, lo, hi;
        mass_entries(xf, p, d, lo, hi);
        if (q == p) return d;
        if (q == p - 1) return lo;
        if (q == p + 1) return hi;
        return 0.0;
    };
    for (int j = 0; j < mc; j++) {
        int c = cpos_of(m, mc, j);
        for (int o = -2; o <= 2; o++) {
            double s = 0.0;
            for (int p = c - 1; p <= c + 1; p++) s += P(p, j) * Mf(p, c + o);
            t.tap[j * 5 + o + 2] = s;
            t.ptap[j * 5 + o + 2] = P(c + o, j);
        }
    }
    // (M_l P)[p][j] for coarse j in a window of three
    for (int p = 0; p < m; p++) {
        int jlo = 1 << 30;
        for (int q = p - 2; q <= p + 2; q++)
            if (q >= 0 && q < m && kept_pos(m, q)) jlo = std::min(jlo, cidx_of(m, mc, q));
        if (jlo + 2 >= mc) jlo = std::max(0, mc - 3);
        t.efirst[p] = jlo;
        for (int i = 0; i < 3; i++) {
            int j = jlo + i;
            if (j >= mc) continue;
            double s = 0.0;
            for (int q = p - 1; q <= p + 1; q++) s += Mf(p, q) * P(q, j);
            t.etap[p * 3 + i] = s;
        }
    }
    // Thomas factors of M_{l-1}, and its rows
    for (int i = 0; i < mc; i++) {
        double d, lo, hi;
        mass_entries(xc, i, d, lo, hi);
        t.mtap[i * 3 + 0] = lo;
        t.mtap[i * 3 + 1] = d;
        t.mtap[i * 3 + 2] = hi;
        double den = (i == 0) ? d : d - lo * t.cp[i - 1];
        t.sub[i] = (i == 0) ? 0.0 : lo;
        t.inv_den[i] = 1.0 / den;
        t.cp[i] = hi / den;
    }
    return t;
}

// infinity norm of G = M_{l-1}^{-1} P^T M_l, one column at a time through the taps
double corr_norm_dim(const HostTab &t)
{
    if (t.mc == t.m) return 1.0;  // inactive
    int m = t.m, mc = t.mc;
    std::vector<double> rows(mc, 0.0), col(mc);
    for (int p = 0; p < m; p++) {
        for (int j = 0; j < mc; j++) {
            int o = p - cpos_of(m, mc, j);
            col[j] = (o >= -2 && o <= 2) ? t.tap[j * 5 + o + 2] : 0.0;
        }
        for (int i = 0; i < mc; i++) col[i] = (col[i] - (i ? t.sub[i] * col[i - 1] : 0.0)) * t.inv_den[i];
        for (int i = mc - 2; i >= 0; i--) col[i] = col[i] - t.cp[i] * col[i + 1];
        for (int i = 0; i < mc; i++) rows[i] += std::fabs(col[i]);
    }
    double mx = 0.0;
    for (double r : rows) mx = std::max(mx, r);
    return mx;
}


}  // namespace

hpdr_status plan_image(int ndim, const size_t *dims, bool f64, Plan *P, PlanImage *img, const double *coords)
{
    if (ndim < 1 || ndim > 3 || !dims) return HPDR_ERR_ARG;
    for (int k = 0; k < ndim; k++)
        if (dims[k] < 2 || dims[k] > (size_t)(1u << 30)) return HPDR_ERR_ARG;
    P->ndim = ndim;
    P->is_f64 = f64;
    int L = levels_of(ndim, dims);
    if (L > kMaxLevels) return HPDR_ERR_ARG;
    P->L = L;
    int pad = 3 - ndim;
    bool active[3];
    std::vector<std::vector<double>> xs[3];  // xs[k][l] coordinates
    P->coords.clear();
    const double *ck = coords;
    for (int k = 0; k < 3; k++) {
        active[k] = k >= pad;
        long long n = active[k] ? (long long)dims[k - pad] : 1;
        P->n[k] = n;
        xs[k].resize(L + 1);
        xs[k][L].resize(n);
        for (long long i = 0; i < n; i++) {
            xs[k][L][i] = (active[k] && ck) ? ck[i] : (double)i;
            if (!std::isfinite(xs[k][L][i]) || (i > 0 && !(xs[k][L][i] > xs[k][L][i - 1]))) return HPDR_ERR_ARG;
        }
        if (active[k] && ck) {
            P->coords.insert(P->coords.end(), ck, ck + n);
            ck += n;
        }
        for (int l = L; l >= 1; l--) {
            const auto &xf = xs[k][l];
            int m = (int)xf.size();
            int mc = active[k] ? coarsen(m) : 1;
            xs[k][l - 1].resize(mc);
            for (int j = 0; j < mc; j++) xs[k][l - 1][j] = active[k] ? xf[cpos_of(m, mc, j)] : 0.0;
        }
        for (int l = 0; l <= L; l++) P->m[k][l] = (int)xs[k][l].size();
    }
    for (int l = 0; l <= L; l++) P->N[l] = (long long)P->m[0][l] * P->m[1][l] * P->m[2][l];

    img->offF.assign((L + 1) * 3, TableOff());
    img->offD.assign((L + 1) * 3, TableOff());
    std::vector<unsigned char> &all = img->bytes;
    all.clear();
    auto append = [&](const void *p, size_t bytes) {
        size_t off = (all.size() + 255) & ~size_t(255);
        all.resize(off + bytes);
        std::memcpy(all.data() + off, p, bytes);
        return off;
    };
    P->corr_norm.assign(L + 1, 0.0);
    for (int l = 1; l <= L; l++) {
        double prod = 1.0;
        for (int k = 0; k < 3; k++) {
            HostTab t = build_tab(xs[k][l], xs[k][l - 1], active[k]);
            prod *= corr_norm_dim(t);
            for (int pass = 0; pass < 2; pass++) {
                TableOff &o = pass == 0 ? img->offF[l * 3 + k] : img->offD[l * 3 + k];
                auto put = [&](const std::vector<double> &v) {
                    if (pass == 0) { std::vector<float> c(v.begin(), v.end()); return append(c.data(), c.size() * 4); }
                    return append(v.data(), v.size() * 8);
                };
                o.wl = put(t.wl); o.wr = put(t.wr); o.tap = put(t.tap); o.ptap = put(t.ptap);
                o.sub = put(t.sub); o.cp = put(t.cp); o.inv_den = put(t.inv_den); o.etap = put(t.etap);
                o.mtap = put(t.mtap);
                o.efirst = append(t.efirst.data(), t.efirst.size() * sizeof(int));
            }
        }
        P->corr_norm[l] = prod;
    }
    if (!P->coords.empty()) P->coords_off = append(P->coords.data(), P->coords.size() * sizeof(double));
    if (all.empty()) all.resize(256);
    return HPDR_OK;
}

void bind_plan(Plan *P, const PlanImage &img, void *tables)
{
    P->tables = tables;
    char *base = (char *)tables;
    P->coords_dev = P->coords.empty() ? nullptr : (const double *)(base + P->coords_off);
    const int L = P->L;
    for (int l = 0; l <= L; l++) {
        P->gf[l].level = P->gd[l].level = l;
        P->gf[l].Nprev = P->gd[l].Nprev = l > 0 ? P->N[l - 1] : 0;
        for (int k = 0; k < 3; k++) {
            DimTables<float> &a = P->gf[l].dim[k];
            DimTables<double> &b = P->gd[l].dim[k];
            a.m = b.m = P->m[k][l];
            a.mc = b.mc = l > 0 ? P->m[k][l - 1] : P->m[k][l];
            if (l == 0) {
                a.wl = a.wr = a.tap = a.ptap = a.sub = a.cp = a.inv_den = a.etap = a.mtap = nullptr; a.efirst = nullptr;
                b.wl = b.wr = b.tap = b.ptap = b.sub = b.cp = b.inv_den = b.etap = b.mtap = nullptr; b.efirst = nullptr;
                continue;
            }
            const TableOff &o = img.offF[l * 3 + k], &q = img.offD[l * 3 + k];
            a.wl = (const float *)(base + o.wl); a.wr = (const float *)(base + o.wr);
            a.tap = (const float *)(base + o.tap); a.ptap = (const float *)(base + o.ptap);
            a.sub = (const float *)(base + o.sub); a.cp = (const float *)(base + o.cp);
            a.inv_den = (const float *)(base + o.inv_den); a.etap = (const float *)(base + o.etap);
            a.efirst = (const int *)(base + o.efirst);
            a.mtap = (const float *)(base + o.mtap);
            b.wl = (const double *)(base + q.wl); b.wr = (const double *)(base + q.wr);
            b.tap = (const double *)(base + q.tap); b.ptap = (const double *)(base + q.ptap);
            b.sub = (const double *)(base + q.sub); b.cp = (const double *)(base + q.cp);
            b.inv_den = (const double *)(base + q.inv_den); b.etap = (const double *)(base + q.etap);
            b.efirst = (const int *)(base + q.efirst);
            b.mtap = (const double *)(base + q.mtap);
        }
    }
}

hpdr_status get_plan(hpdr_ctx *ctx, int ndim, const size_t *dims, bool f64, Plan **out, const double *coords)
{
    if (ndim < 1 || ndim > 3 || !dims) return HPDR_ERR_ARG;
    for (int k = 0; k < ndim; k++)
        if (dims[k] < 2 || dims[k] > (size_t)(1u << 30)) return HPDR_ERR_ARG;
    std::string key = std::to_string(ndim) + (f64 ? "d" : "f");
    for (int k = 0; k < ndim; k++) key += ":" + std::to_string(dims[k]);
    size_t nco = 0;
    if (coords) {
        // plans of given coordinates are keyed by the coordinates' bytes
        for (int k = 0; k < ndim; k++) nco += dims[k];
        uint64_t hsh = 1469598103934665603ull;
        const unsigned char *cb = (const unsigned char *)coords;
        for (size_t i = 0; i < nco * sizeof(double); i++) hsh = (hsh ^ cb[i]) * 1099511628211ull;
        key += ":c" + std::to_string(hsh);
    }
    auto it = ctx->plans.find(key);
    if (it != ctx->plans.end()) {
        const Plan *Q = it->second;
        if (!coords || (Q->coords.size() == nco && memcmp(Q->coords.data(), coords, nco * sizeof(double)) == 0)) {
            *out = it->second;
            return HPDR_OK;
        }
        // a hash collision: build this plan under a longer key
        key += ":" + std::to_string(ctx->plans.size());
    }
    Plan *P = new Plan();
    PlanImage img;
    hpdr_status st = plan_image(ndim, dims, f64, P, &img, coords);
    if (st != HPDR_OK) { delete P; return st; }
    int dev_prev = -1;
    cudaGetDevice(&dev_prev);
    if (dev_prev != ctx->device) cudaSetDevice(ctx->device);
    void *tables = nullptr;
    cudaError_t e = cudaMalloc(&tables, img.bytes.size());
    if (e == cudaSuccess) e = cudaMemcpy(tables, img.bytes.data(), img.bytes.size(), cudaMemcpyHostToDevice);
    if (dev_prev != ctx->device) cudaSetDevice(dev_prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(tables);
        delete P;
        return e == cudaErrorMemoryAllocation ? HPDR_ERR_NOMEM : HPDR_ERR_CUDA;
    }
    bind_plan(P, img, tables);
    ctx->plans[key] = P;
    *out = P;
    return HPDR_OK;
}

unsigned long long g_launches = 0;

ProfScope::ProfScope(hpdr_ctx *c, const char *name, cudaStream_t st) : ctx(c), s(st)
{
    if (!ctx || !ctx->prof_on) return;
    if (ctx->prof_used + 2 > ctx->prof_pool.size()) return;
    int id = -1;
    for (size_t i = 0; i < ctx->prof_names.size(); i++)
        if (ctx->prof_names[i] == name) { id = (int)i; break; }
    if (id < 0) {
        id = (int)ctx->prof_names.size();
        ctx->prof_names.push_back(name);
        ctx->prof_ms.push_back(0.0);
        ctx->prof_cnt.push_back(0);
    }
    hpdr_prof_rec r;
    r.id = id;
    r.a = ctx->prof_pool[ctx->prof_used++];
    r.b = ctx->prof_pool[ctx->prof_used++];
    cudaEventRecord(r.a, s);
    slot = (int)ctx->prof_recs.size();
    ctx->prof_recs.push_back(r);
}

ProfScope::~ProfScope()
{
    if (slot >= 0) cudaEventRecord(ctx->prof_recs[slot].b, s);
}

hpdr_status ensure_workspace(hpdr_ctx *ctx, size_t bytes)
{
    if (ctx->ws.bytes >= bytes) return HPDR_OK;
    if (ctx->ws.base) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return HPDR_ERR_CUDA;
        cudaFree(ctx->ws.base);
        ctx->ws.base = nullptr;
        ctx->ws.bytes = 0;
    }
    size_t want = (bytes + (1u << 20) - 1) & ~size_t((1u << 20) - 1);
    cudaError_t e = cudaMalloc(&ctx->ws.base, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->ws.base = nullptr;
        return e == cudaErrorMemoryAllocation ? HPDR_ERR_NOMEM : HPDR_ERR_CUDA;
    }
    ctx->ws.bytes = want;
    return HPDR_OK;
}

}  // namespace hpdr
