// levels.cuh -- launchers of the per-level kernels (levels.cu).
#pragma once
#include "internal.cuh"

namespace hpdr {

// Where a restriction reads its fine-level values w from.
enum class WSrc : int {
    FIELD = 0,     // w = new-node coefficients computed from a level-l field (Alg. 1 lerp)
    STREAM = 1,    // w = coefficients read from a level-major stream (type T)
    SYMBOLS = 2,   // w = dequantized symbols of a level-major stream
    DENSE = 3,     // w = a dense level-l array (all nodes; used by the transposes)
};
// What the FIELD source does with the coefficients it computes.
enum class Sink : int { NONE = 0, STREAM = 1, QUANT = 2 };

struct QuantOut {
    uint16_t *sym;                 // stream of symbols
    unsigned long long *hist;      // global histogram [D]
    long long *esc;                // [N] code k at every escaped stream position (symbol 0)
    unsigned int D;
    Scalars *sc;
};

struct SymIn {
    const uint16_t *sym;
    unsigned int D;
    const Scalars *sc;               // q per level
    const long long *esc;            // [N] code k at every escaped stream position
    unsigned int *status;
};

template <typename T>
struct RestrictArgs {
    LevelGeom<T> g;
    const T *v;          // FIELD / DENSE: level-l array
    const T *coef_in;    // STREAM source
    SymIn symin;         // SYMBOLS source
    T *coef_out;         // Sink::STREAM
    QuantOut qo;         // Sink::QUANT
    T *b;                // coarse output (level l-1 grid)
    T *vc;               // coarse copy of v (FIELD with a sink), may be null
    int use_ptap;        // 0: P^T M_l taps, 1: P^T taps
    int dense_new_only;  // DENSE: 1 = use only the new nodes (E_new^T of the input)
    const void *src_end; // one past the last byte of the staged source (FIELD: v, SYMBOLS: sym)
    unsigned int *status;  // device status word (timeouts)
    int wait_limit;      // polls of a pipeline wait before it gives up (0: use the library's limit)
};

template <typename T>
cudaError_t launch_restrict(WSrc src, Sink sink, const RestrictArgs<T> &a, cudaStream_t s);

// decomp.cu: the level kernel of decomposition and compression (FIELD
// source; Sink::QUANT or Sink::STREAM) and the restriction of decompression
// (SYMBOLS source), warp-specialised plane pipelines.
template <typename T>
cudaError_t launch_decomp(Sink sink, const RestrictArgs<T> &a, cudaStream_t s);
template <typename T>
cudaError_t launch_restrict_symbols(const RestrictArgs<T> &a, cudaStream_t s);
// the same plane pipeline over any decompression-side source: SYMBOLS,
// STREAM (a coefficient stream) or DENSE (a level-l grid, all or new nodes)
template <typename T>
cudaError_t launch_restrict_planes(WSrc src, const RestrictArgs<T> &a, cudaStream_t s);
template <typename T>
cudaError_t launch_expand_planes(WSrc src, const LevelGeom<T> &g, const T *vc, const T *coef_in,
                                 const SymIn &symin, T *out, cudaStream_t s);

// Polls of a bounded pipeline wait before the kernel gives up with
// DS_TIMEOUT (set through hpdr_debug_set_wait_limit; default kWaitPolls).
// The drain of copies in flight after a give-up always uses kWaitPolls.
extern int g_wait_limit;

// Solve (x)_k M_{l-1} along every active dimension of the coarse array b, in
// place; the last solve optionally adds (sign=+1) or subtracts (sign=-1) the
// result into vc instead of storing it into b.
template <typename T>
cudaError_t launch_solves(const LevelGeom<T> &g, T *b, T *vc, int sign, cudaStream_t s);

// Recomposition of level l: out (level-l grid) = kept nodes from vc (level
// l-1 grid), new nodes = coefficient + interpolant of vc.
template <typename T>
cudaError_t launch_expand(WSrc src, const LevelGeom<T> &g, const T *vc, const T *coef_in,
                          const SymIn &symin, T *out, cudaStream_t s);

// Level 0: quantize (Sink::QUANT) or copy (Sink::STREAM) the coarsest grid.
template <typename T>
cudaError_t launch_level0(Sink sink, const T *v0, long long N0, T *coef_out, const QuantOut &qo,
                          cudaStream_t s);
// Level 0 of recomposition: v0 = coefficient stream entries [0, N0).
template <typename T>
cudaError_t launch_level0_in(WSrc src, const T *coef_in, const SymIn &symin, long long N0, T *v0,
                             cudaStream_t s);

// max|u| and sum u^2 (deterministic), then bins (one thread block).
template <typename T>
cudaError_t launch_norm(const T *u, long long N, double *partials, int nparts, cudaStream_t s);
struct BinArgs {
    int L;
    double c[kMaxLevels + 1];
    double tol;
    int tol_kind, mode;
    double eps;
    long long N;
};
cudaError_t launch_bins(const BinArgs &ba, const double *partials, int nparts, Scalars *sc,
                        cudaStream_t s);

// Transposes: dense level-l array from a coarse array through (x)_k M_l P
template <typename T>
cudaError_t launch_mass_prolong(const LevelGeom<T> &g, const T *yc, T *yf, T *tmp,
                                cudaStream_t s);

int norm_parts();

// The coarse levels in one CTA (levels.cu): levels 1..ls and level 0, with
// ls = coarse_top(), the largest level whose shared arrays fit kCoarseSmem.
// mode 0: compression (v_in -> symbols), 1: decomposition (v_in -> coef_out),
// 2: decompression (symbols -> v_out), 3: recomposition (coef_in -> v_out).
constexpr int kCoarseMaxLevels = 16;
constexpr size_t kCoarseSmem = 200 * 1024;
template <typename T>
int coarse_top(const Plan *P, const LevelGeom<T> *geo);
template <typename T>
struct CoarseArgs {
    LevelGeom<T> g[kCoarseMaxLevels + 1];   // levels 1..ls
    int ls;
    long long N0;
    const T *v_in;       // compression / decomposition: the level-ls grid
    T *v_out;            // recomposition: the level-ls grid
    QuantOut qo;         // compression
    T *coef_out;         // decomposition
    SymIn symin;         // decompression
    const T *coef_in;    // recomposition
};
template <typename T>
cudaError_t launch_coarse(int mode, const Plan *P, const LevelGeom<T> *geo, int ls, const T *v_in, T *v_out,
                          const QuantOut &qo, T *coef_out, const SymIn &symin, const T *coef_in, cudaStream_t s);
// the arguments of that launch (host), and its dynamic shared memory
template <typename T>
CoarseArgs<T> coarse_args(const Plan *P, const LevelGeom<T> *geo, int ls, const T *v_in, T *v_out,
                          const QuantOut &qo, T *coef_out, const SymIn &symin, const T *coef_in, size_t *smem);
// the coarse levels of n fields in one launch (one block per field; jobs:
// device [n]; smem: the largest of the fields' shared-memory sizes)
template <typename T>
cudaError_t launch_coarse_batch(int mode, const CoarseArgs<T> *jobs, int n, size_t smem, cudaStream_t s);

// adjoint.cu: transposes of recomposition / decomposition over all levels.
// ga, gb, y, R hold N_{L-1} elements; t1, t2 the partial prolongations
// (max over levels of c0*c1*m2 and c0*m1*m2 elements).
template <typename T>
cudaError_t recompose_adjoint_run(const Plan &P, const LevelGeom<T> *geo, const T *gu, T *gcoef, T *ga, T *gb,
                                  T *y, T *t1, T *t2, unsigned *status, cudaStream_t s);
template <typename T>
cudaError_t decompose_adjoint_run(const Plan &P, const LevelGeom<T> *geo, const T *gcoef, T *gu, T *ga, T *gb,
                                  T *y, T *t1, T *t2, T *R, unsigned *status, cudaStream_t s);

}  // namespace hpdr
