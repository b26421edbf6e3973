/*
 * hierarchy.c -- FP64 oracle of the multilevel decomposition of Sec. IV-A
 * (Alg. 1: lerp, mass_trans, tridiag, add) and of its inverse and transposes.
 * TEST INFRASTRUCTURE ONLY (see hpdr_oracle.h).
 *
 * Readings of the paper fixed here:
 *   - The data is a piecewise multilinear function on the finest grid, node
 *     i of a dimension at coordinate i (unit spacing) or at the coordinate
 *     the caller gives (any strictly increasing values: MGARD's non-uniform
 *     grids).  Weights, mass matrices and the correction use the node
 *     coordinates of every level.  One level of coarsening keeps
 *     every other node of each dimension plus the last node, so sizes 2^j+1
 *     give uniform levels and other sizes give a short last interval.  All
 *     dimensions coarsen together; L is the smallest per-dimension count of
 *     coarsenings that reaches 2 nodes.
 *   - mc_l = (I - Pi_{l-1}) Q_l u on the nodes that are new on level l: the
 *     node value minus its multilinear interpolant from the coarse nodes.
 *   - The correction is the L2 projection of the piecewise-linear function
 *     carrying mc_l onto the coarse space:
 *         z = (M_{l-1})^{-1} P^T M_l w,    v_{l-1} = v|coarse + z,
 *     with M the P1 mass matrices and P the prolongation (interpolation),
 *     applied one dimension at a time because both are Kronecker products.
 */
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include "hpdr_oracle.h"
#include "oracle_internal.h"

/* ------------------------------------------------------------------------ */
/* Hierarchy (Sec. IV-A: the function is decomposed level by level).          */

static size_t coarsen_size(size_t m) { return (m % 2) ? (m + 1) / 2 : m / 2 + 1; }

static int dim_levels(size_t n)
{
    int c = 0;
    while (n > 2) { n = coarsen_size(n); c++; }
    return c;
}

int ohier_build(ohier *H, int d, const size_t *n, const double *coords)
{
    if (d < 1 || d > OMAXD || !n) return -1;
    memset(H, 0, sizeof(*H));
    H->d = d;
    int L = 1 << 30;
    for (int k = 0; k < d; k++) {
        if (n[k] < 2) return -1;
        H->n[k] = n[k];
        int lk = dim_levels(n[k]);
        if (lk < L) L = lk;
    }
    if (L > OMAXL) return -1;
    H->L = L;
    const double *ck = coords;
    for (int k = 0; k < d; k++) {
        H->m[k][L] = n[k];
        H->x[k][L] = (double *)malloc(n[k] * sizeof(double));
        if (!H->x[k][L]) return -1;
        for (size_t i = 0; i < n[k]; i++) {
            H->x[k][L][i] = ck ? ck[i] : (double)i;
            if (!isfinite(H->x[k][L][i]) || (i > 0 && !(H->x[k][L][i] > H->x[k][L][i - 1]))) return -1;
        }
        if (ck) ck += n[k];
        for (int l = L; l >= 1; l--) {
            size_t m = H->m[k][l];
            size_t mc = coarsen_size(m);
            H->m[k][l - 1] = mc;
            H->x[k][l - 1] = (double *)malloc(mc * sizeof(double));
            if (!H->x[k][l - 1]) return -1;
            for (size_t j = 0; j < mc; j++) H->x[k][l - 1][j] = H->x[k][l][ocpos(m, mc, j)];
        }
    }
    return 0;
}

void ohier_free(ohier *H)
{
    for (int k = 0; k < OMAXD; k++)
        for (int l = 0; l <= OMAXL; l++) { free(H->x[k][l]); H->x[k][l] = NULL; }
}

size_t ohier_count(const ohier *H, int l)
{
    size_t c = 1;
    for (int k = 0; k < H->d; k++) c *= H->m[k][l];
    return c;
}

/* level-l position of the coarse node j (level l-1), for a level of m nodes
 * whose coarsening has mc nodes */
size_t ocpos(size_t m, size_t mc, size_t j) { return (j + 1 < mc) ? 2 * j : m - 1; }

/* is position p of a level with m nodes kept on the next coarser level? */
int ois_coarse(size_t m, size_t p) { return (p % 2 == 0) || (p == m - 1); }

/* coarse index of a kept position p */
static size_t ocidx(size_t m, size_t p) { return (p == m - 1) ? coarsen_size(m) - 1 : p / 2; }

/* interpolation weights of a new position p from its coarse neighbours
 * p-1 (left) and p+1 (right): piecewise-linear in the coordinates x. */
static void interp_weights(const double *x, size_t p, double *wl, double *wr)
{
    double a = (double)x[p - 1], b = (double)x[p + 1], c = (double)x[p];
    *wl = (b - c) / (b - a);
    *wr = (c - a) / (b - a);
}

/* ------------------------------------------------------------------------ */
/* 1-D operators on one line.                                                  */

/* y = M x, the P1 mass matrix on coordinates xc[0..m-1]:
 * diagonal (h_{i-1}+h_i)/3, off-diagonal h_i/6. */
static void mass_mul(const double *xc, size_t m, const double *x, double *y)
{
    for (size_t i = 0; i < m; i++) {
        double hl = (i > 0) ? (double)(xc[i] - xc[i - 1]) : 0.0;
        double hr = (i + 1 < m) ? (double)(xc[i + 1] - xc[i]) : 0.0;
        double s = (hl + hr) / 3.0 * x[i];
        if (i > 0) s += hl / 6.0 * x[i - 1];
        if (i + 1 < m) s += hr / 6.0 * x[i + 1];
        y[i] = s;
    }
}

/* Solve M z = b in place (Thomas algorithm), M the mass matrix on xc. */
static void mass_solve(const double *xc, size_t m, double *b)
{
    double *cp = (double *)malloc(m * sizeof(double));
    double diag0 = (double)(xc[1] - xc[0]) / 3.0;
    double off0 = (double)(xc[1] - xc[0]) / 6.0;
    cp[0] = off0 / diag0;
    b[0] = b[0] / diag0;
    for (size_t i = 1; i < m; i++) {
        double hl = (double)(xc[i] - xc[i - 1]);
        double hr = (i + 1 < m) ? (double)(xc[i + 1] - xc[i]) : 0.0;
        double diag = (hl + hr) / 3.0, sub = hl / 6.0, sup = hr / 6.0;
        double den = diag - sub * cp[i - 1];
        cp[i] = sup / den;
        b[i] = (b[i] - sub * b[i - 1]) / den;
    }
    for (size_t i = m - 1; i-- > 0;) b[i] = b[i] - cp[i] * b[i + 1];
    free(cp);
}

/* out = P^T y for a level with coordinates xf (m nodes) and its coarsening
 * (mc nodes): every coarse node collects its own value and, from each new
 * neighbour, the interpolation weight that neighbour gives it. */
static void prolong_T(const double *xf, size_t m, size_t mc, const double *y, double *out)
{
    for (size_t j = 0; j < mc; j++) {
        size_t c = ocpos(m, mc, j);
        double s = y[c];
        double wl, wr;
        if (c >= 1 && !ois_coarse(m, c - 1)) { interp_weights(xf, c - 1, &wl, &wr); s += wr * y[c - 1]; }
        if (c + 1 < m && !ois_coarse(m, c + 1)) { interp_weights(xf, c + 1, &wl, &wr); s += wl * y[c + 1]; }
        out[j] = s;
    }
}

/* out = P z: coarse values copied, new positions interpolated */
static void prolong(const double *xf, size_t m, size_t mc, const double *z, double *out)
{
    for (size_t p = 0; p < m; p++) {
        if (ois_coarse(m, p)) { out[p] = z[ocidx(m, p)]; continue; }
        double wl, wr;
        interp_weights(xf, p, &wl, &wr);
        out[p] = wl * z[ocidx(m, p - 1)] + wr * z[ocidx(m, p + 1)];
    }
    (void)mc;
}

/* ------------------------------------------------------------------------ */
/* Operators along one dimension of a d-dimensional row-major array.           */

enum { OP_RESTRICT, OP_SOLVE, OP_MASS_PROLONG };

/* Apply op along dim k.  a has shape s; the result b has shape s with s[k]
 * replaced by mo.  Level l is the fine level of the pair (l, l-1). */
static void along_dim(const ohier *H, int l, int op, const size_t *s, int k,
                      const double *a, size_t mo, double *b)
{
    size_t inner = 1, outer = 1;
    for (int j = k + 1; j < H->d; j++) inner *= s[j];
    for (int j = 0; j < k; j++) outer *= s[j];
    size_t mi = s[k];
    size_t mmax = (mi > mo) ? mi : mo;
    double *lin = (double *)malloc(mmax * sizeof(double));
    double *tmp = (double *)malloc(mmax * sizeof(double));
    double *lout = (double *)malloc(mmax * sizeof(double));
    const double *xf = H->x[k][l];
    const double *xc = H->x[k][l - 1];
    size_t mf = H->m[k][l], mcn = H->m[k][l - 1];
    for (size_t o = 0; o < outer; o++) {
        for (size_t i = 0; i < inner; i++) {
            for (size_t p = 0; p < mi; p++) lin[p] = a[(o * mi + p) * inner + i];
            if (op == OP_RESTRICT) {          /* (P^T M_l) : fine -> coarse */
                mass_mul(xf, mf, lin, tmp);
                prolong_T(xf, mf, mcn, tmp, lout);
            } else if (op == OP_SOLVE) {      /* M_{l-1}^{-1} : coarse -> coarse */
                memcpy(lout, lin, mi * sizeof(double));
                mass_solve(xc, mcn, lout);
            } else {                          /* (M_l P) : coarse -> fine */
                prolong(xf, mf, mcn, lin, tmp);
                mass_mul(xf, mf, tmp, lout);
            }
            for (size_t p = 0; p < mo; p++) b[(o * mo + p) * inner + i] = lout[p];
        }
    }
    free(lin); free(tmp); free(lout);
}

/* z = (x)_k M_{l-1}^{-1} (x)_k P^T M_l w, w on the level-l grid, z on level l-1 */
static double *correction(const ohier *H, int l, const double *w)
{
    size_t s[OMAXD];
    for (int k = 0; k < H->d; k++) s[k] = H->m[k][l];
    size_t cnt = ohier_count(H, l);
    double *t = (double *)malloc(cnt * sizeof(double));
    memcpy(t, w, cnt * sizeof(double));
    for (int k = 0; k < H->d; k++) {
        size_t mo = H->m[k][l - 1];
        size_t ncnt = cnt / s[k] * mo;
        double *t2 = (double *)malloc(ncnt * sizeof(double));
        along_dim(H, l, OP_RESTRICT, s, k, t, mo, t2);
        free(t); t = t2; s[k] = mo; cnt = ncnt;
    }
    for (int k = 0; k < H->d; k++) {
        double *t2 = (double *)malloc(cnt * sizeof(double));
        along_dim(H, l, OP_SOLVE, s, k, t, s[k], t2);
        free(t); t = t2;
    }
    return t;
}

/* y = (x)_k M_l P_k (x)_k M_{l-1}^{-1} g, g on level l-1, y on level l:
 * the transpose of correction() */
static double *correction_T(const ohier *H, int l, const double *g)
{
    size_t s[OMAXD];
    for (int k = 0; k < H->d; k++) s[k] = H->m[k][l - 1];
    size_t cnt = ohier_count(H, l - 1);
    double *t = (double *)malloc(cnt * sizeof(double));
    memcpy(t, g, cnt * sizeof(double));
    for (int k = 0; k < H->d; k++) {
        double *t2 = (double *)malloc(cnt * sizeof(double));
        along_dim(H, l, OP_SOLVE, s, k, t, s[k], t2);
        free(t); t = t2;
    }
    for (int k = 0; k < H->d; k++) {
        size_t mo = H->m[k][l];
        size_t ncnt = cnt / s[k] * mo;
        double *t2 = (double *)malloc(ncnt * sizeof(double));
        along_dim(H, l, OP_MASS_PROLONG, s, k, t, mo, t2);
        free(t); t = t2; s[k] = mo; cnt = ncnt;
    }
    return t;
}

/* ------------------------------------------------------------------------ */
/* Node helpers on the level-l grid.                                           */

static void unflatten(const ohier *H, int l, size_t f, size_t *p)
{
    for (int k = H->d - 1; k >= 0; k--) { p[k] = f % H->m[k][l]; f /= H->m[k][l]; }
}

static size_t flatten(const ohier *H, int l, const size_t *p)
{
    size_t f = 0;
    for (int k = 0; k < H->d; k++) f = f * H->m[k][l] + p[k];
    return f;
}

static int all_coarse(const ohier *H, int l, const size_t *p)
{
    for (int k = 0; k < H->d; k++) if (!ois_coarse(H->m[k][l], p[k])) return 0;
    return 1;
}

/* Corners of the multilinear interpolant at node p of level l: for each dim,
 * a kept position contributes itself with weight 1 and a new position its two
 * neighbours with the piecewise-linear weights.  Returns the corner count;
 * corner i is the level-l flat index cf[i] (a node kept on level l-1), its
 * level-(l-1) flat index cc[i] and its weight cw[i]. */
static int corners(const ohier *H, int l, const size_t *p, size_t *cf, size_t *cc, double *cw)
{
    int nc = 1;
    size_t pf[8][OMAXD];
    double w[8];
    w[0] = 1.0;
    for (int k = 0; k < H->d; k++) pf[0][k] = p[k];
    for (int k = 0; k < H->d; k++) {
        size_t m = H->m[k][l];
        if (ois_coarse(m, p[k])) continue;
        double wl, wr;
        interp_weights(H->x[k][l], p[k], &wl, &wr);
        for (int i = 0; i < nc; i++) {
            for (int j = 0; j < H->d; j++) pf[nc + i][j] = pf[i][j];
            pf[i][k] = p[k] - 1;
            pf[nc + i][k] = p[k] + 1;
            w[nc + i] = w[i] * wr;
            w[i] = w[i] * wl;
        }
        nc *= 2;
    }
    for (int i = 0; i < nc; i++) {
        size_t q[OMAXD];
        for (int k = 0; k < H->d; k++) q[k] = ocidx(H->m[k][l], pf[i][k]);
        cf[i] = flatten(H, l, pf[i]);
        cc[i] = flatten(H, l - 1, q);
        cw[i] = w[i];
    }
    return nc;
}

/* ------------------------------------------------------------------------ */
/* Alg. 1: decomposition.                                                      */

int oracle_levels(int d, const size_t *n, int *L, size_t *m_out)
{
    ohier H;
    if (ohier_build(&H, d, n, NULL)) { ohier_free(&H); return -1; }
    *L = H.L;
    if (m_out)
        for (int k = 0; k < 3; k++)
            for (int l = 0; l <= H.L; l++) m_out[k * (H.L + 1) + l] = (k < d) ? H.m[k][l] : 1;
    ohier_free(&H);
    return 0;
}

int oracle_decompose(int d, const size_t *n, const double *u, double *coef)
{
    return oracle_decompose_c(d, n, NULL, u, coef);
}

int oracle_decompose_c(int d, const size_t *n, const double *coords, const double *u, double *coef)
{
    ohier H;
    if (ohier_build(&H, d, n, coords)) { ohier_free(&H); return -1; }
    size_t N = ohier_count(&H, H.L);
    double *v = (double *)malloc(N * sizeof(double));
    memcpy(v, u, N * sizeof(double));
    for (int l = H.L; l >= 1; l--) {
        size_t Nf = ohier_count(&H, l), Nc = ohier_count(&H, l - 1);
        double *w = (double *)calloc(Nf, sizeof(double));
        size_t r = Nc;                       /* level l's section starts at N_{l-1} */
        for (size_t f = 0; f < Nf; f++) {
            size_t p[OMAXD], cf[8], cc[8];
            double cw[8];
            unflatten(&H, l, f, p);
            if (all_coarse(&H, l, p)) continue;
            int nc = corners(&H, l, p, cf, cc, cw);
            double lerp = 0.0;                 /* Pi_{l-1} Q_l u at p ("lerp") */
            for (int i = 0; i < nc; i++) lerp += cw[i] * v[cf[i]];
            double mc = v[f] - lerp;
            w[f] = mc;
            coef[r++] = mc;
        }
        double *z = correction(&H, l, w);    /* mass_trans + tridiag */
        double *vc = (double *)malloc(Nc * sizeof(double));
        for (size_t c = 0; c < Nc; c++) {    /* add(correction) */
            size_t q[OMAXD], p[OMAXD];
            unflatten(&H, l - 1, c, q);
            for (int k = 0; k < H.d; k++) p[k] = ocpos(H.m[k][l], H.m[k][l - 1], q[k]);
            vc[c] = v[flatten(&H, l, p)] + z[c];
        }
        free(w); free(z); free(v);
        v = vc;
    }
    memcpy(coef, v, ohier_count(&H, 0) * sizeof(double));
    free(v);
    ohier_free(&H);
    return 0;
}

/* Inverse of Alg. 1: for l = 1..L, remove the correction from the coarse
 * values, then rebuild the new nodes as coefficient plus interpolant. */
int oracle_recompose(int d, const size_t *n, const double *coef, double *u)
{
    return oracle_recompose_c(d, n, NULL, coef, u);
}

int oracle_recompose_c(int d, const size_t *n, const double *coords, const double *coef, double *u)
{
    ohier H;
    if (ohier_build(&H, d, n, coords)) { ohier_free(&H); return -1; }
    size_t N0 = ohier_count(&H, 0);
    double *v = (double *)malloc(N0 * sizeof(double));
    memcpy(v, coef, N0 * sizeof(double));
    for (int l = 1; l <= H.L; l++) {
        size_t Nf = ohier_count(&H, l), Nc = ohier_count(&H, l - 1);
        double *w = (double *)calloc(Nf, sizeof(double));
        size_t r = Nc;
        for (size_t f = 0; f < Nf; f++) {
            size_t p[OMAXD];
            unflatten(&H, l, f, p);
            if (!all_coarse(&H, l, p)) w[f] = coef[r++];
        }
        double *z = correction(&H, l, w);
        double *vf = (double *)malloc(Nf * sizeof(double));
        for (size_t c = 0; c < Nc; c++) {
            size_t q[OMAXD], p[OMAXD];
            unflatten(&H, l - 1, c, q);
            for (int k = 0; k < H.d; k++) p[k] = ocpos(H.m[k][l], H.m[k][l - 1], q[k]);
            vf[flatten(&H, l, p)] = v[c] - z[c];
        }
        for (size_t f = 0; f < Nf; f++) {
            size_t p[OMAXD], cf[8], cc[8];
            double cw[8];
            unflatten(&H, l, f, p);
            if (all_coarse(&H, l, p)) continue;
            int nc = corners(&H, l, p, cf, cc, cw);
            double lerp = 0.0;
            for (int i = 0; i < nc; i++) lerp += cw[i] * vf[cf[i]];
            vf[f] = w[f] + lerp;
        }
        free(w); free(z); free(v);
        v = vf;
    }
    memcpy(u, v, ohier_count(&H, H.L) * sizeof(double));
    free(v);
    ohier_free(&H);
    return 0;
}

/* Transpose of recomposition.  One level of recomposition is
 *   v_l = P (v_{l-1} - S c_l) + E_f c_l,  S = correction restricted to new nodes,
 * so, from the level-l gradient g_l,
 *   g_{v_{l-1}} = P^T g_l,   g_{c_l} = g_l|new - S^T P^T g_l. */
int oracle_recompose_adjoint(int d, const size_t *n, const double *g_u, double *g_coef)
{
    return oracle_recompose_adjoint_c(d, n, NULL, g_u, g_coef);
}

int oracle_recompose_adjoint_c(int d, const size_t *n, const double *coords, const double *g_u, double *g_coef)
{
    ohier H;
    if (ohier_build(&H, d, n, coords)) { ohier_free(&H); return -1; }
    size_t N = ohier_count(&H, H.L);
    double *g = (double *)malloc(N * sizeof(double));
    memcpy(g, g_u, N * sizeof(double));
    for (int l = H.L; l >= 1; l--) {
        size_t Nf = ohier_count(&H, l), Nc = ohier_count(&H, l - 1);
        double *gc = (double *)malloc(Nc * sizeof(double));
        for (size_t c = 0; c < Nc; c++) {    /* P^T g_l: kept nodes first */
            size_t q[OMAXD], p[OMAXD];
            unflatten(&H, l - 1, c, q);
            for (int k = 0; k < H.d; k++) p[k] = ocpos(H.m[k][l], H.m[k][l - 1], q[k]);
            gc[c] = g[flatten(&H, l, p)];
        }
        for (size_t f = 0; f < Nf; f++) {    /* ... then what the new nodes interpolated */
            size_t p[OMAXD], cf[8], cc[8];
            double cw[8];
            unflatten(&H, l, f, p);
            if (all_coarse(&H, l, p)) continue;
            int nc = corners(&H, l, p, cf, cc, cw);
            for (int i = 0; i < nc; i++) gc[cc[i]] += cw[i] * g[f];
        }
        double *y = correction_T(&H, l, gc);
        size_t r = Nc;
        for (size_t f = 0; f < Nf; f++) {
            size_t p[OMAXD];
            unflatten(&H, l, f, p);
            if (all_coarse(&H, l, p)) continue;
            g_coef[r++] = g[f] - y[f];
        }
        free(y); free(g);
        g = gc;
    }
    memcpy(g_coef, g, ohier_count(&H, 0) * sizeof(double));
    free(g);
    ohier_free(&H);
    return 0;
}

/* Transpose of decomposition.  One level of decomposition is
 *   c_l = A v_l,  A v = (v - P v|kept)|new,   v_{l-1} = v_l|kept + S c_l,
 * so, from the gradients g_{c_l} and g_{v_{l-1}},
 *   h = g_{c_l} + S^T g_{v_{l-1}},
 *   g_{v_l} = E_new h + E_kept (g_{v_{l-1}} - P^T E_new h). */
int oracle_decompose_adjoint(int d, const size_t *n, const double *g_coef, double *g_u)
{
    return oracle_decompose_adjoint_c(d, n, NULL, g_coef, g_u);
}

int oracle_decompose_adjoint_c(int d, const size_t *n, const double *coords, const double *g_coef, double *g_u)
{
    ohier H;
    if (ohier_build(&H, d, n, coords)) { ohier_free(&H); return -1; }
    size_t N0 = ohier_count(&H, 0);
    double *gv = (double *)malloc(N0 * sizeof(double));
    memcpy(gv, g_coef, N0 * sizeof(double));
    for (int l = 1; l <= H.L; l++) {
        size_t Nf = ohier_count(&H, l), Nc = ohier_count(&H, l - 1);
        double *y = correction_T(&H, l, gv);
        double *gn = (double *)calloc(Nf, sizeof(double));
        double *gcc = (double *)malloc(Nc * sizeof(double));
        memcpy(gcc, gv, Nc * sizeof(double));
        size_t r = Nc;
        for (size_t f = 0; f < Nf; f++) {
            size_t p[OMAXD], cf[8], cc[8];
            double cw[8];
            unflatten(&H, l, f, p);
            if (all_coarse(&H, l, p)) continue;
            double h = g_coef[r++] + y[f];
            gn[f] = h;
            int nc = corners(&H, l, p, cf, cc, cw);
            for (int i = 0; i < nc; i++) gcc[cc[i]] -= cw[i] * h;
        }
        for (size_t c = 0; c < Nc; c++) {
            size_t q[OMAXD], p[OMAXD];
            unflatten(&H, l - 1, c, q);
            for (int k = 0; k < H.d; k++) p[k] = ocpos(H.m[k][l], H.m[k][l - 1], q[k]);
            gn[flatten(&H, l, p)] = gcc[c];
        }
        free(y); free(gcc); free(gv);
        gv = gn;
    }
    memcpy(g_u, gv, ohier_count(&H, H.L) * sizeof(double));
    free(gv);
    ohier_free(&H);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Level-scaled bins (Sec. IV-A: a different bin size for each level).         */

/* c_l = prod_k ||G_k||_inf with G_k = M_{l-1}^{-1} P^T M_l along dim k: the
 * infinity-norm amplification of one level's correction. */
int oracle_correction_norms(int d, const size_t *n, double *c)
{
    return oracle_correction_norms_c(d, n, NULL, c);
}

int oracle_correction_norms_c(int d, const size_t *n, const double *coords, double *c)
{
    ohier H;
    if (ohier_build(&H, d, n, coords)) { ohier_free(&H); return -1; }
    c[0] = 0.0;
    for (int l = 1; l <= H.L; l++) {
        double prod = 1.0;
        for (int k = 0; k < H.d; k++) {
            size_t mf = H.m[k][l], mc = H.m[k][l - 1];
            double *rows = (double *)calloc(mc, sizeof(double));
            double *e = (double *)calloc(mf, sizeof(double));
            double *t = (double *)malloc(mf * sizeof(double));
            double *col = (double *)malloc(mc * sizeof(double));
            for (size_t p = 0; p < mf; p++) {
                memset(e, 0, mf * sizeof(double));
                e[p] = 1.0;
                mass_mul(H.x[k][l], mf, e, t);
                prolong_T(H.x[k][l], mf, mc, t, col);
                mass_solve(H.x[k][l - 1], mc, col);
                for (size_t i = 0; i < mc; i++) rows[i] += fabs(col[i]);
            }
            double mx = 0.0;
            for (size_t i = 0; i < mc; i++) if (rows[i] > mx) mx = rows[i];
            prod *= mx;
            free(rows); free(e); free(t); free(col);
        }
        c[l] = prod;
    }
    ohier_free(&H);
    return 0;
}

/* q_0 = 2 tau'/(L+1), q_l = 2 tau'/((L+1)(1+c_l)) with
 * tau' = tau_abs - 32 (L+1) eps ||u||_inf.  Recomposing level l moves every
 * node by at most (1+c_l) q_l / 2 and interpolation does not grow errors, so
 * the reconstruction error stays below tau'.  A field of zeros gets unit bins
 * (all codes are zero and the reconstruction is exact). */
int oracle_bins(int d, const size_t *n, double tau_abs, double norm_inf, double eps, double *q)
{
    return oracle_bins_c(d, n, NULL, tau_abs, norm_inf, eps, q);
}

int oracle_bins_c(int d, const size_t *n, const double *coords, double tau_abs, double norm_inf, double eps,
                  double *q)
{
    int L;
    if (oracle_levels(d, n, &L, NULL)) return -1;
    if (norm_inf == 0.0) {
        for (int l = 0; l <= L; l++) q[l] = 1.0;
        return 0;
    }
    double tp = tau_abs - 32.0 * (double)(L + 1) * eps * norm_inf;
    if (!(tp > 0.0)) return -2;
    double *c = (double *)malloc((size_t)(L + 1) * sizeof(double));
    if (oracle_correction_norms_c(d, n, coords, c)) { free(c); return -1; }
    q[0] = 2.0 * tp / (double)(L + 1);
    for (int l = 1; l <= L; l++) q[l] = 2.0 * tp / ((double)(L + 1) * (1.0 + c[l]));
    free(c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Statistical L2 bins (mode 2).  The paper gives no formula for an L2 bound,
 * so this reading is fixed here.  The level components (Q_l - Q_{l-1}) u are
 * L2-orthogonal, so coefficient errors delta_l on the new nodes of level l
 * reach the reconstruction as (I - Q_{l-1}) f_l with f_l = sum_i delta_i
 * phi_i (level-l hat functions), and ||u - u~||^2 <= sum_l ||f_l||^2.  With
 * errors independent and uniform on [-q_l/2, q_l/2], E||f_l||^2 =
 * (q_l^2 / 12) S_l, S_l = sum over the new nodes of the mass-matrix diagonal.
 * The budget is tau'^2 T, T = trace of the finest mass matrix (the L2 norm of
 * a field of uncorrelated nodal errors of RMS tau'), split evenly over the
 * L + 1 levels:  q_l = sqrt(12 tau'^2 T / ((L+1) S_l)).  tau' carries the
 * same precision margin as the max-norm bins.  The bound is on the expected
 * error, not on every field. */

/* diagonal entry i of the 1-D P1 mass matrix on nodes x[0..m-1] */
static double mass_diag(const double *x, size_t m, size_t i)
{
    double h = 0.0;
    if (i > 0) h += x[i] - x[i - 1];
    if (i + 1 < m) h += x[i + 1] - x[i];
    return h / 3.0;
}

/* compensated (Neumaier) running sum: the sums below run over every node of
 * a level, and a plain recursive sum of n terms may drift by n units of
 * roundoff; this one stays within a few */
typedef struct { double s, c; } ksum;
static void ksum_add(ksum *k, double x)
{
    double t = k->s + x;
    if (fabs(k->s) >= fabs(x)) k->c += (k->s - t) + x;
    else k->c += (x - t) + k->s;
    k->s = t;
}

int oracle_l2s_weights_c(int d, const size_t *n, const double *coords, double *S, double *T)
{
    ohier H;
    if (ohier_build(&H, d, n, coords)) { ohier_free(&H); return -1; }
    for (int l = 0; l <= H.L; l++) {
        /* every node of level l, row-major; new unless kept in every dimension */
        size_t cnt = ohier_count(&H, l);
        ksum sum = {0.0, 0.0}, all = {0.0, 0.0};
        size_t p[OMAXD] = {0};
        for (size_t idx = 0; idx < cnt; idx++) {
            size_t r = idx;
            for (int k = H.d - 1; k >= 0; k--) { p[k] = r % H.m[k][l]; r /= H.m[k][l]; }
            double w = 1.0;
            int kept = 1;
            for (int k = 0; k < H.d; k++) {
                w *= mass_diag(H.x[k][l], H.m[k][l], p[k]);
                if (!ois_coarse(H.m[k][l], p[k])) kept = 0;
            }
            ksum_add(&all, w);
            if (l == 0 || !kept) ksum_add(&sum, w);
        }
        S[l] = sum.s + sum.c;
        if (l == H.L) *T = all.s + all.c;
    }
    ohier_free(&H);
    return 0;
}

int oracle_bins_l2s_c(int d, const size_t *n, const double *coords, double tau_abs, double norm_inf, double eps,
                      double *q)
{
    int L;
    if (oracle_levels(d, n, &L, NULL)) return -1;
    if (norm_inf == 0.0) {
        for (int l = 0; l <= L; l++) q[l] = 1.0;
        return 0;
    }
    double tp = tau_abs - 32.0 * (double)(L + 1) * eps * norm_inf;
    if (!(tp > 0.0)) return -2;
    double *S = (double *)malloc((size_t)(L + 1) * sizeof(double));
    double T = 0.0;
    if (oracle_l2s_weights_c(d, n, coords, S, &T)) { free(S); return -1; }
    for (int l = 0; l <= L; l++) q[l] = sqrt(12.0 * (tp * tp) * T / ((double)(L + 1) * S[l]));
    free(S);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Linear quantization (MapAndProcess over levels, Sec. IV-A).                 */

/* level of stream index i: level l occupies [N_{l-1}, N_l) (level 0: [0, N_0)) */
static int level_of(const size_t *Nl, int L, uint64_t i)
{
    int l = 0;
    while (l < L && i >= Nl[l]) l++;
    return l;
}

/* k = sign(x) floor(|x| rho + 1/2), rho = 1/q rounded to the working
 * precision; in binary32 mode every operation is rounded to binary32. */
static int64_t quant1(double x, double q, int precision)
{
    if (precision == 32) {
        volatile float rho = (float)(1.0 / q);
        volatile float ax = (float)fabs(x);
        volatile float y = ax * rho;
        volatile float t = y + 0.5f;
        int64_t k = (int64_t)floorf(t);
        return (x < 0) ? -k : k;
    }
    volatile double rho = 1.0 / q;
    volatile double y = fabs(x) * rho;
    volatile double t = y + 0.5;
    int64_t k = (int64_t)floor(t);
    return (x < 0) ? -k : k;
}

int oracle_quantize(int d, const size_t *n, const double *coef, const double *q, int precision,
                    uint32_t D, uint16_t *symbols, uint64_t *n_out,
                    uint64_t *out_idx, int64_t *out_k, uint64_t out_cap)
{
    ohier H;
    if (D < 4 || D > 65536 || (D % 2)) return -1;
    if (ohier_build(&H, d, n, NULL)) { ohier_free(&H); return -1; }
    size_t Nl[OMAXL + 1];
    for (int l = 0; l <= H.L; l++) Nl[l] = ohier_count(&H, l);
    uint64_t N = Nl[H.L], no = 0;
    int64_t half = (int64_t)(D / 2);
    for (uint64_t i = 0; i < N; i++) {
        int l = level_of(Nl, H.L, i);
        int64_t k = quant1(coef[i], q[l], precision);
        int64_t s = k + half;
        if (s >= 1 && s <= (int64_t)D - 1) {
            symbols[i] = (uint16_t)s;
        } else {
            symbols[i] = 0;
            if (out_idx && no < out_cap) { out_idx[no] = i; out_k[no] = k; }
            no++;
        }
    }
    *n_out = no;
    ohier_free(&H);
    return 0;
}

int oracle_dequantize(int d, const size_t *n, const uint16_t *symbols, const double *q, uint32_t D,
                      uint64_t n_out, const uint64_t *out_idx, const int64_t *out_k, double *coef)
{
    ohier H;
    if (ohier_build(&H, d, n, NULL)) { ohier_free(&H); return -1; }
    size_t Nl[OMAXL + 1];
    for (int l = 0; l <= H.L; l++) Nl[l] = ohier_count(&H, l);
    uint64_t N = Nl[H.L], j = 0;
    int64_t half = (int64_t)(D / 2);
    for (uint64_t i = 0; i < N; i++) {
        int l = level_of(Nl, H.L, i);
        int64_t k;
        if (symbols[i] != 0) {
            k = (int64_t)symbols[i] - half;
        } else {
            if (j >= n_out || out_idx[j] != i) { ohier_free(&H); return -4; }
            k = out_k[j++];
        }
        coef[i] = (double)k * q[l];
    }
    ohier_free(&H);
    return (j == n_out) ? 0 : -4;
}
