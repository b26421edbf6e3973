"""Pins of the oracle's multilevel decomposition (Sec. IV-A, Alg. 1) against
what the mathematics fixes, independently of the oracle's own code:

* a dense brute force that builds P1 mass matrices by Gauss quadrature of hat
  functions, prolongations by evaluating coarse hats at fine nodes, and takes
  the L2 projection of the whole level function by a dense Kronecker solve;
* closed forms (1-D, 3 nodes) and the multilinear invariance (a multilinear
  field has no detail on any finer level);
* the Galerkin identity and the L2-orthogonality of the details;
* the identity recompose(decompose(u)) = u;
* dot-product and dense-transpose identities of both adjoints.
"""
import math

import numpy as np
import pytest

SHAPES_SMALL = [(2,), (3,), (4,), (5,), (6,), (17,), (3, 3), (5, 5), (6, 5), (3, 5, 4),
                (6, 5, 4), (9, 6, 5), (5, 9, 7)]


# ---------------------------------------------------------------------------
# Independent dense brute force

def _kept(m):
    return sorted(set(range(0, m, 2)) | {m - 1})


def _coords(n, L):
    """Coordinates of every level, finest (level L) first."""
    xs = [np.arange(n, dtype=float)]
    for _ in range(L):
        x = xs[-1]
        xs.append(x[_kept(len(x))])
    return xs


def _num_levels(shape):
    def cnt(n):
        c = 0
        while n > 2:
            n = len(_kept(n))
            c += 1
        return c
    return min(cnt(n) for n in shape)


def _hat(nodes, i, x):
    e = np.zeros(len(nodes))
    e[i] = 1.0
    return np.interp(x, nodes, e)


def _mass_quad(nodes):
    g = np.array([-1.0, 1.0]) / math.sqrt(3.0)
    pts, wts = [], []
    for a, b in zip(nodes[:-1], nodes[1:]):
        pts += list((a + b) / 2 + (b - a) / 2 * g)
        wts += [(b - a) / 2] * 2
    pts, wts = np.array(pts), np.array(wts)
    Phi = np.stack([_hat(nodes, i, pts) for i in range(len(nodes))])
    return (Phi * wts) @ Phi.T


def _prolong(fine, coarse):
    return np.stack([_hat(coarse, j, fine) for j in range(len(coarse))], axis=1)


def _kron(mats):
    out = np.ones((1, 1))
    for m in mats:
        out = np.kron(out, m)
    return out


def brute_decompose(u):
    shape = u.shape
    L = _num_levels(shape)
    xs = [_coords(n, L) for n in shape]
    v = u.reshape(-1).astype(float)
    details = []
    for lev in range(L):                     # lev = 0 is the finest pair
        fine = [x[lev] for x in xs]
        coarse = [x[lev + 1] for x in xs]
        P = _kron([_prolong(f, c) for f, c in zip(fine, coarse)])
        M = _kron([_mass_quad(f) for f in fine])
        sel = _kron([np.eye(len(f))[[list(f).index(c) for c in cc]] for f, cc in zip(fine, coarse)])
        vc = sel @ v
        detail = v - P @ vc
        kept = np.zeros(len(v), bool)
        kept[np.flatnonzero(sel.sum(axis=0))] = True
        details.append(detail[~kept])
        v = np.linalg.solve(P.T @ M @ P, P.T @ M @ v)   # L2 projection of the level function
    return np.concatenate([v] + details[::-1])


# ---------------------------------------------------------------------------

def test_level_counts(oracle):
    assert oracle.levels((513,))[0] == 9
    assert oracle.levels((129, 129))[0] == 7
    assert oracle.levels((513, 513, 513))[0] == 9
    L, m = oracle.levels((500, 500, 100))
    assert L == 7
    assert list(m[0]) == [5, 9, 17, 33, 64, 126, 251, 500]
    assert list(m[2]) == [2, 3, 5, 8, 14, 26, 51, 100]
    assert oracle.levels((2,))[0] == 0
    assert oracle.level_sizes((3,)) == [2, 3]


@pytest.mark.parametrize("shape", SHAPES_SMALL)
def test_matches_dense_l2_projection(oracle, shape):
    u = np.random.default_rng(len(shape) * 100 + sum(shape)).standard_normal(shape)
    ref = brute_decompose(u)
    got = oracle.decompose(u)
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_closed_form_three_nodes(oracle):
    u = np.array([0.3, 2.0, -1.1])
    mc = u[1] - (u[0] + u[2]) / 2
    # projecting a hat of height mc on [0,2] onto linear functions gives the constant mc/2
    ref = np.array([u[0] + mc / 2, u[2] + mc / 2, mc])
    assert np.allclose(oracle.decompose(u), ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("shape", [(17,), (9, 5), (6, 5, 4), (33, 17), (12, 7, 10), (100, 7)])
def test_multilinear_field_has_no_detail(oracle, shape):
    rng = np.random.default_rng(7)
    grids = np.meshgrid(*[np.arange(n, dtype=float) for n in shape], indexing="ij")
    f = rng.standard_normal() * np.ones(shape)
    for g in grids:
        f += rng.standard_normal() * g
    for i in range(len(shape)):
        for j in range(i + 1, len(shape)):
            f += rng.standard_normal() * grids[i] * grids[j]
    if len(shape) == 3:
        f += rng.standard_normal() * grids[0] * grids[1] * grids[2]
    c = oracle.decompose(f)
    N0 = oracle.level_sizes(shape)[0]
    assert np.abs(c[N0:]).max() <= 1e-10 * np.abs(f).max()
    L, m = oracle.levels(shape)
    idx = [np.array(_coords(n, L)[-1], dtype=int) for n in shape]
    assert np.allclose(c[:N0], f[np.ix_(*idx)].reshape(-1), rtol=0, atol=1e-10 * np.abs(f).max())


@pytest.mark.parametrize("n", [5, 6, 9, 10, 17, 31])
def test_galerkin_identity(n):
    x = np.arange(n, dtype=float)
    xc = x[_kept(n)]
    P = _prolong(x, xc)
    assert np.abs(P.T @ _mass_quad(x) @ P - _mass_quad(xc)).max() < 1e-13


@pytest.mark.parametrize("shape", [(9,), (5, 9), (3, 5, 9), (17, 9)])
def test_details_orthogonal_to_coarse_space(oracle, shape):
    """One level: P^T M_l (Q_l u - P Q_{l-1} u) = 0 with Q_{l-1}u from the oracle.

    Uniform sizes only: their coarse grid is itself a (scaled) hierarchy root,
    so recomposing the coarse part of the stream yields Q_{l-1}u."""
    u = np.random.default_rng(3).standard_normal(shape)
    L = _num_levels(shape)
    xs = [_coords(n, L) for n in shape]
    # oracle's level-(L-1) values: decompose then recompose all but the finest detail
    c = oracle.decompose(u)
    sizes = oracle.level_sizes(shape)
    # rebuild Q_{L-1}u by recomposing the coarse part on the level-(L-1) grid
    coarse_shape = tuple(len(x[1]) for x in xs)
    if L >= 1 and all(s >= 2 for s in coarse_shape) and _num_levels(coarse_shape) == L - 1:
        qc = oracle.recompose(c[:sizes[L - 1]], coarse_shape).reshape(-1)
    else:
        pytest.skip("coarse grid is not itself a hierarchy root")
    fine = [x[0] for x in xs]
    coarse = [x[1] for x in xs]
    P = _kron([_prolong(f, cc) for f, cc in zip(fine, coarse)])
    M = _kron([_mass_quad(f) for f in fine])
    r = P.T @ M @ (u.reshape(-1) - P @ qc)
    assert np.abs(r).max() < 1e-12 * np.abs(u).max()


@pytest.mark.parametrize("shape", [(2,), (3,), (6,), (33,), (9, 6, 5), (17, 33), (12, 7, 10),
                                   (65, 9), (100, 7, 5), (20, 20, 20)])
def test_identity(oracle, shape):
    u = np.random.default_rng(11).standard_normal(shape)
    r = oracle.recompose(oracle.decompose(u), shape)
    assert np.abs(r - u).max() <= 1e-12 * np.abs(u).max()


@pytest.mark.parametrize("shape", [(17,), (9, 6, 5), (33, 17), (12, 7, 10)])
def test_adjoint_dot_products(oracle, shape):
    rng = np.random.default_rng(5)
    N = int(np.prod(shape))
    c, g = rng.standard_normal(N), rng.standard_normal(N)
    u, h = rng.standard_normal(N), rng.standard_normal(N)
    Rc = oracle.recompose(c, shape).reshape(-1)
    RTg = oracle.recompose_adjoint(g.reshape(shape))
    assert abs(Rc @ g - c @ RTg) <= 1e-12 * np.abs(Rc).max() * np.abs(g).sum()
    Du = oracle.decompose(u.reshape(shape))
    DTh = oracle.decompose_adjoint(h, shape).reshape(-1)
    assert abs(Du @ h - u @ DTh) <= 1e-12 * np.abs(Du).max() * np.abs(h).sum()


@pytest.mark.parametrize("shape", [(6,), (5, 6), (3, 5, 4)])
def test_adjoints_are_dense_transposes(oracle, shape):
    N = int(np.prod(shape))
    E = np.eye(N)
    R = np.stack([oracle.recompose(E[i], shape).reshape(-1) for i in range(N)], axis=1)
    RT = np.stack([oracle.recompose_adjoint(E[i].reshape(shape)) for i in range(N)], axis=1)
    D = np.stack([oracle.decompose(E[i].reshape(shape)) for i in range(N)], axis=1)
    DT = np.stack([oracle.decompose_adjoint(E[i], shape).reshape(-1) for i in range(N)], axis=1)
    assert np.abs(RT - R.T).max() < 1e-12 * np.abs(R).max()
    assert np.abs(DT - D.T).max() < 1e-12 * np.abs(D).max()
    assert np.abs(R @ D - np.eye(N)).max() < 1e-12
    assert np.abs(DT @ RT - np.eye(N)).max() < 1e-12


def _dense_correction_norm(shape):
    L = _num_levels(shape)
    xs = [_coords(n, L) for n in shape]
    out = [0.0]
    for lev in range(L):
        prod = 1.0
        for x in xs:
            f, c = x[lev], x[lev + 1]
            G = np.linalg.solve(_mass_quad(c), _prolong(f, c).T @ _mass_quad(f))
            prod *= np.abs(G).sum(axis=1).max()
        out.append(prod)
    return np.array(out[:1] + out[1:][::-1])


@pytest.mark.parametrize("shape", [(3,), (3, 3, 3), (9, 6, 5), (17, 33), (100,)])
def test_correction_norms_dense(oracle, shape):
    assert np.allclose(oracle.correction_norms(shape), _dense_correction_norm(shape),
                       rtol=1e-12, atol=0)


def test_correction_norm_closed_forms(oracle):
    # three nodes: G = [[3/4, 1/2, -1/4], [-1/4, 1/2, 3/4]], row sums 3/2
    assert oracle.correction_norms((3,))[1] == pytest.approx(1.5, abs=1e-15)
    assert oracle.correction_norms((3, 3))[1] == pytest.approx(2.25, abs=1e-15)
    # long uniform lines: the row sum tends to 1 + sqrt(3)/2
    c = oracle.correction_norms((513, 513, 513))
    assert c[9] == pytest.approx((1 + math.sqrt(3) / 2) ** 3, rel=1e-12)
