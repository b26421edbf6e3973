"""Pins of the oracle on non-uniform node coordinates (MGARD's non-uniform
grids; Sec. IV-A's decomposition on piecewise-linear spaces), by properties
that fix the coordinates' role independently of the oracle's operators:

  * a field linear in the coordinates is reproduced exactly by the
    interpolant, so every coefficient above level 0 vanishes;
  * the correction is the L2 projection onto nested P1 spaces, so the level-0
    values are the L2 projection of the finest piecewise-linear function onto
    the coarsest space (computed here with a Gram matrix and Simpson's rule,
    exact for these products);
  * coefficients are invariant under affine coordinate maps x -> a + h x;
  * recomposition inverts decomposition, and containers carry the coordinates.
"""
import numpy as np
import pytest

import oracle


def _rand_coords(rng, shape):
    return [np.cumsum(rng.uniform(0.3, 2.5, size=n)) for n in shape]


def _kept_chain(n, L=None):
    """Finest-grid indices of the level-0 nodes: every level keeps its even
    positions and its last node, L times (default: until two nodes remain;
    all dimensions coarsen together, L times)."""
    idx = np.arange(n)
    while (idx.size > 2) if L is None else (L > 0):
        L = None if L is None else L - 1
        m = idx.size
        keep = [p for p in range(m) if p % 2 == 0 or p == m - 1]
        idx = idx[keep]
    return idx


def _project_1d(x, v, X):
    """L2 projection of the P1 function (x, v) onto the P1 hats on nodes X
    (a subset of x): Gram matrix and right-hand side by Simpson's rule on the
    fine elements, where every integrand is a product of two linear pieces."""
    def hat(j, t):
        y = np.zeros_like(t)
        if j > 0:
            a, b = X[j - 1], X[j]
            s = (t >= a) & (t <= b)
            y[s] = (t[s] - a) / (b - a)
        if j + 1 < len(X):
            a, b = X[j], X[j + 1]
            s = (t >= a) & (t <= b)
            y[s] = np.maximum(y[s], (b - t[s]) / (b - a))
        if j == 0:
            y[t == X[0]] = 1.0
        return y
    nc = len(X)
    G = np.zeros((nc, nc))
    r = np.zeros(nc)
    for k in range(len(x) - 1):
        t = np.array([x[k], 0.5 * (x[k] + x[k + 1]), x[k + 1]])
        w = (x[k + 1] - x[k]) / 6.0 * np.array([1.0, 4.0, 1.0])
        f = np.interp(t, x, v)
        H = np.array([hat(j, t) for j in range(nc)])
        G += (H * w) @ H.T
        r += H @ (w * f)
    return np.linalg.solve(G, r)


@pytest.mark.parametrize("shape", [(9,), (10,), (33,), (17, 6), (9, 5, 7)], ids=str)
def test_linear_field_has_no_coefficients_above_level_0(shape):
    rng = np.random.default_rng(len(shape) * 100 + shape[0])
    co = _rand_coords(rng, shape)
    X = np.meshgrid(*co, indexing="ij")
    u = 0.5 + sum((k + 1.5) * X[k] for k in range(len(shape)))
    c = oracle.decompose(u, coords=co)
    n0 = oracle.level_sizes(shape)[0]
    assert np.abs(c[n0:]).max() <= 1e-12 * np.abs(u).max()
    # ... and the same field on unit spacing (not linear in these coordinates' map) does not
    v = 0.5 + sum((k + 1.5) * np.cumsum(co[k]).reshape([-1 if j == k else 1 for j in range(len(shape))])
                  for k in range(len(shape)))
    assert np.abs(oracle.decompose(v, coords=co)[n0:]).max() > 1e-6


@pytest.mark.parametrize("n", [3, 9, 10, 23], ids=str)
def test_level_0_is_the_l2_projection_1d(n):
    rng = np.random.default_rng(n)
    x = np.cumsum(rng.uniform(0.2, 3.0, size=n))
    v = rng.standard_normal(n)
    c = oracle.decompose(v, coords=[x])
    X = x[_kept_chain(n)]
    ref = _project_1d(x, v, X)
    assert np.allclose(c[:X.size], ref, rtol=0, atol=1e-11 * np.abs(v).max())


def test_level_0_is_the_l2_projection_2d():
    rng = np.random.default_rng(7)
    shape = (11, 6)
    co = _rand_coords(rng, shape)
    v = rng.standard_normal(shape)
    c = oracle.decompose(v, coords=co)
    # the projection onto a tensor-product space is the tensor product of the 1-D projections
    L, _ = oracle.levels(shape)
    k0, k1 = _kept_chain(shape[0], L), _kept_chain(shape[1], L)
    t = np.stack([_project_1d(co[0], v[:, j], co[0][k0]) for j in range(shape[1])], axis=1)
    ref = np.stack([_project_1d(co[1], t[i, :], co[1][k1]) for i in range(t.shape[0])], axis=0)
    assert np.allclose(c[:ref.size], ref.reshape(-1), rtol=0, atol=1e-11 * np.abs(v).max())


@pytest.mark.parametrize("shape", [(33,), (17, 9), (9, 10, 6)], ids=str)
def test_affine_coordinates_equal_unit_spacing(shape):
    rng = np.random.default_rng(3)
    v = rng.standard_normal(shape)
    co = [-4.0 + 0.37 * (k + 1) * np.arange(n) for k, n in enumerate(shape)]
    a, b = oracle.decompose(v, coords=co), oracle.decompose(v)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    assert np.allclose(oracle.correction_norms(shape, coords=co), oracle.correction_norms(shape),
                       rtol=1e-12, atol=0)


@pytest.mark.parametrize("shape", [(40,), (17, 9), (9, 10, 6)], ids=str)
def test_round_trip_and_container(shape):
    rng = np.random.default_rng(11)
    co = _rand_coords(rng, shape)
    u = rng.standard_normal(shape)
    c = oracle.decompose(u, coords=co)
    assert np.abs(oracle.recompose(c, shape, coords=co) - u).max() <= 1e-12 * np.abs(u).max()
    buf = oracle.compress(u, 1e-3, coords=co)
    h = oracle.parse_header(buf)
    assert h["has_coords"] and np.array_equal(h["coords"], np.concatenate(co))
    assert np.abs(oracle.decompress(buf) - u).max() <= 1e-3 * np.abs(u).max()
    # the bins follow the coordinates' correction norms
    eps = 2.0 ** -53
    assert np.allclose(h["q"], oracle.bins(shape, 1e-3 * np.abs(u).max(), np.abs(u).max(), eps, coords=co),
                       rtol=1e-15, atol=0)
    # containers without coordinates are unchanged
    assert not oracle.parse_header(oracle.compress(u, 1e-3))["has_coords"]


def test_rejects_bad_coordinates():
    u = np.zeros((5, 4))
    with pytest.raises(Exception):
        oracle.decompose(u, coords=[np.arange(5.0), np.array([0.0, 1.0, 1.0, 2.0])])
    with pytest.raises(Exception):
        oracle.decompose(u, coords=[np.arange(5.0), np.array([0.0, 1.0, np.nan, 2.0])])
    with pytest.raises(ValueError):
        oracle.decompose(u, coords=[np.arange(5.0)])


@pytest.mark.parametrize("shape", [(9,), (7, 6), (5, 4, 6), (17, 9)], ids=str)
def test_adjoints_with_coordinates(shape):
    """The transposes on a non-uniform grid: dot-product identities against
    the coordinate recomposition and decomposition, and the explicit
    transpose of the recomposition matrix on small grids."""
    rng = np.random.default_rng(len(shape) * 7 + shape[0])
    co = _rand_coords(rng, shape)
    N = int(np.prod(shape))
    c, g = rng.standard_normal(N), rng.standard_normal(shape)
    lhs = float(np.sum(oracle.recompose(c, shape, coords=co) * g))
    rhs = float(np.dot(c, oracle.recompose_adjoint(g, coords=co)))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))
    u, gc = rng.standard_normal(shape), rng.standard_normal(N)
    lhs = float(np.dot(oracle.decompose(u, coords=co), gc))
    rhs = float(np.sum(u * oracle.decompose_adjoint(gc, shape, coords=co)))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))
    if N <= 200:
        R = np.stack([oracle.recompose(np.eye(N)[i], shape, coords=co).reshape(-1) for i in range(N)], axis=1)
        Rt = np.stack([oracle.recompose_adjoint(np.eye(N)[i].reshape(shape), coords=co) for i in range(N)], axis=1)
        assert np.allclose(Rt, R.T, atol=1e-12)
    # unit spacing given explicitly is the plain transpose
    unit = [np.arange(n, dtype=float) for n in shape]
    assert np.allclose(oracle.recompose_adjoint(g, coords=unit), oracle.recompose_adjoint(g), atol=1e-13)
