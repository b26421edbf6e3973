"""Pins of the oracle's statistical L2 bins (mode 2), CPU only.

The paper names an L2 mode but gives no bin formula; the reading (oracle
hierarchy.c) bounds the expected squared L2 error of the reconstruction by
sum_l (q_l^2 / 12) S_l, S_l = sum of the level-l mass-matrix diagonal over the
nodes new on level l, and splits the budget tau'^2 T (T = trace of the finest
mass matrix) evenly over the levels.  Pinned here:
  * S_l and T against hand values, closed forms and a quadrature-built mass
    matrix on random node coordinates;
  * the bound itself: uniform coefficient errors pushed through the oracle's
    recomposition (a linear map) give a mean squared L2 error, measured with
    the quadrature mass matrix, at most sum_l S_l q_l^2 / 12 per level and in
    total;
  * compression in mode 2: RMS error below tau on seeded fields, a smaller
    container than the max-norm bins, codes and bins recorded as stated.
"""
import math

import numpy as np
import pytest

import oracle


def _hat(nodes, i, x):
    e = np.zeros(len(nodes))
    e[i] = 1.0
    return np.interp(x, nodes, e)


def _mass_quad(nodes):
    # two-point Gauss rule per cell: exact for products of two linear pieces
    g = np.array([-1.0, 1.0]) / math.sqrt(3.0)
    pts, wts = [], []
    for a, b in zip(nodes[:-1], nodes[1:]):
        pts += list((a + b) / 2 + (b - a) / 2 * g)
        wts += [(b - a) / 2] * 2
    pts, wts = np.array(pts), np.array(wts)
    Phi = np.stack([_hat(nodes, i, pts) for i in range(len(nodes))])
    return (Phi * wts) @ Phi.T


def _kron(mats):
    out = np.ones((1, 1))
    for m in mats:
        out = np.kron(out, m)
    return out


def _coarsen(x):
    m = len(x)
    keep = [p for p in range(m) if p % 2 == 0 or p == m - 1]
    return x[keep], keep


def test_hand_values():
    S, T = oracle.l2s_weights((5,))
    # diag of the 5-node mass matrix: 1/3, 2/3, 2/3, 2/3, 1/3; new on level 2: nodes 1, 3;
    # level 1 (nodes 0, 2, 4): diag 2/3, 4/3, 2/3, new: node 2; level 0 (0, 4): 4/3, 4/3
    assert np.allclose(S, [8 / 3, 4 / 3, 4 / 3], rtol=1e-15) and math.isclose(T, 8 / 3, rel_tol=1e-15)
    S, T = oracle.l2s_weights((3, 3))
    # all but the four corners (1/3 * 1/3 each) are new on level 1
    assert np.allclose(S, [16 / 9, 16 / 9 - 4 / 9], rtol=1e-15) and math.isclose(T, 16 / 9, rel_tol=1e-15)


@pytest.mark.parametrize("shape", [(9, 9, 9), (17, 33), (65,), (33, 17, 9)], ids=str)
def test_uniform_dyadic_closed_form(shape):
    """Unit spacing, sizes 2^j + 1: T = prod (2/3)(n_k - 1); every level's new
    nodes carry T (1 - 2^-d) of it, level 0 all of it."""
    S, T = oracle.l2s_weights(shape)
    d = len(shape)
    T_ref = float(np.prod([(2.0 / 3.0) * (n - 1) for n in shape]))
    assert math.isclose(T, T_ref, rel_tol=1e-13)
    assert math.isclose(S[0], T_ref, rel_tol=1e-13)
    assert np.allclose(S[1:], T_ref * (1 - 2.0 ** -d), rtol=1e-13)


@pytest.mark.parametrize("shape", [(7, 6), (5, 4, 6), (12,)], ids=str)
def test_against_quadrature_mass_matrix(shape):
    """S_l from the diagonal of a Kronecker product of quadrature-built 1-D
    mass matrices on random coordinates, level by level."""
    rng = np.random.default_rng(sum(shape))
    co = [np.cumsum(rng.uniform(0.2, 3.0, size=n)) for n in shape]
    S, T = oracle.l2s_weights(shape, coords=co)
    L = len(S) - 1
    xs = [list(co)]
    for _ in range(L):
        xs.append([_coarsen(x)[0] for x in xs[-1]])
    xs = xs[::-1]                      # xs[l][k]: coordinates of dim k on level l
    for l in range(L + 1):
        diag = np.diag(_kron([_mass_quad(x) for x in xs[l]]))
        if l == 0:
            ref = diag.sum()
        else:
            kept = [np.zeros(len(x), bool) for x in xs[l]]
            for k, x in enumerate(xs[l]):
                kept[k][_coarsen(x)[1]] = True
            kk = kept[0]
            for k in range(1, len(shape)):
                kk = np.logical_and.outer(kk, kept[k]).reshape(-1)
            ref = diag[~kk].sum()
        assert math.isclose(S[l], ref, rel_tol=1e-12), (l, S[l], ref)
    assert math.isclose(T, np.diag(_kron([_mass_quad(x) for x in co])).sum(), rel_tol=1e-12)


@pytest.mark.parametrize("shape,coords", [((17, 17), False), ((9, 9, 9), False), ((33,), True), ((12, 10), True)],
                         ids=str)
def test_expected_error_bound(shape, coords):
    """Uniform errors of width q_l on level l's stream entries, recomposed:
    the mean squared L2 error stays below sum_l S_l q_l^2 / 12 (each level
    alone and all together), and within a factor of it."""
    rng = np.random.default_rng(3)
    co = [np.cumsum(rng.uniform(0.3, 2.5, size=n)) for n in shape] if coords else None
    S, T = oracle.l2s_weights(shape, coords=co)
    L = len(S) - 1
    Nl = oracle.level_sizes(shape)
    M = _kron([_mass_quad(c if coords else np.arange(n, dtype=float)) for c, n in
               zip(co if coords else [None] * len(shape), shape)])
    q = rng.uniform(0.5, 2.0, size=L + 1)
    trials = 400

    def mean_sq(levels):
        acc = 0.0
        for _ in range(trials):
            c = np.zeros(int(np.prod(shape)))
            for l in levels:
                a = 0 if l == 0 else Nl[l - 1]
                c[a:Nl[l]] = rng.uniform(-q[l] / 2, q[l] / 2, size=Nl[l] - a)
            e = oracle.recompose(c, shape, coords=co).reshape(-1)
            acc += e @ M @ e
        return acc / trials

    pred = S * q ** 2 / 12
    for l in (0, L):
        got = mean_sq([l])
        assert got <= 1.1 * pred[l], (l, got, pred[l])
    got = mean_sq(range(L + 1))
    assert 0.2 * pred.sum() <= got <= 1.1 * pred.sum(), (got, pred.sum())


@pytest.mark.parametrize("shape,tol", [((65, 65), 1e-3), ((33, 17, 9), 1e-2), ((1000,), 1e-3),
                                       ((40, 30, 20), 1e-3)], ids=str)
def test_compression_in_statistical_l2_mode(shape, tol):
    from paper_2503_06322_gb300 import fields
    u = fields.powerlaw_field(shape, seed=8, dtype=np.float64) if len(shape) > 1 else \
        np.random.default_rng(8).standard_normal(shape)
    b2 = oracle.compress(u, tol, mode=oracle.L2_STAT)
    h = oracle.parse_header(b2)
    assert h["mode"] == 2
    rms = math.sqrt(float(np.mean(u * u)))
    tau = tol * rms
    assert math.isclose(h["tau_abs"], tau, rel_tol=1e-12)
    assert np.allclose(h["q"], oracle.bins_l2s(shape, tau, np.abs(u).max(), 2.0 ** -53), rtol=1e-15)
    err = oracle.decompress(b2) - u
    e_rms = math.sqrt(float(np.mean(err * err)))
    assert 0.05 * tau <= e_rms <= tau, (e_rms, tau)
    b1 = oracle.compress(u, tol, mode=oracle.L2)
    assert b2.size < b1.size
    # the max-norm L2 mode bounds the maximum error instead
    assert np.abs(oracle.decompress(b1) - u).max() <= tau


def test_zero_field_and_floor():
    z = np.zeros((9, 9))
    b = oracle.compress(z, 1e-3, mode=oracle.L2_STAT)
    assert np.array_equal(oracle.decompress(b), z)
    assert np.all(oracle.parse_header(b)["q"] == 1.0)
    with pytest.raises(Exception):
        oracle.bins_l2s((9, 9), 1e-20, 1.0, 2.0 ** -24)
