"""Non-uniform grids (Sec. IV-A: MGARD reduces uniform and non-uniform grids)
on the GPU against the FP64 oracle given the same node coordinates.

Same tolerances as the unit-spacing parity tests: coefficients within
1e-5 x max|coef| (FP32 data) or 1e-12 (FP64); codes bit-exact when the oracle
quantizes the GPU's own coefficients with the container's bins; bins equal to
the oracle's up to rounding; every reconstruction within the bound."""
import numpy as np
import pytest
import torch
from _codes import assert_codes_match_fp64

pytestmark = pytest.mark.gpu

SHAPES = [(2,), (33,), (1000,), (6, 5), (129, 129), (300, 200), (65, 33), (9, 6, 5),
          (33, 17, 9), (70, 70, 70), (100, 60, 40)]


@pytest.fixture(scope="module")
def H():
    from paper_2503_06322_gb300 import hpdr
    return hpdr


def _inputs(shape, seed, dtype, kind="random"):
    from paper_2503_06322_gb300 import fields
    if len(shape) == 1:
        u = (np.random.default_rng(seed).standard_normal(shape) * 2 + 0.5).astype(dtype)
    else:
        u = fields.powerlaw_field(shape, seed=seed, dtype=dtype)
    return u, fields.node_coords(shape, seed + 100, kind)


@pytest.mark.parametrize("shape", SHAPES, ids=str)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_decompose_recompose_parity(oracle, H, shape, dtype):
    u, co = _inputs(shape, 1, dtype)
    ut = torch.from_numpy(u).cuda()
    got = H.hpdr_decompose(ut, coords=co).cpu().numpy().astype(np.float64)
    ref = oracle.decompose(u.astype(np.float64), coords=co)
    tol = 1e-5 if dtype == np.float32 else 1e-12
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    # unit spacing gives other coefficients (the coordinates are really used)
    if len(shape) > 1 or shape[0] > 2:
        assert np.abs(ref - oracle.decompose(u.astype(np.float64))).max() > 100 * tol * np.abs(ref).max()
    ct = torch.from_numpy(ref.astype(dtype)).cuda()
    rec = H.hpdr_recompose(ct, shape, coords=co).cpu().numpy().astype(np.float64)
    rref = oracle.recompose(ref.astype(dtype).astype(np.float64), shape, coords=co)
    assert np.abs(rec - rref).max() <= tol * np.abs(rref).max()
    back = H.hpdr_recompose(H.hpdr_decompose(ut, coords=co), shape, coords=co).cpu().numpy()
    assert np.abs(back.astype(np.float64) - u).max() <= tol * np.abs(u).max()


@pytest.mark.parametrize("shape", [(129, 129), (33, 17, 9), (65, 65, 65), (1000,)], ids=str)
def test_stretched_grid_parity(oracle, H, shape):
    u, co = _inputs(shape, 4, np.float64, kind="stretched")
    got = H.hpdr_decompose(torch.from_numpy(u).cuda(), coords=co).cpu().numpy()
    ref = oracle.decompose(u, coords=co)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("shape", [(65, 65), (17, 9, 33), (257,)], ids=str)
def test_multilinear_in_coordinates_has_no_fine_coefficients(H, shape):
    """A field multilinear in the node coordinates is reproduced by every
    coarser level's interpolant: all coefficients above level 0 vanish."""
    from paper_2503_06322_gb300 import fields
    co = fields.node_coords(shape, 5)
    grids = np.meshgrid(*co, indexing="ij")
    u = 1.0 + sum((k + 1) * 0.3 * g for k, g in enumerate(grids))
    if len(shape) >= 2:
        u = u + 0.05 * grids[0] * grids[1]
    c = H.hpdr_decompose(torch.from_numpy(u).cuda(), coords=co).cpu().numpy()
    L = 0
    m = list(shape)
    while min(m) > 2:
        m = [(x + 2) // 2 for x in m]
        L += 1
    n0 = int(np.prod(m))
    assert np.abs(c[n0:]).max() <= 1e-11 * np.abs(u).max()


@pytest.mark.parametrize("shape,tol", [((129, 129), 1e-3), ((33, 17, 9), 1e-2), ((70, 70, 70), 1e-4),
                                       ((1000,), 1e-3), ((300, 200), 1e-3)], ids=str)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_compress_codes_bins_and_cross_decoding(oracle, H, shape, tol, dtype):
    u, co = _inputs(shape, 3, dtype)
    ut = torch.from_numpy(u).cuda()
    buf = H.hpdr_compress(ut, tol, coords=co).cpu().numpy()
    h = oracle.parse_header(buf)
    assert h["has_coords"] and np.array_equal(h["coords"], np.concatenate(co))
    sym, esc = oracle.decode(h["words"], h["chunk"], h["N"], h["K"], h["lengths"], esc_width=h["esc_width"])
    coef = H.hpdr_decompose(ut, coords=co).cpu().numpy().astype(np.float64)
    assert_codes_match_fp64(oracle, sym, esc, coef, shape, h["q"], h["D"])
    eps = 2.0 ** -24 if dtype == np.float32 else 2.0 ** -53
    a = np.abs(u.astype(np.float64)).max()
    q_ref = oracle.bins(shape, tol * a, a, eps, coords=co)
    assert np.allclose(h["q"], q_ref, rtol=1e-12, atol=0)
    assert not np.allclose(q_ref, oracle.bins(shape, tol * a, a, eps), rtol=1e-6, atol=0)
    tau = tol * a
    # the oracle decodes the GPU container (coordinates carried in it) ...
    assert np.abs(oracle.decompress(buf) - u.astype(np.float64)).max() <= tau
    # ... the GPU decodes it ...
    rec = H.hpdr_decompress(torch.from_numpy(buf).cuda()).cpu().numpy().astype(np.float64)
    assert np.abs(rec - u).max() <= tau
    # ... and the GPU decodes the oracle's container of the same grid
    ob = oracle.compress(u, tol, coords=co)
    rec2 = H.hpdr_decompress(torch.from_numpy(np.asarray(ob)).cuda()).cpu().numpy().astype(np.float64)
    assert np.abs(rec2 - u).max() <= tau


def test_unit_spacing_coordinates_give_the_plain_container(H):
    from paper_2503_06322_gb300 import fields
    u = fields.powerlaw_field((65, 33), seed=6, dtype=np.float32)
    ut = torch.from_numpy(u).cuda()
    plain = H.hpdr_compress(ut, 1e-3).cpu().numpy()
    with_co = H.hpdr_compress(ut, 1e-3, coords=[np.arange(65.0), np.arange(33.0)]).cpu().numpy()
    # same codes and bitstream, the coordinate section and flag added
    assert (int.from_bytes(with_co[48:52].tobytes(), "little") & 0x100) and not \
        (int.from_bytes(plain[48:52].tobytes(), "little") & 0x100)
    assert with_co.size == plain.size + ((128 + 8 * 6 + 8 * 98 + 15) // 16 * 16 - (128 + 8 * 6 + 15) // 16 * 16)
    assert plain.size <= H.hpdr_compress_bound((65, 33))


def test_bad_coordinates_are_rejected(H):
    u = torch.zeros(5, 4, device="cuda")
    for co in ([np.arange(5.0), np.array([0.0, 1.0, 1.0, 2.0])],
               [np.arange(5.0), np.array([0.0, 1.0, np.inf, 2.0])],
               [np.arange(5.0)[::-1].copy(), np.arange(4.0)]):
        with pytest.raises(H.HpdrError) as e:
            H.hpdr_decompose(u, coords=co)
        assert e.value.status == -1
        with pytest.raises(H.HpdrError):
            H.hpdr_compress(u, 1e-3, coords=co)
    with pytest.raises(ValueError):
        H.hpdr_decompose(u, coords=[np.arange(5.0)])


@pytest.mark.parametrize("shape", [(33,), (65, 33), (17, 9, 33), (40, 30, 20)], ids=str)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_adjoints_parity(oracle, H, shape, dtype):
    """Both transposes on a non-uniform grid against the oracle's."""
    from paper_2503_06322_gb300 import fields
    co = fields.node_coords(shape, 31)
    rng = np.random.default_rng(32)
    g = rng.standard_normal(shape).astype(dtype)
    got = H.hpdr_recompose_adjoint(torch.from_numpy(g).cuda(), coords=co).cpu().numpy().astype(np.float64)
    ref = oracle.recompose_adjoint(g.astype(np.float64), coords=co)
    tol = 1e-5 if dtype == np.float32 else 1e-12
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    gc = rng.standard_normal(int(np.prod(shape))).astype(dtype)
    got = H.hpdr_decompose_adjoint(torch.from_numpy(gc).cuda(), shape, coords=co).cpu().numpy().astype(np.float64)
    ref = oracle.decompose_adjoint(gc.astype(np.float64), shape, coords=co)
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
