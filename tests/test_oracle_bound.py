"""The max-norm guarantee of the bins, pinned by brute force (CPU only).

Quantization leaves every coefficient of level l within q_l / 2 of its true
value, and the reconstruction error is R delta, R the (linear) recomposition.
The worst case over all such delta at output node i is
    sum_j |R_ij| q_{l(j)} / 2,
so the bins of Sec. IV-A (as read here: q_0 = 2 tau' / (L+1),
q_l = 2 tau' / ((L+1)(1 + c_l))) guarantee max |u - u~| <= tau' exactly when
that sum stays below tau' for every i.  R is built column by column from the
oracle's recomposition on small grids (uniform, non-dyadic and non-uniform),
so the check covers the interpolation, the correction and the norms c_l
together, with nothing assumed about them."""
import numpy as np
import pytest

import oracle


def _worst_case(shape, coords):
    N = int(np.prod(shape))
    R = np.stack([oracle.recompose(np.eye(N)[j], shape, coords=coords).reshape(-1) for j in range(N)], axis=1)
    q = oracle.bins(shape, 1.0, 1.0, 0.0, coords=coords)      # tau' = tau = 1
    Nl = oracle.level_sizes(shape)
    lev = np.zeros(N, dtype=int)
    for l in range(1, len(Nl)):
        lev[Nl[l - 1]:Nl[l]] = l
    return float(np.max(np.abs(R) @ (q[lev] / 2.0)))


@pytest.mark.parametrize("shape", [(9,), (17,), (12,), (33,), (7, 6), (9, 9), (10, 7), (5, 4, 6), (9, 5, 3)],
                         ids=str)
@pytest.mark.parametrize("nonuniform", [False, True])
def test_worst_case_error_within_tau(shape, nonuniform):
    rng = np.random.default_rng(sum(shape) + nonuniform)
    co = [np.cumsum(rng.uniform(0.3, 2.5, size=n)) for n in shape] if nonuniform else None
    w = _worst_case(shape, co)
    assert w <= 1.0 + 1e-12, w
    # and the bound is not vacuous: the worst case uses a fair share of it
    assert w >= 0.2, w
