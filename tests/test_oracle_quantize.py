"""Pins of the oracle's linear quantization (Sec. IV-A: level-scaled linear
quantization of the multilevel coefficients; reading R5 of the design notes:
k = sign(x) floor(|x| rho + 1/2), rho = 1/q, symbol D/2 + k).

Every GPU code-parity test checks the kernels' codes against
oracle.quantize, so the oracle's decision is fixed here by values worked out
by hand from that definition, independently of the oracle's code:

  * the binary32 decision (FP32 fields): rho, |x| rho and the + 1/2 each
    rounded to binary32, round to nearest even.  Each fixture below differs
    from at least one plausible mistake (rho kept in binary64, the product or
    the + 1/2 left in binary64, the whole decision in binary64);
  * exact ties x = (k + 1/2) q with q a power of two round away from zero;
  * the level of every stream index: levels are stored coarsest first, level
    l at [N_{l-1}, N_l), and each index is quantized with its own q_l.
"""
import numpy as np
import pytest

D = 8192


def _q1(oracle, x, q, precision):
    """Code of a single coefficient, decided by the oracle (1-D field of 2
    nodes: both are level 0, so both use q[0])."""
    sym, idx, k = oracle.quantize(np.array([x, x]), (2,), np.array([q]), D=D, precision=precision)
    assert idx.size == 0
    return int(sym[0]) - D // 2


# (x, q, k in binary32, k in binary64).  Derivations (u = 2^-24):
#  A. x = 1/2 - u/2, q = 1: rho = 1, y = x; y + 1/2 = 1 - u/2 is halfway
#     between 1 - u and 1 in binary32 and rounds to the even 1 -> k = 1.
#     In binary64 the sum is exact, floor 0.  (Catches "+ 1/2 in binary64".)
#  B. x = 0x3e199999 = 0.149999991059..., q = 0.3: rho = fl32(1/0.3) =
#     0x40555555 = 3.33333325386 (the 24-bit significand rounds down);
#     |x| rho = 0.4999999582... lies 1.4 ulp (ulp 2^-25) below 1/2 and rounds
#     to 1/2 - 2^-25; adding 1/2 gives 1 - u/2, a tie that rounds to 1 ->
#     k = 1.  Unrounded, the product plus 1/2 = 0.99999995828 rounds to 1 - u
#     -> 0 (catches "product in binary64"); in binary64 throughout -> 0.
#  C. x = 0x43d37fff = 422.99996948..., q = 6: rho = fl32(1/6) = 0x3e2aaaab =
#     0.166666671634 (rounds up); |x| rho = 70.4999970 is 3.0e-6 below 70.5,
#     within half an ulp (ulp 2^-17 = 7.6e-6), so it rounds to 70.5 and
#     70.5 + 1/2 = 71 -> k = 71.  With rho in binary64 (1/6), |x| rho =
#     70.4999949 rounds to 70.5 - 2^-17 and the sum stays below 71 -> 70
#     (catches "rho in binary64"); binary64 throughout -> 70.
#  D. x = 0x3eb58106 = 0.354499995708..., q = 0.001: 1/q rounds to 1000 in
#     both precisions; |x| rho = 354.499995708 rounds in binary32 (ulp 2^-15
#     = 3.05e-5) to 354.5, so t = 355 -> k = 355; in binary64 the product
#     stays 354.4999957 and t = 354.9999957 -> 354.
FIXTURES = [
    (0.5 - 2.0 ** -25, 1.0, 1, 0),
    (np.frombuffer(np.uint32(0x3E199999).tobytes(), np.float32)[0], 0.3, 1, 0),
    (np.frombuffer(np.uint32(0x43D37FFF).tobytes(), np.float32)[0], 6.0, 71, 70),
    (np.frombuffer(np.uint32(0x3EB58106).tobytes(), np.float32)[0], 0.001, 355, 354),
]


@pytest.mark.parametrize("x,q,k32,k64", FIXTURES, ids=["A_half_tie", "B_product", "C_rho", "D_binary64"])
def test_binary32_decision_hand_values(oracle, x, q, k32, k64):
    x = float(x)
    assert _q1(oracle, x, q, 32) == k32
    assert _q1(oracle, -x, q, 32) == -k32
    assert _q1(oracle, x, q, 64) == k64
    assert _q1(oracle, -x, q, 64) == -k64


# exact ties (k + 1/2) q with q = 1/4: both precisions round away from zero
# (round-half-even would give 0, 2, -2, 4, 12, -18 instead)
TIES = [(0.125, 1), (0.625, 3), (-0.625, -3), (1.125, 5), (-0.125, -1), (2.875, 12), (-4.625, -19)]


@pytest.mark.parametrize("precision", [32, 64])
def test_ties_round_away_from_zero(oracle, precision):
    for x, k in TIES:
        assert _q1(oracle, x, 0.25, precision) == k, (x, precision)


def test_zero_and_escapes(oracle):
    """Zero codes to D/2; |k| >= D/2 escapes (symbol 0) with its exact k."""
    q = np.array([0.5])
    x = np.array([0.0, -0.0, 0.24, 0.25, 4095.4 * 0.5, 4096.0 * 0.5, -4096.0 * 0.5, 1e6])
    n = x.size
    for i in range(n):
        sym, idx, k = oracle.quantize(np.array([x[i], x[i]]), (2,), q, D=D, precision=64)
        want = [0, 0, 0, 1, 4095, 4096, -4096, 2000000][i]
        if abs(want) < D // 2:
            assert idx.size == 0 and int(sym[0]) == D // 2 + want
        else:
            assert list(idx) == [0, 1] and list(k) == [want, want] and sym[0] == 0


@pytest.mark.parametrize("shape,sizes", [((9,), [2, 3, 5, 9]), ((5, 9), [6, 15, 45]),
                                         ((5, 5, 5), [8, 27, 125]), ((17, 9), [6, 15, 45, 153])],
                         ids=str)
@pytest.mark.parametrize("precision", [32, 64])
def test_level_of_every_stream_index(oracle, shape, sizes, precision):
    """Levels are stored coarsest first: level l holds stream indices
    [N_{l-1}, N_l).  With q_l = 10^l and coefficients (l + 3 + 1/4) q_l,
    every index must code to l + 3; an index quantized with a neighbouring
    level's bin would code to (l + 3.25) 10^{+-1} rounded instead."""
    assert list(oracle.level_sizes(shape)) == sizes
    L = len(sizes) - 1
    q = np.array([10.0 ** l for l in range(L + 1)])
    lev = np.zeros(sizes[-1], dtype=int)
    for l in range(1, L + 1):
        lev[sizes[l - 1]:sizes[l]] = l
    coef = (lev + 3.25) * q[lev]
    sym, idx, k = oracle.quantize(coef, shape, q, D=D, precision=precision)
    assert idx.size == 0
    assert np.array_equal(sym.astype(int) - D // 2, lev + 3)
