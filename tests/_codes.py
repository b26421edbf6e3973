"""Shared check of quantization codes against the oracle.

The kernels take the quantization decision k = sign(x) floor(|x| rho + 1/2)
with binary64 semantics (Sec. IV-A's linear quantization; for FP32 data in
binary32 arithmetic on a double-word product).  On the GPU's own coefficients
the codes must agree with the oracle's binary64 decision everywhere except at
half-bin ties -- at most 1e-5 of the elements, each a neighbouring code with
|x| / q within 2^-40 |x| / q of a half-integer.
"""
import numpy as np


def codes_of(sym, esc, D):
    k = sym.astype(np.int64) - D // 2
    k[sym == 0] = esc
    return k


def assert_codes_match_fp64(oracle, sym, esc, coef, shape, q, D):
    k_gpu = codes_of(sym, esc, D)
    ref_sym, ref_idx, ref_k = oracle.quantize(coef, shape, q, D=D, precision=64)
    k_ref = ref_sym.astype(np.int64) - D // 2
    k_ref[ref_idx] = ref_k
    bad = np.flatnonzero(k_gpu != k_ref)
    assert bad.size <= 1e-5 * coef.size, bad.size
    if bad.size:
        sizes = np.asarray(oracle.level_sizes(shape))
        lev = np.searchsorted(sizes, bad, side="right")
        t = np.abs(coef[bad]) / np.asarray(q)[lev]
        assert np.all(np.abs(k_gpu[bad] - k_ref[bad]) == 1)
        assert np.all(np.abs(t - (np.floor(t) + 0.5)) <= 2.0 ** -40 * np.maximum(t, 1.0))
    return bad.size
